// Tensor-memory-accelerator (TMA) plumbing for the z-marching kernels: tensor maps over the field
// arrays, and the inline-PTX wrappers for mbarriers and tiled bulk tensor loads (sm_90 and later;
// built here for sm_103a).
//
// A field map describes `ncomp` consecutive arrays of a field buffer (components c = 0..ncomp-1, each
// [nz][ny][nxp] float32 with pitch nxp and component stride vol) as a 4-d tensor (x, y, z, c) with the
// logical extent (nx, ny, nz, ncomp): everything outside it, including the pitch padding x >= nx and
// negative coordinates, reads as 0, which is the value the PEC walls give the tangential fields.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "fdtd_internal.cuh"

namespace fdtd {

// Boxes the maps are encoded with; the kernels that use them rely on exactly these shapes.
struct MapBox {
  int w, h;  // x and y extent of one box (z extent 1, all components)
};

// Encode a field map (see above). Returns FDTD_OK or an FDTD_ERR_* code (with fdtd_last_error set).
int encode_field_map(CUtensorMap* m, const float* base, const Geo& g, int ncomp, MapBox box);

// The maps one forward step reads: E (3 components) and H (3) of the `cur` buffer, and a.
struct FwdMaps {
  CUtensorMap e, h, a;
};

// Box shapes of the forward kernel's maps, and its one-time set-up (dynamic shared memory limit).
MapBox fwd_box_e();
MapBox fwd_box_h();
MapBox fwd_box_a();
int prepare_fwd_fused(int nstage, int* blocks_per_sm);
void launch_fwd_fused(const FwdArgs& a, const FwdMaps& m, cudaStream_t s);

// The maps the reverse-step kernels read (F = fields, B = adjoint fields): "own" boxes cover the
// TX x TY tile, "high" boxes the tile plus one cell at +x and +y, "low" boxes the tile plus one cell
// at -x and -y (origin 4 cells left of the tile).
struct RevMaps {
  CUtensorMap e_own, e_high, h_own, h_low, eb_own, eb_high, hb_own, hb_low, a_high;
};

MapBox rev_box_own();
MapBox rev_box_wide();
int prepare_rev(int nstage, int* blocks_per_sm);
void launch_rev_E(const RevArgs& a, const RevMaps& m, cudaStream_t s);
void launch_rev_H(const RevArgs& a, const RevMaps& m, cudaStream_t s);

// The maps the fused inverse step reads (fdtd_inverse.cu): E^{n+1} and a over the tile plus the high
// halo, H^{n+1/2} over the tile plus both halos.
struct InvMaps {
  CUtensorMap e, h, a;
};
MapBox inv_box_e();   // E^{n+1} and a
MapBox inv_box_h();   // H^{n+1/2}
int prepare_inv(int nstage, int* blocks_per_sm);
int inv_max_tz();
void launch_inv(const InvArgs& a, const InvMaps& m, cudaStream_t s);

// The maps the fused adjoint step reads (fdtd_adjoint.cu): Ebar and a over the tile with both halos,
// Hbar over the tile with the low halo, all from the adjoint buffer being read.
struct AdjMaps {
  CUtensorMap eb, hb, a;
};
MapBox adj_box_e();   // Ebar and a
MapBox adj_box_h();   // Hbar
int prepare_adj(int nstage, int* blocks_per_sm);
int adj_max_tz();
// returns the launches made; s2 (with the events fork and join), if not null: the stream on which a
// split step's frame launch runs beside its plain launch on s
int launch_adj(const AdjArgs& a, const AdjMaps& m, cudaStream_t s, cudaStream_t s2 = nullptr,
               cudaEvent_t fork = nullptr, cudaEvent_t join = nullptr);
int adj_tiles_x(const Geo& g);                    // tile columns and rows of the adjoint step
int adj_tiles_y(const Geo& g);
bool adj_tile_xy(const Geo& g, int axis, int b);  // column (axis 0) / row (axis 1) b needs the x/y CPML loop

// ---- grouped launches: several requests (solver handles) advanced by one launch -------------------
constexpr int kMaxGroup = 8;

// The flat grid of a grouped launch: request r owns blocks blk0[r] .. blk0[r + 1] - 1, laid out as its
// own grid would be (tile x fastest, then tile y, then the z-chunk).
struct GroupGrid {
  int n;
  int blk0[kMaxGroup + 1];
  int nbx[kMaxGroup], nby[kMaxGroup];
};

// Fill G's prefix from each request's grid (nb: tiles along x and y, z-chunks); returns the total.
template <class F>
inline int group_fill(GroupGrid& G, int n, F grid_of) {
  G.n = n;
  G.blk0[0] = 0;
  for (int r = 0; r < n; ++r) {
    int nb[3];
    grid_of(r, nb);
    G.nbx[r] = nb[0];
    G.nby[r] = nb[1];
    G.blk0[r + 1] = G.blk0[r] + nb[0] * nb[1] * nb[2];
  }
  return G.blk0[n];
}

struct FwdGroup {
  GroupGrid grid;
  int n;
  FwdArgs a[kMaxGroup];
  FwdMaps m[kMaxGroup];
};
struct InvGroup {
  GroupGrid grid;
  int n;
  InvArgs a[kMaxGroup];
  InvMaps m[kMaxGroup];
};
struct AdjGroup {
  GroupGrid grid;
  int n;
  AdjArgs a[kMaxGroup];
  AdjMaps m[kMaxGroup];
};
struct RevGroup {
  GroupGrid grid;
  int n;
  RevArgs a[kMaxGroup];
  RevMaps m[kMaxGroup];
};
// which = 0: the inverse-E / adjoint-H kernel, 1: the inverse-H / adjoint-E kernel
void launch_rev_group(RevGroup& G, int which, cudaStream_t s);
// One launch per kernel for the G.n requests (their nstage must agree; a[r].tz sets each grid).
void launch_fwd_group(FwdGroup& G, cudaStream_t s);
void launch_inv_group(InvGroup& G, cudaStream_t s);
void launch_adj_group(AdjGroup& G, cudaStream_t s);

#if defined(__CUDACC__)

// The request of this block in a grouped launch, and the block's tile and z-chunk within it.
__device__ __forceinline__ int group_locate(const GroupGrid& G, int& bx, int& by, int& bz) {
  const int b = blockIdx.x;
  int r = 0;
  while (r + 1 < G.n && b >= G.blk0[r + 1]) ++r;
  const int local = b - G.blk0[r];
  const int nbx = G.nbx[r], nby = G.nby[r];
  bx = local % nbx;
  by = (local / nbx) % nby;
  bz = local / (nbx * nby);
  return r;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the barrier initialisation visible to the async proxy (the TMA unit) before first use.
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's earlier generic-proxy accesses to shared memory before later async-proxy ones.
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One arrival that also announces `bytes` of transactions the next phase waits for.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete; false if it gave up (the caller
// records a timeout status and carries on, so the block's barriers stay matched). It gives up after
// limit_ns nanoseconds of the global timer (read every 64 polls, from the first poll that fails) or
// kWaitLimit polls (a backstop far beyond the time limit), whichever comes first; a TMA copy of a
// plane lands within microseconds.
constexpr int kWaitLimit = 1 << 30;
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  uint64_t t0 = 0;
  for (int it = 0; it < kWaitLimit; ++it) {
    if (mbar_test(bar, parity)) return true;
    if ((it & 63) == 0) {
      const uint64_t t = global_ns();
      if (it == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
  return false;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) { return mbar_wait_for(bar, parity, kWaitNs); }

// Tiled 4-d bulk tensor load of one box at (x, y, z, c) into shared memory, completing on `bar`.
// x * 4 bytes must be a multiple of 16 (x a multiple of 4); the destination 128-byte aligned.
__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* map, int x, int y, int z, int c,
                                             uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(c), "r"(smem_addr(bar))
      : "memory");
}

#endif  // __CUDACC__

}  // namespace fdtd
