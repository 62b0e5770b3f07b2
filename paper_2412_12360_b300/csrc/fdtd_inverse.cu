// Fused inverse step of arXiv 2412.12360 Sec. 2.2: the E and H updates of one time step undone in a
// single sweep over the grid on the PML-free region R, with dL/da accumulated on the design box.
//
//   E^n     = E^{n+1} - src - S a curl_b(H^{n+1/2})     (the E update of Eq. 2 solved for E^n)
//   H^{n-1/2} = H^{n+1/2} + S curl_f(E^n)               (the H update of Eq. 1 solved for H^{n-1/2})
//   dL/da  += S Ebar^{n+1} . curl_b(H^{n+1/2})          on the design cells (FP64)
//
// The sweep reads buffer `cur` (E^{n+1}, and H^{n+1/2} with the recorded boundary faces written back
// just outside R) and writes buffer `nxt`, so neighbouring tiles never see half-updated fields.
// It is the mirror image of the forward sweep: a block owns a TX x TY column tile and marches its
// z-chunk DOWNWARDS; per plane it computes E^n for its cells and, redundantly, for the column
// x = i0 + TX and the row y = j0 + TY that its H update reads, then H^{n-1/2} from E^n of this plane
// and of the plane above (kept in registers from the previous plane). The chunk's top plane needs
// E^n of the plane above the chunk, which the block recomputes first. Planes arrive through a TMA
// ring as in the forward kernel (E^{n+1} with the high halo, H^{n+1/2} with both halos, a with the
// high halo). Every own cell of `nxt` is written (E^n, H^{n-1/2} on R; the old values elsewhere), so
// every store is a full row segment. Each thread updates two x-adjacent cells.
//
// Inside R the CPML terms vanish (1/kappa = 1, c = 0 and psi = 0, exactly), so the update is the plain
// Yee formula. E^n of a cell is computed by one function, whether for the block's own cells or for the
// halo of a neighbouring tile, so both give the same bits and the result does not depend on the
// z-chunk or the tile a cell falls in.
#include "../../include/fdtd.h"
#include "fdtd_internal.cuh"
#include "fdtd_tma.cuh"

namespace fdtd {

namespace {

constexpr int TX = 32, TY = 16, NT = 256;
constexpr int LX = TX / 2;  // threads per tile row (two cells each)
static_assert(NT == LX * TY && LX == 16, "one thread per cell pair, two tile rows per warp");

// staged boxes of one plane: E^{n+1} and a over the tile plus the high halo (origin (i0, j0)),
// H^{n+1/2} over the tile plus both halos (origin (i0 - 4, j0 - 1): the x coordinate of every copy
// stays 16-byte aligned; the first three columns are not used)
constexpr int EW = TX + 4, EH = TY + 1;
constexpr int HW = TX + 8, HH = TY + 2;
constexpr int HXO = 4;  // x offset of the tile in the H box (its y offset is 1)
constexpr uint32_t E_BYTES = 3 * EW * EH * 4, H_BYTES = 3 * HW * HH * 4, A_BYTES = EW * EH * 4;
constexpr uint32_t STAGE_TX = E_BYTES + H_BYTES + A_BYTES;
constexpr int round128(int b) { return (b + 127) / 128 * 128; }
constexpr int E_OFF = 0, H_OFF = round128(E_BYTES), A_OFF = H_OFF + round128(H_BYTES);
constexpr int STAGE_BYTES = round128(A_OFF + A_BYTES);
// E^n of a plane with the high halo: [3][NY][NX], column TX and row TY the halo (column TX + 1 pad)
constexpr int NX = TX + 2, NY = TY + 1;
static_assert(EW % 2 == 0 && HW % 2 == 0 && NX % 2 == 0 && HXO % 2 == 0, "float2 pairs");
static_assert((EW * EH) % 2 == 0 && (HW * HH) % 2 == 0 && (NX * NY) % 2 == 0, "float2 pairs");
constexpr int MAXTZ = 256;
constexpr int SE_OFF = 0;                                  // new E: [2][3][NY][NX]
constexpr int PF_OFF = SE_OFF + round128(2 * 3 * NY * NX * 4);  // per-plane flags [MAXTZ]
constexpr int BAR_OFF = round128(PF_OFF + MAXTZ);          // up to 4 mbarriers
constexpr int RING_OFF = round128(BAR_OFF + 4 * 8);
constexpr int smem_bytes(int ns) { return RING_OFF + ns * STAGE_BYTES + 128; }

__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }

__device__ __forceinline__ int box_offset(const int lo[3], const int hi[3], int x, int y, int k) {
  return ((k - lo[2]) * (hi[1] - lo[1]) + (y - lo[1])) * (hi[0] - lo[0]) + (x - lo[0]);
}

struct Ring {
  unsigned char* base;
  uint64_t* bar;
  int kstart;  // first plane staged (the ring is filled downwards from it)
  int ns;
  __device__ int slot(int p) const { return (kstart - p) % ns; }
  __device__ uint32_t parity(int p) const { return ((kstart - p) / ns) & 1; }
  __device__ const float (*E(int p) const)[EH][EW] {
    return reinterpret_cast<const float(*)[EH][EW]>(base + slot(p) * STAGE_BYTES + E_OFF);
  }
  __device__ const float (*H(int p) const)[HH][HW] {
    return reinterpret_cast<const float(*)[HH][HW]>(base + slot(p) * STAGE_BYTES + H_OFF);
  }
  __device__ const float (*Av(int p) const)[EW] {
    return reinterpret_cast<const float(*)[EW]>(base + slot(p) * STAGE_BYTES + A_OFF);
  }
  __device__ bool wait(int p) const { return mbar_wait(&bar[slot(p)], parity(p)); }
  // one thread: fill the stage of plane p
  __device__ void issue(const InvMaps& M, int i0, int j0, int p) const {
    unsigned char* st = base + slot(p) * STAGE_BYTES;
    uint64_t* b = &bar[slot(p)];
    mbar_arrive_expect(b, STAGE_TX);
    tma_load_box(st + E_OFF, &M.e, i0, j0, p, 0, b);
    tma_load_box(st + H_OFF, &M.h, i0 - HXO, j0 - 1, p, 0, b);
    tma_load_box(st + A_OFF, &M.a, i0, j0, p, 0, b);
  }
};

// Sum of the source terms (soft sources and TFSF E corrections) on component c at (x, y, k) for this
// step, in source order.
__device__ __forceinline__ float source_at(const InvArgs& A, int c, int x, int y, int k) {
  float v = 0.f;
  for (int s = 0; s < A.nsrc; ++s) {
    const SrcDev& sd = A.src[s];
    if (sd.comp != c || x < sd.lo[0] || x >= sd.hi[0] || y < sd.lo[1] || y >= sd.hi[1] || k < sd.lo[2] ||
        k >= sd.hi[2])
      continue;
    v = __fadd_rn(v, __fmul_rn(sd.w[box_offset(sd.lo, sd.hi, x, y, k)], sd.g[A.step]));
  }
  return v;
}

// E^n of one component from E^{n+1} (e1), S a (sa), the two curl differences (da - db) and the source
// term (src): (e1 - src) - sa (da - db), rounded in that order. Used for own and halo cells alike.
__device__ __forceinline__ float inv_e(float e1, float src, float sa, float da, float db) {
  return __fsub_rn(__fsub_rn(e1, src), __fmul_rn(sa, __fsub_rn(da, db)));
}

// H^{n-1/2} of one component: h1 + S (da - db).
__device__ __forceinline__ float inv_h(float h1, float S, float da, float db) {
  return __fadd_rn(h1, __fmul_rn(S, __fsub_rn(da, db)));
}

// The inverse step of one request for the block at tile (bx, by), z-chunk bz.
template <int NSTAGE>
__device__ __forceinline__ void inv_body(const InvArgs& A, const InvMaps& M, const int bx, const int by, const int bz) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
  float(*sEn)[3][NY][NX] = reinterpret_cast<float(*)[3][NY][NX]>(sm + SE_OFF);
  unsigned char* pflag = sm + PF_OFF;

  const Geo& g = A.g;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int lx = lane & (LX - 1), ty = 2 * warp + (lane >> 4);
  const int i0 = bx * TX, j0 = by * TY;
  const int k0 = bz * A.tz;
  const int k1 = min(g.n[2], k0 + A.tz);
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int plane = (int)g.plane;
  const int i = i0 + 2 * lx, j = j0 + ty;  // the thread's cells (i, j) and (i + 1, j)
  const bool own0 = i < nx && j < ny, own1 = i + 1 < nx && j < ny;
  const int q0 = j * g.nxp + i;
  const float S = g.S;
  const int kstart = k1 < nz ? k1 : k1 - 1;  // planes staged: kstart down to kend
  const int kend = k0 > 0 ? k0 - 1 : 0;
  const Ring R{sm + RING_OFF, reinterpret_cast<uint64_t*>(sm + BAR_OFF), kstart, NSTAGE};
  bool waited = true;

  if (tid == 0) {
    for (int b = 0; b < NSTAGE; ++b) mbar_init(&R.bar[b], 1);
    mbar_init_fence();
  }
  {
    // per-plane flags of the chunk (and the plane above it): bit 0 a source meets the tile with its
    // high halo, bit 1 the design box meets the tile
    const int xa = i0, xb = min(i0 + TX + 1, nx), ya = j0, yb = min(j0 + TY + 1, ny);
    for (int p = tid; p <= k1 - k0 && p < MAXTZ; p += NT) {
      const int k = k0 + p;
      int f = 0;
      for (int s = 0; s < A.nsrc; ++s) {
        const SrcDev& sd = A.src[s];
        if (k >= sd.lo[2] && k < sd.hi[2] && sd.lo[0] < xb && sd.hi[0] > xa && sd.lo[1] < yb && sd.hi[1] > ya) f |= 1;
      }
      if (A.dLda && k >= A.dlo[2] && k < A.dhi[2] && A.dlo[0] < min(i0 + TX, nx) && A.dhi[0] > i0 &&
          A.dlo[1] < min(j0 + TY, ny) && A.dhi[1] > j0)
        f |= 2;
      pflag[p] = (unsigned char)f;
    }
  }
  pdl_wait();  // the fields come after the previous kernel of the stream
  if (tid == 0)
    for (int p = kstart; p >= max(kstart - NSTAGE + 1, kend); --p) R.issue(M, i0, j0, p);
  __syncthreads();

  // R membership along x and y of the own pair, the halo column x = i0 + TX and the halo row
  // y = j0 + TY (E_c: half position along c, integer along the others; H_c the other way round)
  auto rx_int = [&](int x) { return x >= g.rint_lo[0] && x <= g.rint_hi[0]; };
  auto rx_half = [&](int x) { return x >= g.rhalf_lo[0] && x <= g.rhalf_hi[0]; };
  auto ry_int = [&](int y) { return y >= g.rint_lo[1] && y <= g.rint_hi[1]; };
  auto ry_half = [&](int y) { return y >= g.rhalf_lo[1] && y <= g.rhalf_hi[1]; };
  auto rz_int = [&](int k) { return k >= g.rint_lo[2] && k <= g.rint_hi[2]; };
  auto rz_half = [&](int k) { return k >= g.rhalf_lo[2] && k <= g.rhalf_hi[2]; };

  // halo roles: warp 3 lanes 0..15 the column x = i0 + TX at y = j0 + lx (E_y, E_z); warp 4 lanes 0..15
  // the row y = j0 + TY at the pair (i, i + 1) (E_x, E_z)
  const int xh = i0 + TX, yc = j0 + lx, yh = j0 + TY;
  const bool hcol = warp == 3 && lane < LX && xh < nx && yc < ny;
  const bool hrow = warp == 4 && lane < LX && yh < ny && i < nx;
  const bool hrow1 = hrow && i + 1 < nx;

  // E^n (components 0..2 selected by `want`, bit c) at (x, y, k) from the staged planes k and k-1;
  // (ex, ey) the cell's position in the E box, (hx, hy) in the H box
  auto e_cell = [&](int c, int x, int y, int k, const float (*Ek)[EH][EW], const float (*Ak)[EW],
                    const float (*Hk)[HH][HW], const float (*Hm)[HH][HW], int ex, int ey, int hx, int hy,
                    bool has_src) -> float {
    const float e1 = Ek[c][ey][ex];
    const float sa = S * Ak[ey][ex];
    float da, db;
    bool in;
    if (c == 0) {
      da = Hk[2][hy][hx] - Hk[2][hy - 1][hx];
      db = Hk[1][hy][hx] - (k > 0 ? Hm[1][hy][hx] : 0.f);
      in = rx_half(x) && ry_int(y) && rz_int(k) && y > 0 && k > 0;
    } else if (c == 1) {
      da = Hk[0][hy][hx] - (k > 0 ? Hm[0][hy][hx] : 0.f);
      db = Hk[2][hy][hx] - Hk[2][hy][hx - 1];
      in = rx_int(x) && ry_half(y) && rz_int(k) && x > 0 && k > 0;
    } else {
      da = Hk[1][hy][hx] - Hk[1][hy][hx - 1];
      db = Hk[0][hy][hx] - Hk[0][hy - 1][hx];
      in = rx_int(x) && ry_int(y) && rz_half(k) && x > 0 && y > 0;
    }
    if (!in) return e1;
    const float src = has_src ? source_at(A, c, x, y, k) : 0.f;
    return inv_e(e1, src, sa, da, db);
  };

  const int ex0 = 2 * lx, ey0 = ty;             // own cell 0 in the E and a boxes
  const int hx0 = 2 * lx + HXO, hy0 = ty + 1;   // own cell 0 in the H box
  // E^n (x, y components) of the own pair at the plane above the one being updated
  float eup_x[2] = {0.f, 0.f}, eup_y[2] = {0.f, 0.f};

  waited &= R.wait(kstart);
  if (k1 < nz) {
    // E^n at plane k1, the plane above the chunk (its owner stores it; this block recomputes it)
    if (k1 - 1 >= kend) waited &= R.wait(k1 - 1);
    const int pf = pflag[k1 - k0];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (!(c == 0 ? own0 : own1)) continue;
      eup_x[c] = e_cell(0, i + c, j, k1, R.E(k1), R.Av(k1), R.H(k1), R.H(k1 - 1), ex0 + c, ey0, hx0 + c, hy0, pf & 1);
      eup_y[c] = e_cell(1, i + c, j, k1, R.E(k1), R.Av(k1), R.H(k1), R.H(k1 - 1), ex0 + c, ey0, hx0 + c, hy0, pf & 1);
    }
    __syncthreads();  // every thread is done with plane k1
    if (tid == 0 && k1 - NSTAGE >= kend) {
      async_proxy_fence();
      R.issue(M, i0, j0, k1 - NSTAGE);
    }
  }

  for (int k = k1 - 1; k >= k0; --k) {
    const int it = k1 - 1 - k;
    const int q = k * plane + q0;
    const int pf = pflag[k - k0];
    if (k - 1 >= kend && k > 0) waited &= R.wait(k - 1);
    const float(*Ek)[EH][EW] = R.E(k);
    const float(*Ak)[EW] = R.Av(k);
    const float(*Hk)[HH][HW] = R.H(k);
    const float(*Hm)[HH][HW] = k > 0 ? R.H(k - 1) : R.H(k);  // not read at k = 0
    float(*sE)[NY][NX] = sEn[it & 1];

    // (a) E^n of the own pair (into registers, the new-E tile and nxt), dL/da on design cells
    float en[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float ho[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};  // H^{n+1/2} of the own pair
    if (own0) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int x = i + c;
        if (c == 1 && !own1) continue;
#pragma unroll
        for (int e = 0; e < 3; ++e)
          en[c][e] = e_cell(e, x, j, k, Ek, Ak, Hk, Hm, ex0 + c, ey0, hx0 + c, hy0, pf & 1);
        ho[c][0] = Hk[0][hy0][hx0 + c];
        ho[c][1] = Hk[1][hy0][hx0 + c];
        ho[c][2] = Hk[2][hy0][hx0 + c];
      }
#pragma unroll
      for (int e = 0; e < 3; ++e)
        st2(&A.nxt.f[e][q], en[0][e], en[1][e]);  // (for odd nx the pair's second cell in the padding is 0)
      if (pf & 2) {  // dL/da += S Ebar . curl_b(H^{n+1/2}) on the design box (inside R: plain curls)
        const float2 bx = ld2(&A.eb[0][q]), by = ld2(&A.eb[1][q]), bz = ld2(&A.eb[2][q]);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int x = i + c;
          if ((c == 1 && !own1) || x < A.dlo[0] || x >= A.dhi[0] || j < A.dlo[1] || j >= A.dhi[1] ||
              k < A.dlo[2] || k >= A.dhi[2])
            continue;
          const int hx = hx0 + c;
          const float hz = Hk[2][hy0][hx], hy = Hk[1][hy0][hx], hxv = Hk[0][hy0][hx];
          float gs = 0.f;
          if (j > 0 && k > 0) gs += (c ? bx.y : bx.x) * ((hz - Hk[2][hy0 - 1][hx]) - (hy - Hm[1][hy0][hx]));
          if (x > 0 && k > 0) gs += (c ? by.y : by.x) * ((hxv - Hm[0][hy0][hx]) - (hz - Hk[2][hy0][hx - 1]));
          if (x > 0 && j > 0) gs += (c ? bz.y : bz.x) * ((hy - Hk[1][hy0][hx - 1]) - (hxv - Hk[0][hy0 - 1][hx]));
          const int m = box_offset(A.dlo, A.dhi, x, j, k);
          A.dLda[m] += (double)S * (double)gs;
        }
      }
    }
    // the tile of E^n (zero at cells beyond the grid: the PEC wall that the H update reads there)
#pragma unroll
    for (int e = 0; e < 3; ++e) st2(&sE[e][ty][ex0], en[0][e], en[1][e]);
    // the high halo column (i0 + TX, j0 + lx): E_y, E_z
    if (hcol) {
      const int ex = TX, ey = lx, hx = TX + HXO, hy = lx + 1;
      sE[1][lx][TX] = e_cell(1, xh, yc, k, Ek, Ak, Hk, Hm, ex, ey, hx, hy, pf & 1);
      sE[2][lx][TX] = e_cell(2, xh, yc, k, Ek, Ak, Hk, Hm, ex, ey, hx, hy, pf & 1);
    } else if (warp == 3 && lane < LX) {
      sE[1][lx][TX] = 0.f;  // beyond the grid: the PEC wall
      sE[2][lx][TX] = 0.f;
    }
    // the high halo row (i, j0 + TY), (i + 1, j0 + TY): E_x, E_z
    if (warp == 4 && lane < LX) {
      float r0[2] = {0.f, 0.f}, r2[2] = {0.f, 0.f};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!(c == 0 ? hrow : hrow1)) continue;
        const int ex = ex0 + c, ey = TY, hx = hx0 + c, hy = TY + 1;
        r0[c] = e_cell(0, i + c, yh, k, Ek, Ak, Hk, Hm, ex, ey, hx, hy, pf & 1);
        r2[c] = e_cell(2, i + c, yh, k, Ek, Ak, Hk, Hm, ex, ey, hx, hy, pf & 1);
      }
      st2(&sE[0][TY][ex0], r0[0], r0[1]);
      st2(&sE[2][TY][ex0], r2[0], r2[1]);
    }
    __syncthreads();  // the new-E tile is complete; every thread is done with plane k's stage
    if (tid == 0 && k - NSTAGE >= kend) {
      async_proxy_fence();
      R.issue(M, i0, j0, k - NSTAGE);
    }

    // (b) H^{n-1/2} of the own pair from E^n of this plane (tile and halo) and of the plane above
    if (own0) {
      const float2 ezy = ld2(&sE[2][ty + 1][ex0]), exy = ld2(&sE[0][ty + 1][ex0]);  // at y + 1
      const float ez2 = sE[2][ty][ex0 + 2], ey2 = sE[1][ty][ex0 + 2];              // at x + 1 of cell 1
      const bool ryh = ry_half(j), ryi = ry_int(j), rzh = rz_half(k), rzi = rz_int(k);
      float hn[2][3];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int x = i + c;
        const float ez_y = c ? ezy.y : ezy.x, ex_y = c ? exy.y : exy.x;
        const float ez_x = c ? ez2 : en[1][2], ey_x = c ? ey2 : en[1][1];
        hn[c][0] = (rx_int(x) && ryh && rzh) ? inv_h(ho[c][0], S, ez_y - en[c][2], eup_y[c] - en[c][1]) : ho[c][0];
        hn[c][1] = (rx_half(x) && ryi && rzh) ? inv_h(ho[c][1], S, eup_x[c] - en[c][0], ez_x - en[c][2]) : ho[c][1];
        hn[c][2] = (rx_half(x) && ryh && rzi) ? inv_h(ho[c][2], S, ey_x - en[c][1], ex_y - en[c][0]) : ho[c][2];
      }
      if (!own1) hn[1][0] = hn[1][1] = hn[1][2] = 0.f;
      st2(&A.nxt.f[3][q], hn[0][0], hn[1][0]);
      st2(&A.nxt.f[4][q], hn[0][1], hn[1][1]);
      st2(&A.nxt.f[5][q], hn[0][2], hn[1][2]);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      eup_x[c] = en[c][0];
      eup_y[c] = en[c][1];
    }
  }
  if (!waited) atomicOr(A.status, kStatusTimeout);
}

template <int NSTAGE>
__global__ void __launch_bounds__(NT, 2) k_inv_fused(const __grid_constant__ InvArgs A, const __grid_constant__ InvMaps M) {
  inv_body<NSTAGE>(A, M, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Several requests in one launch (see k_fwd_fused_group).
template <int NSTAGE>
__global__ void __launch_bounds__(NT, 2) k_inv_fused_group(const __grid_constant__ InvGroup G) {
  int bx, by, bz;
  const int r = group_locate(G.grid, bx, by, bz);
  inv_body<NSTAGE>(G.a[r], G.m[r], bx, by, bz);
}

}  // namespace

void launch_inv_group(InvGroup& G, cudaStream_t s) {
  const int total = group_fill(G.grid, G.n, [&](int r, int* nb) {
    const Geo& g = G.a[r].g;
    nb[0] = (g.n[0] + TX - 1) / TX;
    nb[1] = (g.n[1] + TY - 1) / TY;
    nb[2] = (g.n[2] + G.a[r].tz - 1) / G.a[r].tz;
  });
  if (total == 0) return;
  if (G.a[0].nstage == 4) launch_pdl(k_inv_fused_group<4>, dim3(total), dim3(NT), smem_bytes(4), s, G);
  else launch_pdl(k_inv_fused_group<3>, dim3(total), dim3(NT), smem_bytes(3), s, G);
}

MapBox inv_box_e() { return {EW, EH}; }
MapBox inv_box_h() { return {HW, HH}; }

int prepare_inv(int nstage, int* blocks_per_sm) {
  auto k = nstage == 4 ? k_inv_fused<4> : k_inv_fused<3>;
  auto kg = nstage == 4 ? k_inv_fused_group<4> : k_inv_fused_group<3>;
  const int smem = smem_bytes(nstage);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kg, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, NT, smem);
  return e == cudaSuccess ? FDTD_OK : set_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
}

int inv_max_tz() { return MAXTZ - 1; }

void launch_inv(const InvArgs& a, const InvMaps& m, cudaStream_t s) {
  const Geo& g = a.g;
  dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + a.tz - 1) / a.tz);
  if (a.nstage == 4) launch_pdl(k_inv_fused<4>, grid, dim3(NT), smem_bytes(4), s, a, m);
  else launch_pdl(k_inv_fused<3>, grid, dim3(NT), smem_bytes(3), s, a, m);
}

}  // namespace fdtd
