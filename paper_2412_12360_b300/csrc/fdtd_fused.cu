// Fused forward step of arXiv 2412.12360 Sec. 2.1: the H update (Eq. 1) and the E update (Eq. 2) of
// one time step in a single sweep over the grid, with the CPML memories, the soft sources and the
// detectors as epilogues of the same sweep.
//
// Each block owns a TX x TY column tile and marches a chunk of z-planes upwards. The planes arrive
// through a ring of shared-memory stages that the TMA unit fills (one thread issues the bulk tensor
// copies of E^n with a one-cell halo, H^{n-1/2} with the low halo, and a; the block waits on one
// mbarrier per stage), so the loads of the next planes are in flight while a plane is computed.
// Per plane the block computes H^{n+1/2} for its cells and, redundantly, for the halo column
// x = i0-1 and row y = j0-1 that its E update reads, then E^{n+1}. Fields are double-buffered (read
// `cur`, write `nxt`) so neighbouring tiles never see a half-updated field; every cell is read and
// written once per step from HBM (52 bytes per cell) and the halos come from L2.
//
// Each thread updates two x-adjacent cells (x0 = i0 + 2 lx and x0 + 1): the staged planes are read
// and the results written as float2 pairs, the x-neighbour one cell needs is the other cell's value
// already in registers, and the per-plane bookkeeping (waits, flags, indices) is shared by two
// cells. A warp covers two rows of the tile (lanes 0..15 and 16..31).
//
// Every cell takes the plain Yee update; cells in a CPML layer add the correction
// (1/kappa - 1) d + psi per curl term, which is exactly 0 off the layers and on their inner edge, so
// the PML-free region R is updated by the plain formula the inverse step mirrors. The CPML memories a
// cell needs are copied ahead by its thread (cp.async into private shared-memory slots) one phase
// before use. Sources and detectors are decided per plane from flags the block computes once.
#include "../../include/fdtd.h"
#include "fdtd_internal.cuh"
#include "fdtd_tma.cuh"

namespace fdtd {

namespace {

constexpr int TX = 32, TY = 16, NT = 256;  // tile of TX x TY cells, two x-adjacent cells per thread
constexpr int LX = TX / 2;                 // threads per tile row
static_assert(NT == LX * TY && LX == 16, "one thread per cell pair, two tile rows per warp");
// new H with the low halo: row r = y - (j0 - 1), column c = x - i0 + 2 (column 1 is the halo
// x = i0 - 1, column 0 is padding so that every pair of own cells starts at an even column)
constexpr int HX = TX + 2, HY = TY + 1;

// CPML correction of one curl term inside a layer: the update uses d / kappa + psi_new where the plain
// Yee update uses d, so the correction is (1/kappa - 1) d + psi_new with psi_new = b psi_old + c d
// (written to pout[z] when STORE). On the layer's inner edge (depth 0) 1/kappa = 1, b = 1, c = 0 and
// psi stays 0, so the correction is 0 there, as it is off the layers (where the caller skips it).
template <bool STORE>
__device__ __forceinline__ float corr(float d, float ik, float b, float c, float psi_old, float* pout, int z) {
  const float v = b * psi_old + c * d;
  if (STORE) pout[z] = v;
  return (ik - 1.f) * d + v;
}

// CPML coefficients at one position along one axis: integer-position (E) and half-position (H) sets
struct Coef {
  float b, c, ik;
};

// compile-time flag for the specialised plane loops
template <bool B>
struct Flag {
  static constexpr bool value = B;
};

// slab index of position x along an axis with n cells and layers p0, p1 (-1 off the layers)
__device__ __forceinline__ int slab_of(int x, int n, int p0, int p1) {
  return x < p0 ? x : (x >= n - p1 ? p0 + x - (n - p1) : -1);
}

// 4-byte asynchronous copy global -> shared (completion tracked per thread with commit groups)
__device__ __forceinline__ void cp4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// 8-byte (two x-adjacent floats) shared or global accesses; the address must be 8-byte aligned
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }

// psi index of the point (x, y, k), slab index s, for the derivative along x, y or z
__device__ __forceinline__ int zx_of(const Geo& g, int y, int k, int s) { return (k * g.n[1] + y) * g.slab[0] + s; }
__device__ __forceinline__ int zy_of(const Geo& g, int x, int k, int s) { return (k * g.slab[1] + s) * g.nxp + x; }
__device__ __forceinline__ int zz_of(const Geo& g, int x, int y, int s) { return (s * g.n[1] + y) * g.nxp + x; }

__device__ __forceinline__ float pick3(int c, float a, float b, float d) { return c == 0 ? a : (c == 1 ? b : d); }

__device__ __forceinline__ int box_offset(const int lo[3], const int hi[3], int x, int y, int k) {
  return ((k - lo[2]) * (hi[1] - lo[1]) + (y - lo[1])) * (hi[0] - lo[0]) + (x - lo[0]);
}

// Shared-memory ring of z-planes filled by the TMA unit. One stage holds, for one plane k of the
// tile, E^n with a halo (x in [i0-4, i0+TX+4), y in [j0-1, j0+TY+1)), H^{n-1/2} with the low halo
// (x in [i0-4, i0+TX), y in [j0-1, j0+TY)) and a (the tile). Both boxes start 4 cells left of the
// tile so that the x coordinate of every copy is 16-byte aligned; the extra columns are not used.
constexpr int EW = TX + 8, EH = TY + 2;
constexpr int HW = TX + 4, HH = TY + 1;
constexpr int XO = 4;  // x offset of the tile inside the E and H boxes
constexpr uint32_t E_BYTES = 3 * EW * EH * 4, H_BYTES = 3 * HW * HH * 4, A_BYTES = TX * TY * 4;
constexpr uint32_t STAGE_TX = E_BYTES + H_BYTES + A_BYTES;  // transaction bytes of one stage
constexpr int round128(int b) { return (b + 127) / 128 * 128; }
constexpr int E_OFF = 0, H_OFF = round128(E_BYTES), A_OFF = H_OFF + round128(H_BYTES);
constexpr int STAGE_BYTES = round128(A_OFF + A_BYTES);
// float2 accesses to the staged boxes and the new-H tile need even row pitches, even component
// planes and an even column for every pair's first cell
static_assert(EW % 2 == 0 && HW % 2 == 0 && HX % 2 == 0 && XO % 2 == 0, "float2 pairs");
static_assert((EW * EH) % 2 == 0 && (HW * HH) % 2 == 0 && (HX * HY) % 2 == 0, "float2 pairs");
// CPML memories of the plane being computed, copied ahead by each thread for itself (cp.async).
// H slots: 6 c + m for own cell c (m: Hy_x, Hz_x, Hx_y, Hz_y, Hx_z, Hy_z). E slots: 6 c + m
// (m: Ey_x, Ez_x, Ex_y, Ez_y, Ex_z, Ey_z). Halo slots, one column per halo thread (hid 0..15 the
// row-halo lanes, 16..31 the column-halo lanes): the row-halo cell c at 4 c + (Hz_x, Hz_y, Hx_y,
// Hx_z), the column-halo point at (Hz_x, Hz_y, Hy_z, Hy_x).
constexpr int NPH = 12, NPE = 12, NHAL = 8, NHT = 32;
// CPML tables of the tile's x and y positions (from i0-1 and j0-1): b, c, 1/kappa at integer then
// half positions
constexpr int TABX = TX + 1, TABY = TY + 1;
// shared memory: the new-H tiles, the psi slots, tables, flags and flux sums, the mbarriers, then
// the ring of NS stages
constexpr int SH_OFF = 0;                                         // new H: [2][3][HY][HX] floats
constexpr int PH_OFF = SH_OFF + round128(2 * 3 * HY * HX * 4);    // [NPH][NT]
constexpr int PE_OFF = PH_OFF + NPH * NT * 4;                     // [NPE][NT]
constexpr int HA_OFF = PE_OFF + NPE * NT * 4;                     // [NHAL][NHT]
constexpr int TX_OFF = HA_OFF + NHAL * NHT * 4;                   // [6][TABX]
constexpr int TY_OFF = TX_OFF + 6 * TABX * 4;                     // [6][TABY]
// per-plane flags of the block's z-chunk: bit 0 a source, bit 1 a detector meets the tile at that
// plane (uniform over the block, so planes without either cost one load)
constexpr int MAXTZ = 256;
constexpr int PF_OFF = TY_OFF + 6 * TABY * 4;                     // [MAXTZ] bytes
constexpr int WF_OFF = round128(PF_OFF + MAXTZ);                  // flux sums per tile row: [kMaxDet][TY]
constexpr int BAR_OFF = round128(WF_OFF + kMaxDet * TY * 8);      // up to 4 mbarriers
constexpr int RING_OFF = round128(BAR_OFF + 4 * 8);
constexpr int smem_bytes(int ns) { return RING_OFF + ns * STAGE_BYTES + 128; }  // + slack to align the base

struct Ring {
  unsigned char* base;
  uint64_t* bar;
  __device__ const float (*E(int b) const)[EH][EW] {
    return reinterpret_cast<const float(*)[EH][EW]>(base + b * STAGE_BYTES + E_OFF);
  }
  __device__ const float (*H(int b) const)[HH][HW] {
    return reinterpret_cast<const float(*)[HH][HW]>(base + b * STAGE_BYTES + H_OFF);
  }
  __device__ const float (*Av(int b) const)[TX] {
    return reinterpret_cast<const float(*)[TX]>(base + b * STAGE_BYTES + A_OFF);
  }
  // one thread: fill stage b with plane k
  __device__ void issue(const FwdMaps& M, int b, int i0, int j0, int k) const {
    unsigned char* st = base + b * STAGE_BYTES;
    mbar_arrive_expect(&bar[b], STAGE_TX);
    tma_load_box(st + E_OFF, &M.e, i0 - XO, j0 - 1, k, 0, &bar[b]);
    tma_load_box(st + H_OFF, &M.h, i0 - XO, j0 - 1, k, 0, &bar[b]);
    tma_load_box(st + A_OFF, &M.a, i0, j0, k, 0, &bar[b]);
  }
};

// the coefficients of table column idx: row0 = 0 for integer (E) positions, 3 for half (H) positions
template <int W>
__device__ __forceinline__ Coef coef_at(const float (*tab)[W], int row0, int idx) {
  return Coef{tab[row0][idx], tab[row0 + 1][idx], tab[row0 + 2][idx]};
}

// The forward step of one request for the block at tile (bx, by), z-chunk bz.
template <int NSTAGE>
__device__ __forceinline__ void fwd_body(const FwdArgs& A, const FwdMaps& M, const int bx, const int by, const int bz) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
  Ring R{sm + RING_OFF, reinterpret_cast<uint64_t*>(sm + BAR_OFF)};
  float(*sHb)[3][HY][HX] = reinterpret_cast<float(*)[3][HY][HX]>(sm + SH_OFF);
  float(*sPH)[NT] = reinterpret_cast<float(*)[NT]>(sm + PH_OFF);
  float(*sPE)[NT] = reinterpret_cast<float(*)[NT]>(sm + PE_OFF);
  float(*sHal)[NHT] = reinterpret_cast<float(*)[NHT]>(sm + HA_OFF);
  float(*tabX)[TABX] = reinterpret_cast<float(*)[TABX]>(sm + TX_OFF);
  float(*tabY)[TABY] = reinterpret_cast<float(*)[TABY]>(sm + TY_OFF);
  unsigned char* pflag = sm + PF_OFF;
  double(*wflux)[TY] = reinterpret_cast<double(*)[TY]>(sm + WF_OFF);

  const Geo& g = A.g;
  const Tables& T = A.T;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int lx = lane & (LX - 1), ty = 2 * warp + (lane >> 4);
  const int i0 = bx * TX, j0 = by * TY;
  const int k0 = bz * A.tz;
  const int k1 = min(g.n[2], k0 + A.tz);
  const int kb = k0 > 0 ? k0 - 1 : k0;  // first plane staged (k0-1 supplies H^{n+1/2} below the chunk)
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int plane = (int)g.plane;
  const int i = i0 + 2 * lx, j = j0 + ty;  // the thread's cells (i, j) and (i + 1, j)
  const bool own0 = i < nx && j < ny, own1 = i + 1 < nx && j < ny;
  const int q0 = j * g.nxp + i;
  const float S = g.S;
  const int ex = 2 * lx + XO, ey = ty + 1;  // cell 0 in the staged boxes
  const int rx = 2 * lx + 2, ry = ty + 1;   // cell 0 in the new-H tile
  const int cx0 = 2 * lx + 1;               // cell 0 in the x table
  bool waited = true;

  if (tid == 0) {
    for (int b = 0; b < NSTAGE; ++b) mbar_init(&R.bar[b], 1);
    mbar_init_fence();
  }
  // CPML tables of the tile's positions (clamped into the grid; out-of-grid entries are not used)
  for (int t = tid; t < 6 * (TABX + TABY); t += NT) {
    const bool isx = t < 6 * TABX;
    const int u = isx ? t : t - 6 * TABX;
    const int row = isx ? u / TABX : u / TABY, col = isx ? u % TABX : u % TABY;
    const int ax = isx ? 0 : 1;
    const int pos = min(max((isx ? i0 : j0) - 1 + col, 0), g.n[ax] - 1);
    const int hf = row / 3, w = row % 3;
    const float* src = w == 0 ? T.b[ax][hf] : (w == 1 ? T.c[ax][hf] : T.ik[ax][hf]);
    (isx ? tabX[row] : tabY[row])[col] = src[pos];
  }
  {
    // epilogue flags of the chunk's planes for this tile
    const int xa = i0, xb = min(i0 + TX, nx), ya = j0, yb = min(j0 + TY, ny);
    for (int p = tid; p < k1 - k0; p += NT) {
      const int k = k0 + p;
      int f = 0;
      for (int s = 0; s < A.nsrc; ++s) {
        const SrcDev& sd = A.src[s];
        if (k >= sd.lo[2] && k < sd.hi[2] && sd.lo[0] < xb && sd.hi[0] > xa && sd.lo[1] < yb && sd.hi[1] > ya) f |= 1;
      }
      for (int s = 0; s < A.ndet; ++s) {
        const DetDev& d = A.det[s];
        if (k >= d.lo[2] && k < d.hi[2] && d.lo[0] < xb && d.hi[0] > xa && d.lo[1] < yb && d.hi[1] > ya) f |= 2;
      }
      pflag[p] = (unsigned char)f;
    }
    if (tid < kMaxDet * TY) wflux[tid / TY][tid % TY] = 0.0;
  }
  // everything above reads only constant tables and arguments; the fields come after the previous step
  pdl_wait();
  if (tid == 0)
    for (int p = kb; p <= min(kb + NSTAGE - 1, k1); ++p) R.issue(M, p - kb, i0, j0, p);
  __syncthreads();

  // halo H: warp 3 lanes 0..15 compute the row y = j0-1 (Hx, Hz) at the pair (i, i+1); warp 4 lanes
  // 0..15 the column x = i0-1 (Hy, Hz) at y = j0 + lx
  const bool hrow = warp == 3 && lane < LX && j0 > 0 && i < nx;
  const bool hrow1 = hrow && i + 1 < nx;
  const int yc = j0 + lx;
  const bool hcol = warp == 4 && lane < LX && i0 > 0 && yc < ny;
  const int hid = (warp == 4 ? LX : 0) + lx;  // the halo thread's slot column

  // slab indices along x and y of the own cells and the halo points (-1 off the layers)
  const int sX0 = slab_of(min(i, nx - 1), nx, g.pml[0], g.pml[1]);
  const int sX1 = slab_of(min(i + 1, nx - 1), nx, g.pml[0], g.pml[1]);
  const int sY = slab_of(min(j, ny - 1), ny, g.pml[2], g.pml[3]);
  const int sYh = slab_of(max(j0 - 1, 0), ny, g.pml[2], g.pml[3]);  // the row halo (block uniform)
  const int sXc = slab_of(max(i0 - 1, 0), nx, g.pml[0], g.pml[1]);  // the column halo (block uniform)
  const int sYc = slab_of(min(yc, ny - 1), ny, g.pml[2], g.pml[3]);
  // whether some lane of this warp has an own cell in an x or a y layer (uniform over the warp, so
  // the per-axis CPML code below is branched over, not predicated, by the warps that have none)
  const bool wx = __any_sync(0xffffffffu, (own0 && sX0 >= 0) || (own1 && sX1 >= 0));
  const bool wy = __any_sync(0xffffffffu, own0 && sY >= 0);
  // whether the tile or its low halo reaches into an x or y layer (uniform over the block): if not,
  // only planes in a z layer have CPML work
  const bool tile_xy = i0 - 1 < g.pml[0] || i0 + TX > nx - g.pml[1] || j0 - 1 < g.pml[2] || j0 + TY > ny - g.pml[3];

  const PsiSet& PHi = A.psiH_cur;
  const PsiSet& PHo = A.psiH_nxt;
  const PsiSet& PEi = A.psiE_cur;
  const PsiSet& PEo = A.psiE_nxt;
  const Fields& N = A.nxt;

  // The plane loop, compiled twice: with or without CPML along x and y in the tile (XY). Each block
  // runs the one it needs, so the common interior path carries none of the code (nor the register
  // pressure) of the x/y layers.
  auto march = [&](auto xy_tag) {
    constexpr bool XY = decltype(xy_tag)::value;
    // copies of psi_old of plane kk into this thread's slots (one commit group each)
    auto fetch_psiH = [&](int kk, int sZk) {
      if (!XY && sZk < 0) {
        cp_commit();
        return;
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!(c == 0 ? own0 : own1)) continue;
        const int sX = c == 0 ? sX0 : sX1, x = i + c;
        if constexpr (XY) {
          if (wx && sX >= 0) {
            const int z = zx_of(g, j, kk, sX);
            cp4(&sPH[6 * c + 0][tid], PHi.p[1][0] + z);
            cp4(&sPH[6 * c + 1][tid], PHi.p[2][0] + z);
          }
          if (wy && sY >= 0) {
            const int z = zy_of(g, x, kk, sY);
            cp4(&sPH[6 * c + 2][tid], PHi.p[0][1] + z);
            cp4(&sPH[6 * c + 3][tid], PHi.p[2][1] + z);
          }
        }
        if (sZk >= 0) {
          const int z = zz_of(g, x, j, sZk);
          cp4(&sPH[6 * c + 4][tid], PHi.p[0][2] + z);
          cp4(&sPH[6 * c + 5][tid], PHi.p[1][2] + z);
        }
      }
      if (hrow) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (c == 1 && !hrow1) continue;
          const int sX = c == 0 ? sX0 : sX1, x = i + c;
          if constexpr (XY) {
            if (sX >= 0) cp4(&sHal[4 * c][hid], PHi.p[2][0] + zx_of(g, j0 - 1, kk, sX));  // Hz along x
            if (sYh >= 0) {
              const int z = zy_of(g, x, kk, sYh);
              cp4(&sHal[4 * c + 1][hid], PHi.p[2][1] + z);  // Hz along y
              cp4(&sHal[4 * c + 2][hid], PHi.p[0][1] + z);  // Hx along y
            }
          }
          if (sZk >= 0) cp4(&sHal[4 * c + 3][hid], PHi.p[0][2] + zz_of(g, x, j0 - 1, sZk));  // Hx along z
        }
      }
      if (hcol) {
        if constexpr (XY) {
          if (sXc >= 0) {
            const int z = zx_of(g, yc, kk, sXc);
            cp4(&sHal[0][hid], PHi.p[2][0] + z);  // Hz along x
            cp4(&sHal[3][hid], PHi.p[1][0] + z);  // Hy along x
          }
          if (sYc >= 0) cp4(&sHal[1][hid], PHi.p[2][1] + zy_of(g, i0 - 1, kk, sYc));  // Hz along y
        }
        if (sZk >= 0) cp4(&sHal[2][hid], PHi.p[1][2] + zz_of(g, i0 - 1, yc, sZk));  // Hy along z
      }
      cp_commit();
    };
    auto fetch_psiE = [&](int kk, int sZk) {
      if (!XY && sZk < 0) {
        cp_commit();
        return;
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!(c == 0 ? own0 : own1)) continue;
        const int sX = c == 0 ? sX0 : sX1, x = i + c;
        if constexpr (XY) {
          if (wx && sX >= 0) {
            const int z = zx_of(g, j, kk, sX);
            cp4(&sPE[6 * c + 0][tid], PEi.p[1][0] + z);
            cp4(&sPE[6 * c + 1][tid], PEi.p[2][0] + z);
          }
          if (wy && sY >= 0) {
            const int z = zy_of(g, x, kk, sY);
            cp4(&sPE[6 * c + 2][tid], PEi.p[0][1] + z);
            cp4(&sPE[6 * c + 3][tid], PEi.p[2][1] + z);
          }
        }
        if (sZk >= 0) {
          const int z = zz_of(g, x, j, sZk);
          cp4(&sPE[6 * c + 4][tid], PEi.p[0][2] + z);
          cp4(&sPE[6 * c + 5][tid], PEi.p[1][2] + z);
        }
      }
      cp_commit();
    };

    waited &= mbar_wait(&R.bar[0], 0);
    // H^{n+1/2} (x and y components) at the own cells of plane k-1, read by the E update of plane k
    float hxm[2] = {0.f, 0.f}, hym[2] = {0.f, 0.f};
    if (k0 > 0) {
      // plane k0-1 (its owner stores it; this block recomputes it from the staged planes)
      waited &= mbar_wait(&R.bar[1], 0);
      const int km = kb;
      const int sZ = slab_of(km, nz, g.pml[4], g.pml[5]);
      const float(*a0)[EH][EW] = R.E(0);
      const float(*a1)[EH][EW] = R.E(1);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!(c == 0 ? own0 : own1)) continue;
        const int x = i + c, e = ex + c;
        const float dzy = a0[2][ey + 1][e] - a0[2][ey][e], dyz = a1[1][ey][e] - a0[1][ey][e];
        const float dxz = a1[0][ey][e] - a0[0][ey][e], dzx = a0[2][ey][e + 1] - a0[2][ey][e];
        // the CPML terms in the order the owner of plane k0 - 1 adds them (x, y, then z), so that both
        // give the same bits and the result does not depend on the z-chunk
        float cx = dzy - dyz, cy = dxz - dzx;
        if constexpr (XY) {
          const int sX = c == 0 ? sX0 : sX1;
          if (sX >= 0) {
            const Coef cxh = coef_at(tabX, 3, cx0 + c);
            cy -= corr<false>(dzx, cxh.ik, cxh.b, cxh.c, PHi.p[1][0][zx_of(g, j, km, sX)], nullptr, 0);
          }
          if (sY >= 0) {
            const Coef cyh = coef_at(tabY, 3, ry);
            cx += corr<false>(dzy, cyh.ik, cyh.b, cyh.c, PHi.p[0][1][zy_of(g, x, km, sY)], nullptr, 0);
          }
        }
        if (sZ >= 0) {
          const Coef cz{T.b[2][1][km], T.c[2][1][km], T.ik[2][1][km]};
          const int zz = zz_of(g, x, j, sZ);
          cx -= corr<false>(dyz, cz.ik, cz.b, cz.c, PHi.p[0][2][zz], nullptr, 0);
          cy += corr<false>(dxz, cz.ik, cz.b, cz.c, PHi.p[1][2][zz], nullptr, 0);
        }
        hxm[c] = R.H(0)[0][ey][e] - S * cx;
        hym[c] = R.H(0)[1][ey][e] - S * cy;
      }
    }
    int sZ = slab_of(k0, nz, g.pml[4], g.pml[5]);  // z slab index of the current plane (-1 off the layers)
    fetch_psiH(k0, sZ);
    fetch_psiE(k0, sZ);
    // stage of the current plane, of the next one and the mbarrier phase of the next one's fill,
    // advanced by one stage per plane (plane p of the chunk sits in stage (p - kb) % NSTAGE)
    int b0 = (k0 - kb) % NSTAGE;
    int b1 = b0 + 1 == NSTAGE ? 0 : b0 + 1;
    uint32_t ph1 = ((k0 - kb + 1) / NSTAGE) & 1;

    for (int k = k0; k < k1; ++k) {
      const int it = k - kb;  // stage use count of plane k
      const int q = k * plane + q0;
      const int sZn = k + 1 < nz ? slab_of(k + 1, nz, g.pml[4], g.pml[5]) : -1;  // of the next plane
      Coef czh{0.f, 0.f, 1.f}, cze{0.f, 0.f, 1.f};
      if (sZ >= 0) {  // uniform over the block
        czh = Coef{T.b[2][1][k], T.c[2][1][k], T.ik[2][1][k]};
        cze = Coef{T.b[2][0][k], T.c[2][0][k], T.ik[2][0][k]};
      }
      const int pf = pflag[k - k0];
      // soft-source terms of this plane, loaded before the H phase so that their latency overlaps it
      float srcv[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
      if (pf & 1) {
        for (int s = 0; s < A.nsrc; ++s) {
          const SrcDev& sd = A.src[s];
          if (j < sd.lo[1] || j >= sd.hi[1] || k < sd.lo[2] || k >= sd.hi[2]) continue;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int x = i + c;
            if (!(c == 0 ? own0 : own1) || x < sd.lo[0] || x >= sd.hi[0]) continue;
            const float v = sd.w[box_offset(sd.lo, sd.hi, x, j, k)] * sd.g[A.step];
            if (sd.comp == 0) srcv[c][0] += v;
            else if (sd.comp == 1) srcv[c][1] += v;
            else srcv[c][2] += v;
          }
        }
      }
      waited &= mbar_wait(&R.bar[b1], ph1);  // plane k+1 (plane k was waited for before)
      cp_wait_all_but_one();                 // psi_old of H at plane k
      const float(*ek)[EH][EW] = R.E(b0);
      const float(*ek1)[EH][EW] = R.E(b1);
      const float(*hk)[HH][HW] = R.H(b0);
      float(*sH)[HY][HX] = sHb[it & 1];

      // (b) H^{n+1/2} on plane k at the own pair (plain Yee update plus the CPML correction in the
      // layers); E^n and a of the pair stay in registers for the E update
      const float2 exa = ld2(&ek[0][ey][ex]), eya = ld2(&ek[1][ey][ex]), eza = ld2(&ek[2][ey][ex]);
      const float2 av = ld2(&R.Av(b0)[ty][2 * lx]);
      float hx[2] = {0.f, 0.f}, hy[2] = {0.f, 0.f}, hz[2] = {0.f, 0.f};
      if (own0) {
        const float2 exb = ld2(&ek[0][ey + 1][ex]), ezb = ld2(&ek[2][ey + 1][ex]);
        const float2 exc = ld2(&ek1[0][ey][ex]), eyc = ld2(&ek1[1][ey][ex]);
        const float ey2 = ek[1][ey][ex + 2], ez2 = ek[2][ey][ex + 2];
        const float2 hxo = ld2(&hk[0][ey][ex]), hyo = ld2(&hk[1][ey][ex]), hzo = ld2(&hk[2][ey][ex]);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float ex_ = c ? exa.y : exa.x, ey_ = c ? eya.y : eya.x, ez_ = c ? eza.y : eza.x;
          const float dzy = (c ? ezb.y : ezb.x) - ez_, dyz = (c ? eyc.y : eyc.x) - ey_;
          const float dxz = (c ? exc.y : exc.x) - ex_, dzx = (c ? ez2 : eza.y) - ez_;
          const float dyx = (c ? ey2 : eya.y) - ey_, dxy = (c ? exb.y : exb.x) - ex_;
          float cx = dzy - dyz, cy = dxz - dzx, cz = dyx - dxy;
          const int x = i + c;
          const bool ok = c == 0 || own1;  // the cell is in the grid (psi is written only then)
          if constexpr (XY) {
            const int sX = c == 0 ? sX0 : sX1;
            if (wx && sX >= 0 && ok) {
              const Coef cc = coef_at(tabX, 3, cx0 + c);
              const int z = zx_of(g, j, k, sX);
              cy -= corr<true>(dzx, cc.ik, cc.b, cc.c, sPH[6 * c + 0][tid], PHo.p[1][0], z);
              cz += corr<true>(dyx, cc.ik, cc.b, cc.c, sPH[6 * c + 1][tid], PHo.p[2][0], z);
            }
            if (wy && sY >= 0 && ok) {
              const Coef cc = coef_at(tabY, 3, ry);
              const int z = zy_of(g, x, k, sY);
              cx += corr<true>(dzy, cc.ik, cc.b, cc.c, sPH[6 * c + 2][tid], PHo.p[0][1], z);
              cz -= corr<true>(dxy, cc.ik, cc.b, cc.c, sPH[6 * c + 3][tid], PHo.p[2][1], z);
            }
          }
          if (sZ >= 0 && ok) {
            const int z = zz_of(g, x, j, sZ);
            cx -= corr<true>(dyz, czh.ik, czh.b, czh.c, sPH[6 * c + 4][tid], PHo.p[0][2], z);
            cy += corr<true>(dxz, czh.ik, czh.b, czh.c, sPH[6 * c + 5][tid], PHo.p[1][2], z);
          }
          hx[c] = (c ? hxo.y : hxo.x) - S * cx;
          hy[c] = (c ? hyo.y : hyo.x) - S * cy;
          hz[c] = (c ? hzo.y : hzo.x) - S * cz;
        }
        if (!own1) hx[1] = hy[1] = hz[1] = 0.f;  // the pitch padding x >= nx holds zeros
        st2(&sH[0][ry][rx], hx[0], hx[1]);
        st2(&sH[1][ry][rx], hy[0], hy[1]);
        st2(&sH[2][ry][rx], hz[0], hz[1]);
        st2(&N.f[3][q], hx[0], hx[1]);
        st2(&N.f[4][q], hy[0], hy[1]);
        st2(&N.f[5][q], hz[0], hz[1]);
      }
      // the low halo row (i, j0-1), (i+1, j0-1): Hx, Hz
      if (hrow) {
        const float2 exr = ld2(&ek[0][0][ex]), exr1 = ld2(&ek[0][1][ex]);
        const float2 eyr = ld2(&ek[1][0][ex]), eyrk = ld2(&ek1[1][0][ex]);
        const float2 ezr = ld2(&ek[2][0][ex]), ezr1 = ld2(&ek[2][1][ex]);
        const float eyr2 = ek[1][0][ex + 2];
        const float2 hxo = ld2(&hk[0][0][ex]), hzo = ld2(&hk[2][0][ex]);
        float hxr[2], hzr[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float eyv = c ? eyr.y : eyr.x;
          const float dyx = (c ? eyr2 : eyr.y) - eyv, dxy = (c ? exr1.y : exr1.x) - (c ? exr.y : exr.x);
          const float dzy = (c ? ezr1.y : ezr1.x) - (c ? ezr.y : ezr.x), dyz = (c ? eyrk.y : eyrk.x) - eyv;
          float cz = dyx - dxy, cx = dzy - dyz;
          const bool ok = c == 0 || hrow1;  // the halo cell is in the grid (its slots were filled)
          if constexpr (XY) {
            const int sX = c == 0 ? sX0 : sX1;
            if (sX >= 0 && ok) {
              const Coef chx = coef_at(tabX, 3, cx0 + c);
              cz += corr<false>(dyx, chx.ik, chx.b, chx.c, sHal[4 * c][hid], nullptr, 0);
            }
            if (sYh >= 0 && ok) {
              const Coef chy = coef_at(tabY, 3, 0);
              cz -= corr<false>(dxy, chy.ik, chy.b, chy.c, sHal[4 * c + 1][hid], nullptr, 0);
              cx += corr<false>(dzy, chy.ik, chy.b, chy.c, sHal[4 * c + 2][hid], nullptr, 0);
            }
          }
          if (sZ >= 0 && ok) cx -= corr<false>(dyz, czh.ik, czh.b, czh.c, sHal[4 * c + 3][hid], nullptr, 0);
          hzr[c] = (c ? hzo.y : hzo.x) - S * cz;
          hxr[c] = (c ? hxo.y : hxo.x) - S * cx;
        }
        st2(&sH[2][0][rx], hzr[0], hzr[1]);
        st2(&sH[0][0][rx], hxr[0], hxr[1]);
      }
      // the low halo column (i0-1, j0+lx): Hy, Hz
      if (hcol) {
        const int r = lx + 1, c = XO - 1;
        const float dyx = ek[1][r][c + 1] - ek[1][r][c], dxy = ek[0][r + 1][c] - ek[0][r][c];
        const float dxz = ek1[0][r][c] - ek[0][r][c], dzx = ek[2][r][c + 1] - ek[2][r][c];
        float cz = dyx - dxy, cy = dxz - dzx;
        if constexpr (XY) {
          if (sXc >= 0) {
            const Coef chx = coef_at(tabX, 3, 0);
            cz += corr<false>(dyx, chx.ik, chx.b, chx.c, sHal[0][hid], nullptr, 0);
            cy -= corr<false>(dzx, chx.ik, chx.b, chx.c, sHal[3][hid], nullptr, 0);
          }
          if (sYc >= 0) {
            const Coef chy = coef_at(tabY, 3, r);
            cz -= corr<false>(dxy, chy.ik, chy.b, chy.c, sHal[1][hid], nullptr, 0);
          }
        }
        if (sZ >= 0) cy += corr<false>(dxz, czh.ik, czh.b, czh.c, sHal[2][hid], nullptr, 0);
        sH[2][r][1] = hk[2][r][c] - S * cz;
        sH[1][r][1] = hk[1][r][c] - S * cy;
      }
      if (k + 1 < k1) fetch_psiH(k + 1, sZn);
      else cp_commit();
      __syncthreads();
      // the H phase is the last reader of plane k's stage (the E phase works from registers and the
      // new-H tile), so every thread being past it frees the stage for plane k+NSTAGE; on the first
      // plane of a chunk that starts above 0 the stage of plane k0-1 (read by the prologue only) is
      // refilled too
      if (tid == 0) {
        async_proxy_fence();
        if (k == k0 && kb < k0 && kb + NSTAGE <= k1) R.issue(M, 0, i0, j0, kb + NSTAGE);
        if (k + NSTAGE <= k1) R.issue(M, b0, i0, j0, k + NSTAGE);
      }
      cp_wait_all_but_one();  // psi_old of E at plane k

      // (c) E^{n+1} on plane k at the own pair (tangential E on a PEC wall at index 0 is held), then
      // sources and detectors
      float ev[2][3] = {{exa.x, eya.x, eza.x}, {exa.y, eya.y, eza.y}};
      if (own0) {
        const float2 hzs = ld2(&sH[2][ry - 1][rx]), hxs = ld2(&sH[0][ry - 1][rx]);  // at y-1
        const float hyl = sH[1][ry][rx - 1], hzl = sH[2][ry][rx - 1];             // at x-1 of cell 0
        const bool ux = j > 0 && k > 0;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float d1x = hz[c] - (c ? hzs.y : hzs.x), d2x = hy[c] - hym[c];              // E_x: along y, z
          const float d1y = hx[c] - hxm[c], d2y = hz[c] - (c ? hz[0] : hzl);                 // E_y: along z, x
          const float d1z = hy[c] - (c ? hy[0] : hyl), d2z = hx[c] - (c ? hxs.y : hxs.x);  // E_z: along x, y
          float cx = d1x - d2x, cy = d1y - d2y, cz = d1z - d2z;
          const int x = i + c;
          // (a component held by a PEC wall keeps psi = 0: its memory is neither updated nor used)
          const bool uy = x > 0 && k > 0, uz = x > 0 && j > 0;
          const bool ok = c == 0 || own1;
          if constexpr (XY) {
            const int sX = c == 0 ? sX0 : sX1;
            if (wx && sX >= 0 && ok) {
              const Coef cc = coef_at(tabX, 0, cx0 + c);
              const int z = zx_of(g, j, k, sX);
              if (uy) cy -= corr<true>(d2y, cc.ik, cc.b, cc.c, sPE[6 * c + 0][tid], PEo.p[1][0], z);
              if (uz) cz += corr<true>(d1z, cc.ik, cc.b, cc.c, sPE[6 * c + 1][tid], PEo.p[2][0], z);
            }
            if (wy && sY >= 0 && ok) {
              const Coef cc = coef_at(tabY, 0, ry);
              const int z = zy_of(g, x, k, sY);
              if (ux) cx += corr<true>(d1x, cc.ik, cc.b, cc.c, sPE[6 * c + 2][tid], PEo.p[0][1], z);
              if (uz) cz -= corr<true>(d2z, cc.ik, cc.b, cc.c, sPE[6 * c + 3][tid], PEo.p[2][1], z);
            }
          }
          if (sZ >= 0 && ok) {
            const int z = zz_of(g, x, j, sZ);
            if (ux) cx -= corr<true>(d2x, cze.ik, cze.b, cze.c, sPE[6 * c + 4][tid], PEo.p[0][2], z);
            if (uy) cy += corr<true>(d1y, cze.ik, cze.b, cze.c, sPE[6 * c + 5][tid], PEo.p[1][2], z);
          }
          const float Sa = S * (c ? av.y : av.x);
          if (ux) ev[c][0] += Sa * cx;
          if (uy) ev[c][1] += Sa * cy;
          if (uz) ev[c][2] += Sa * cz;
          ev[c][0] += srcv[c][0];
          ev[c][1] += srcv[c][1];
          ev[c][2] += srcv[c][2];
        }
        if (!own1) ev[1][0] = ev[1][1] = ev[1][2] = 0.f;  // the pitch padding x >= nx holds zeros
        st2(&N.f[0][q], ev[0][0], ev[1][0]);
        st2(&N.f[1][q], ev[0][1], ev[1][1]);
        st2(&N.f[2][q], ev[0][2], ev[1][2]);
      }
      // detectors (block-uniform branch; flux partials are reduced over each tile row in a fixed
      // order and summed per row over the planes)
      if (pf & 2) {
#pragma unroll
        for (int s = 0; s < kMaxDet; ++s) {
          if (s >= A.ndet) break;
          const DetDev& d = A.det[s];
          const bool iny = j >= d.lo[1] && j < d.hi[1] && k >= d.lo[2] && k < d.hi[2];
          double f = 0.0;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int x = i + c;
            const bool in = (c == 0 ? own0 : own1) && iny && x >= d.lo[0] && x < d.hi[0];
            const float e0 = ev[c][0], e1 = ev[c][1], e2 = ev[c][2];
            if (d.kind == 0) {
              if (in) A.det_out[d.off + A.step] = (double)(d.comp < 3 ? pick3(d.comp, e0, e1, e2) : pick3(d.comp - 3, hx[c], hy[c], hz[c]));
            } else if (d.kind == 1) {
              if (in) A.det_out[d.off + box_offset(d.lo, d.hi, x, j, k)] += (double)e0 * e0 + (double)e1 * e1 + (double)e2 * e2;
            } else if (in) {
              const int a1 = (d.axis + 1) % 3, a2 = (d.axis + 2) % 3;
              f += (double)pick3(a1, e0, e1, e2) * (double)pick3(a2, hx[c], hy[c], hz[c]) -
                   (double)pick3(a2, e0, e1, e2) * (double)pick3(a1, hx[c], hy[c], hz[c]);
            }
          }
          if (d.kind == 2 && k >= d.lo[2] && k < d.hi[2]) {  // sum over the row's 16 lanes, then one add
#pragma unroll
            for (int o = LX / 2; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o, LX);
            if (lx == 0) wflux[s][ty] += f;
          }
        }
      }
      if (k + 1 < k1) fetch_psiE(k + 1, sZn);
      else cp_commit();
      hxm[0] = hx[0];
      hxm[1] = hx[1];
      hym[0] = hy[0];
      hym[1] = hy[1];
      sZ = sZn;
      b0 = b1;
      b1 = b1 + 1 == NSTAGE ? 0 : b1 + 1;
      if (b1 == 0) ph1 ^= 1u;
    }
  };
  if (tile_xy) march(Flag<true>{});
  else march(Flag<false>{});
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (!waited) atomicOr(A.status, 1);
  __syncthreads();  // every row's flux sums are in place

  // flux detectors: this block's partial sum (row sums in row order) into its slot
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < kMaxDet; ++s) {
      if (s >= A.ndet) break;
      const DetDev& d = A.det[s];
      if (d.kind != 2) continue;
      const int bx0 = d.lo[0] / TX, bx1 = (d.hi[0] - 1) / TX;
      const int by0 = d.lo[1] / TY, by1 = (d.hi[1] - 1) / TY;
      const int bz0 = d.lo[2] / A.tz, bz1 = (d.hi[2] - 1) / A.tz;
      if (bx < bx0 || bx > bx1 || by < by0 || by > by1 || bz < bz0 || bz > bz1) continue;
      double sum = 0.0;
      for (int r = 0; r < TY; ++r) sum += wflux[s][r];
      const int64_t slotid = ((int64_t)(bz - bz0) * (by1 - by0 + 1) + (by - by0)) * (bx1 - bx0 + 1) + (bx - bx0);
      A.partial[d.poff + (int64_t)A.step * d.nblk + slotid] = sum;
    }
  }
}

template <int NSTAGE>
__global__ void __launch_bounds__(NT, 2) k_fwd_fused(const __grid_constant__ FwdArgs A, const __grid_constant__ FwdMaps M) {
  fwd_body<NSTAGE>(A, M, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Several requests in one launch: the grid is the concatenation of their grids (x fastest, then y,
// then the z-chunk), and each block finds its request by the prefix of block counts.
template <int NSTAGE>
__global__ void __launch_bounds__(NT, 2) k_fwd_fused_group(const __grid_constant__ FwdGroup G) {
  int bx, by, bz;
  const int r = group_locate(G.grid, bx, by, bz);
  fwd_body<NSTAGE>(G.a[r], G.m[r], bx, by, bz);
}

}  // namespace

int fused_tile_x() { return TX; }
int fused_max_tz() { return MAXTZ; }
int fused_tile_y() { return TY; }

MapBox fwd_box_e() { return {EW, EH}; }
MapBox fwd_box_h() { return {HW, HH}; }
MapBox fwd_box_a() { return {TX, TY}; }

int prepare_fwd_fused(int nstage, int* blocks_per_sm) {
  auto k = nstage == 4 ? k_fwd_fused<4> : k_fwd_fused<3>;
  auto kg = nstage == 4 ? k_fwd_fused_group<4> : k_fwd_fused_group<3>;
  const int smem = smem_bytes(nstage);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kg, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, NT, smem);
  return e == cudaSuccess ? FDTD_OK : set_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
}

void launch_fwd_group(FwdGroup& G, cudaStream_t s) {
  const int total = group_fill(G.grid, G.n, [&](int r, int* nb) {
    const Geo& g = G.a[r].g;
    nb[0] = (g.n[0] + TX - 1) / TX;
    nb[1] = (g.n[1] + TY - 1) / TY;
    nb[2] = (g.n[2] + G.a[r].tz - 1) / G.a[r].tz;
  });
  if (total == 0) return;
  if (G.a[0].nstage == 4) launch_pdl(k_fwd_fused_group<4>, dim3(total), dim3(NT), smem_bytes(4), s, G);
  else launch_pdl(k_fwd_fused_group<3>, dim3(total), dim3(NT), smem_bytes(3), s, G);
}

void launch_fwd_fused(const FwdArgs& a, const FwdMaps& m, cudaStream_t s) {
  const Geo& g = a.g;
  dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + a.tz - 1) / a.tz);
  if (a.nstage == 4) launch_pdl(k_fwd_fused<4>, grid, dim3(NT), smem_bytes(4), s, a, m);
  else launch_pdl(k_fwd_fused<3>, grid, dim3(NT), smem_bytes(3), s, a, m);
}

}  // namespace fdtd
