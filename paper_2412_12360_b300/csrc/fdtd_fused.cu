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

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int HX = TX + 1, HY = TY + 1;  // new H with the low halo

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
// CPML memories of the plane being computed, copied ahead by each thread for itself (cp.async):
// H slots 0..5 own point (Hy_x, Hz_x, Hx_y, Hz_y, Hx_z, Hy_z), 6..9 the halo point; E slots 0..5.
constexpr int NPH = 10, NPE = 6;
// CPML tables of the tile's x and y positions (from i0-1 and j0-1): b, c, 1/kappa at integer then
// half positions
constexpr int TABX = TX + 1, TABY = TY + 1;
// shared memory: the new-H tiles, the psi slots, tables, flags and flux sums, the mbarriers, then
// the ring of NS stages (3 or 4: more stages keep more planes in flight per block, fewer let more
// blocks reside per SM)
constexpr int SH_OFF = 0;                                         // new H: [2][3][HY][HX] floats
constexpr int PH_OFF = SH_OFF + round128(2 * 3 * HY * HX * 4);    // [NPH][NT]
constexpr int PE_OFF = PH_OFF + NPH * NT * 4;                     // [NPE][NT]
constexpr int TX_OFF = PE_OFF + NPE * NT * 4;                     // [6][TABX]
constexpr int TY_OFF = TX_OFF + 6 * TABX * 4;                     // [6][TABY]
// per-plane flags of the block's z-chunk: bit 0 a source, bit 1 a detector meets the tile at that
// plane (uniform over the block, so planes without either cost one load)
constexpr int MAXTZ = 1024;
constexpr int PF_OFF = TY_OFF + 6 * TABY * 4;                     // [MAXTZ] bytes
constexpr int WF_OFF = round128(PF_OFF + MAXTZ);                  // flux sums per warp: [kMaxDet][NT/32]
constexpr int BAR_OFF = round128(WF_OFF + kMaxDet * (NT / 32) * 8);  // up to 4 mbarriers
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

template <int NSTAGE>
__global__ void __launch_bounds__(NT, NSTAGE == 3 ? 4 : 3) k_fwd_fused(const FwdArgs A, const __grid_constant__ FwdMaps M) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
  Ring R{sm + RING_OFF, reinterpret_cast<uint64_t*>(sm + BAR_OFF)};
  float(*sHb)[3][HY][HX] = reinterpret_cast<float(*)[3][HY][HX]>(sm + SH_OFF);
  float(*sPH)[NT] = reinterpret_cast<float(*)[NT]>(sm + PH_OFF);
  float(*sPE)[NT] = reinterpret_cast<float(*)[NT]>(sm + PE_OFF);
  float(*tabX)[TABX] = reinterpret_cast<float(*)[TABX]>(sm + TX_OFF);
  float(*tabY)[TABY] = reinterpret_cast<float(*)[TABY]>(sm + TY_OFF);
  unsigned char* pflag = sm + PF_OFF;
  double(*wflux)[NT / 32] = reinterpret_cast<double(*)[NT / 32]>(sm + WF_OFF);

  const Geo& g = A.g;
  const Tables& T = A.T;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * A.tz;
  const int k1 = min(g.n[2], k0 + A.tz);
  const int kb = k0 > 0 ? k0 - 1 : k0;  // first plane staged (k0-1 supplies H^{n+1/2} below the chunk)
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int plane = (int)g.plane;
  const int i = i0 + tx, j = j0 + ty;
  const bool own = i < nx && j < ny;
  const int q0 = j * g.nxp + i;
  const float S = g.S;
  const int ex = tx + XO, ey = ty + 1;  // own cell in the staged boxes
  const int rx = tx + 1, ry = ty + 1;   // own cell in the new-H tile
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
    if (tid < kMaxDet * (NT / 32)) wflux[tid / (NT / 32)][tid % (NT / 32)] = 0.0;
  }
  // everything above reads only constant tables and arguments; the fields come after the previous step
  pdl_wait();
  if (tid == 0)
    for (int p = kb; p <= min(kb + NSTAGE - 1, k1); ++p) R.issue(M, p - kb, i0, j0, p);
  __syncthreads();

  // halo H: warp 3 computes the row y = j0-1 (Hx, Hz), warp 4 lanes 0..TY-1 the column x = i0-1 (Hy, Hz)
  const bool hrow = ty == 3 && j0 > 0 && i < nx;
  const bool hcol = ty == 4 && tx < TY && i0 > 0 && (j0 + tx) < ny;
  const int xh = hcol ? i0 - 1 : min(i, nx - 1);
  const int yh = hcol ? j0 + tx : max(j0 - 1, 0);
  const int hrx = hcol ? 0 : tx + 1, hry = hcol ? tx + 1 : 0;  // the halo point in the new-H tile
  const int hex = hrx + XO - 1, hey = hry;                      // and in the staged boxes

  // slab indices along x and y of the own and the halo point (-1 off the layers)
  const int sX = slab_of(min(i, nx - 1), nx, g.pml[0], g.pml[1]);
  const int sY = slab_of(min(j, ny - 1), ny, g.pml[2], g.pml[3]);
  const int sXh = slab_of(xh, nx, g.pml[0], g.pml[1]), sYh = slab_of(yh, ny, g.pml[2], g.pml[3]);
  // whether some lane of this warp has its own cell in an x or a y layer (uniform over the warp, so
  // the per-axis CPML code below is branched over, not predicated, by the warps that have none)
  const bool wx = __any_sync(0xffffffffu, own && sX >= 0);
  const bool wy = __any_sync(0xffffffffu, own && sY >= 0);
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
      if constexpr (XY) {
        if (wx && own && sX >= 0) {
          const int z = zx_of(g, j, kk, sX);
          cp4(&sPH[0][tid], PHi.p[1][0] + z);
          cp4(&sPH[1][tid], PHi.p[2][0] + z);
        }
        if (wy && own && sY >= 0) {
          const int z = zy_of(g, i, kk, sY);
          cp4(&sPH[2][tid], PHi.p[0][1] + z);
          cp4(&sPH[3][tid], PHi.p[2][1] + z);
        }
      }
      if (sZk >= 0 && own) {
        const int z = zz_of(g, i, j, sZk);
        cp4(&sPH[4][tid], PHi.p[0][2] + z);
        cp4(&sPH[5][tid], PHi.p[1][2] + z);
      }
      if ((ty == 3 || ty == 4) && (hrow || hcol)) {
        if constexpr (XY) {
          if (sXh >= 0) cp4(&sPH[6][tid], PHi.p[2][0] + zx_of(g, yh, kk, sXh));  // Hz along x
          if (sYh >= 0) cp4(&sPH[7][tid], PHi.p[2][1] + zy_of(g, xh, kk, sYh));  // Hz along y
          if (hrow && sYh >= 0) cp4(&sPH[8][tid], PHi.p[0][1] + zy_of(g, xh, kk, sYh));  // Hx along y
          if (hcol && sXh >= 0) cp4(&sPH[9][tid], PHi.p[1][0] + zx_of(g, yh, kk, sXh));  // Hy along x
        }
        if (hrow && sZk >= 0) cp4(&sPH[9][tid], PHi.p[0][2] + zz_of(g, xh, yh, sZk));  // Hx along z
        if (hcol && sZk >= 0) cp4(&sPH[8][tid], PHi.p[1][2] + zz_of(g, xh, yh, sZk));  // Hy along z
      }
      cp_commit();
    };
    auto fetch_psiE = [&](int kk, int sZk) {
      if (!XY && sZk < 0) {
        cp_commit();
        return;
      }
      if constexpr (XY) {
        if (wx && own && sX >= 0) {
          const int z = zx_of(g, j, kk, sX);
          cp4(&sPE[0][tid], PEi.p[1][0] + z);
          cp4(&sPE[1][tid], PEi.p[2][0] + z);
        }
        if (wy && own && sY >= 0) {
          const int z = zy_of(g, i, kk, sY);
          cp4(&sPE[2][tid], PEi.p[0][1] + z);
          cp4(&sPE[3][tid], PEi.p[2][1] + z);
        }
      }
      if (sZk >= 0 && own) {
        const int z = zz_of(g, i, j, sZk);
        cp4(&sPE[4][tid], PEi.p[0][2] + z);
        cp4(&sPE[5][tid], PEi.p[1][2] + z);
      }
      cp_commit();
    };

    waited &= mbar_wait(&R.bar[0], 0);
    float hxm = 0.f, hym = 0.f;
    if (k0 > 0) {
      // H^{n+1/2} at (i, j, k0-1), read by the first plane's E update (its owner stores it)
      waited &= mbar_wait(&R.bar[1], 0);
      const int km = kb;
      const int sZ = slab_of(km, nz, g.pml[4], g.pml[5]);
      if (own) {
        const float(*a0)[EH][EW] = R.E(0);
        const float(*a1)[EH][EW] = R.E(1);
        const float dzy = a0[2][ey + 1][ex] - a0[2][ey][ex], dyz = a1[1][ey][ex] - a0[1][ey][ex];
        const float dxz = a1[0][ey][ex] - a0[0][ey][ex], dzx = a0[2][ey][ex + 1] - a0[2][ey][ex];
        float cx = dzy - dyz, cy = dxz - dzx;
        if constexpr (XY) {
          if (sY >= 0) {
            const Coef cyh = coef_at(tabY, 3, ry);
            cx += corr<false>(dzy, cyh.ik, cyh.b, cyh.c, PHi.p[0][1][zy_of(g, i, km, sY)], nullptr, 0);
          }
        }
        if (sZ >= 0) {
          const Coef cz{T.b[2][1][km], T.c[2][1][km], T.ik[2][1][km]};
          const int zz = zz_of(g, i, j, sZ);
          cx -= corr<false>(dyz, cz.ik, cz.b, cz.c, PHi.p[0][2][zz], nullptr, 0);
          cy += corr<false>(dxz, cz.ik, cz.b, cz.c, PHi.p[1][2][zz], nullptr, 0);
        }
        if constexpr (XY) {
          if (sX >= 0) {
            const Coef cxh = coef_at(tabX, 3, rx);
            cy -= corr<false>(dzx, cxh.ik, cxh.b, cxh.c, PHi.p[1][0][zx_of(g, j, km, sX)], nullptr, 0);
          }
        }
        hxm = R.H(0)[0][ey][ex] - S * cx;
        hym = R.H(0)[1][ey][ex] - S * cy;
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
      float sx = 0.f, sy = 0.f, sz = 0.f;
      if (pf & 1) {
        for (int s = 0; s < A.nsrc; ++s) {
          const SrcDev& sd = A.src[s];
          if (!own || i < sd.lo[0] || i >= sd.hi[0] || j < sd.lo[1] || j >= sd.hi[1] || k < sd.lo[2] || k >= sd.hi[2])
            continue;
          const float v = sd.w[box_offset(sd.lo, sd.hi, i, j, k)] * sd.g[A.step];
          if (sd.comp == 0) sx += v;
          else if (sd.comp == 1) sy += v;
          else sz += v;
        }
      }
      waited &= mbar_wait(&R.bar[b1], ph1);  // plane k+1 (plane k was waited for before)
      cp_wait_all_but_one();                                      // psi_old of H at plane k
      const float(*ek)[EH][EW] = R.E(b0);
      const float(*ek1)[EH][EW] = R.E(b1);
      const float(*hk)[HH][HW] = R.H(b0);
      float(*sH)[HY][HX] = sHb[it & 1];

      // (b) H^{n+1/2} on plane k: own cell (plain Yee update plus the CPML correction in the layers)
      float hx = 0.f, hy = 0.f, hz = 0.f;
      if (own) {
        const float dzy = ek[2][ey + 1][ex] - ek[2][ey][ex], dyz = ek1[1][ey][ex] - ek[1][ey][ex];
        const float dxz = ek1[0][ey][ex] - ek[0][ey][ex], dzx = ek[2][ey][ex + 1] - ek[2][ey][ex];
        const float dyx = ek[1][ey][ex + 1] - ek[1][ey][ex], dxy = ek[0][ey + 1][ex] - ek[0][ey][ex];
        float cx = dzy - dyz, cy = dxz - dzx, cz = dyx - dxy;
        if constexpr (XY) {
          if (wx && sX >= 0) {
            const Coef c = coef_at(tabX, 3, rx);
            const int z = zx_of(g, j, k, sX);
            cy -= corr<true>(dzx, c.ik, c.b, c.c, sPH[0][tid], PHo.p[1][0], z);
            cz += corr<true>(dyx, c.ik, c.b, c.c, sPH[1][tid], PHo.p[2][0], z);
          }
          if (wy && sY >= 0) {
            const Coef c = coef_at(tabY, 3, ry);
            const int z = zy_of(g, i, k, sY);
            cx += corr<true>(dzy, c.ik, c.b, c.c, sPH[2][tid], PHo.p[0][1], z);
            cz -= corr<true>(dxy, c.ik, c.b, c.c, sPH[3][tid], PHo.p[2][1], z);
          }
        }
        if (sZ >= 0) {
          const int z = zz_of(g, i, j, sZ);
          cx -= corr<true>(dyz, czh.ik, czh.b, czh.c, sPH[4][tid], PHo.p[0][2], z);
          cy += corr<true>(dxz, czh.ik, czh.b, czh.c, sPH[5][tid], PHo.p[1][2], z);
        }
        hx = hk[0][ey][ex] - S * cx;
        hy = hk[1][ey][ex] - S * cy;
        hz = hk[2][ey][ex] - S * cz;
        sH[0][ry][rx] = hx;
        sH[1][ry][rx] = hy;
        sH[2][ry][rx] = hz;
        N.f[3][q] = hx;
        N.f[4][q] = hy;
        N.f[5][q] = hz;
      }
      // the low halo: (i, j0-1) gives Hx, Hz; (i0-1, j0+r) gives Hy, Hz
      if ((ty == 3 || ty == 4) && (hrow || hcol)) {
        const int r = hey, c = hex;
        const float dyx = ek[1][r][c + 1] - ek[1][r][c], dxy = ek[0][r + 1][c] - ek[0][r][c];
        float cz = dyx - dxy;
        if constexpr (XY) {
          if (sXh >= 0) {
            const Coef chx = coef_at(tabX, 3, hrx);
            cz += corr<false>(dyx, chx.ik, chx.b, chx.c, sPH[6][tid], nullptr, 0);
          }
          if (sYh >= 0) {
            const Coef chy = coef_at(tabY, 3, hry);
            cz -= corr<false>(dxy, chy.ik, chy.b, chy.c, sPH[7][tid], nullptr, 0);
          }
        }
        sH[2][hry][hrx] = hk[2][r][c] - S * cz;
        if (hrow) {  // Hx
          const float dzy = ek[2][r + 1][c] - ek[2][r][c], dyz = ek1[1][r][c] - ek[1][r][c];
          float cx = dzy - dyz;
          if constexpr (XY) {
            if (sYh >= 0) {
              const Coef chy = coef_at(tabY, 3, hry);
              cx += corr<false>(dzy, chy.ik, chy.b, chy.c, sPH[8][tid], nullptr, 0);
            }
          }
          if (sZ >= 0) cx -= corr<false>(dyz, czh.ik, czh.b, czh.c, sPH[9][tid], nullptr, 0);
          sH[0][hry][hrx] = hk[0][r][c] - S * cx;
        } else {  // Hy
          const float dxz = ek1[0][r][c] - ek[0][r][c], dzx = ek[2][r][c + 1] - ek[2][r][c];
          float cy = dxz - dzx;
          if (sZ >= 0) cy += corr<false>(dxz, czh.ik, czh.b, czh.c, sPH[8][tid], nullptr, 0);
          if constexpr (XY) {
            if (sXh >= 0) {
              const Coef chx = coef_at(tabX, 3, hrx);
              cy -= corr<false>(dzx, chx.ik, chx.b, chx.c, sPH[9][tid], nullptr, 0);
            }
          }
          sH[1][hry][hrx] = hk[1][r][c] - S * cy;
        }
      }
      if (k + 1 < k1) fetch_psiH(k + 1, sZn);
      else cp_commit();
      __syncthreads();
      // every thread is past plane k-1, so its stage can take plane k-1+NSTAGE
      if (tid == 0 && it >= 1 && k - 1 + NSTAGE <= k1) {
        async_proxy_fence();
        R.issue(M, b0 == 0 ? NSTAGE - 1 : b0 - 1, i0, j0, k - 1 + NSTAGE);  // the stage of plane k-1
      }
      cp_wait_all_but_one();  // psi_old of E at plane k

      // (c) E^{n+1} on plane k at the own cell (tangential E on a PEC wall at index 0 is held), then
      // sources and detectors
      float exv = 0.f, eyv = 0.f, ezv = 0.f;
      if (own) {
        const float Sa = S * R.Av(b0)[ty][tx];
        exv = ek[0][ey][ex];
        eyv = ek[1][ey][ex];
        ezv = ek[2][ey][ex];
        const float d1x = hz - sH[2][ry - 1][rx], d2x = hy - hym;   // E_x: along y, along z
        const float d1y = hx - hxm, d2y = hz - sH[2][ry][rx - 1];   // E_y: along z, along x
        const float d1z = hy - sH[1][ry][rx - 1], d2z = hx - sH[0][ry - 1][rx];  // E_z: along x, along y
        float cx = d1x - d2x, cy = d1y - d2y, cz = d1z - d2z;
        // (a component held by a PEC wall keeps psi = 0: its memory is neither updated nor used)
        const bool ux = j > 0 && k > 0, uy = i > 0 && k > 0, uz = i > 0 && j > 0;
        if constexpr (XY) {
          if (wx && sX >= 0) {
            const Coef c = coef_at(tabX, 0, rx);
            const int z = zx_of(g, j, k, sX);
            if (uy) cy -= corr<true>(d2y, c.ik, c.b, c.c, sPE[0][tid], PEo.p[1][0], z);
            if (uz) cz += corr<true>(d1z, c.ik, c.b, c.c, sPE[1][tid], PEo.p[2][0], z);
          }
          if (wy && sY >= 0) {
            const Coef c = coef_at(tabY, 0, ry);
            const int z = zy_of(g, i, k, sY);
            if (ux) cx += corr<true>(d1x, c.ik, c.b, c.c, sPE[2][tid], PEo.p[0][1], z);
            if (uz) cz -= corr<true>(d2z, c.ik, c.b, c.c, sPE[3][tid], PEo.p[2][1], z);
          }
        }
        if (sZ >= 0) {
          const int z = zz_of(g, i, j, sZ);
          if (ux) cx -= corr<true>(d2x, cze.ik, cze.b, cze.c, sPE[4][tid], PEo.p[0][2], z);
          if (uy) cy += corr<true>(d1y, cze.ik, cze.b, cze.c, sPE[5][tid], PEo.p[1][2], z);
        }
        if (j > 0 && k > 0) exv += Sa * cx;
        if (i > 0 && k > 0) eyv += Sa * cy;
        if (i > 0 && j > 0) ezv += Sa * cz;
        exv += sx;
        eyv += sy;
        ezv += sz;
        N.f[0][q] = exv;
        N.f[1][q] = eyv;
        N.f[2][q] = ezv;
      }
      // detectors (block-uniform branch; flux partials are reduced over the warp in a fixed order and
      // summed per warp over the planes)
      if (pf & 2) {
  #pragma unroll
        for (int s = 0; s < kMaxDet; ++s) {
          if (s >= A.ndet) break;
          const DetDev& d = A.det[s];
          const bool in = own && i >= d.lo[0] && i < d.hi[0] && j >= d.lo[1] && j < d.hi[1] && k >= d.lo[2] && k < d.hi[2];
          if (d.kind == 0) {
            if (in) A.det_out[d.off + A.step] = (double)(d.comp < 3 ? pick3(d.comp, exv, eyv, ezv) : pick3(d.comp - 3, hx, hy, hz));
          } else if (d.kind == 1) {
            if (in) A.det_out[d.off + box_offset(d.lo, d.hi, i, j, k)] += (double)exv * exv + (double)eyv * eyv + (double)ezv * ezv;
          } else if (k >= d.lo[2] && k < d.hi[2]) {
            const int a1 = (d.axis + 1) % 3, a2 = (d.axis + 2) % 3;
            double f = in ? (double)pick3(a1, exv, eyv, ezv) * (double)pick3(a2, hx, hy, hz) -
                                (double)pick3(a2, exv, eyv, ezv) * (double)pick3(a1, hx, hy, hz)
                          : 0.0;
            if (d.axis == 0) {  // an x-normal plane holds at most one lane of each warp
              if (in) wflux[s][ty] += f;
            } else {
  #pragma unroll
              for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
              if (tx == 0) wflux[s][ty] += f;
            }
          }
        }
      }
      if (k + 1 < k1) fetch_psiE(k + 1, sZn);
      else cp_commit();
      hxm = hx;
      hym = hy;
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
  __syncthreads();  // every warp's flux sums are in place

  // flux detectors: this block's partial sum (warp sums in warp order) into its slot
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < kMaxDet; ++s) {
      if (s >= A.ndet) break;
      const DetDev& d = A.det[s];
      if (d.kind != 2) continue;
      const int bx0 = d.lo[0] / TX, bx1 = (d.hi[0] - 1) / TX;
      const int by0 = d.lo[1] / TY, by1 = (d.hi[1] - 1) / TY;
      const int bz0 = d.lo[2] / A.tz, bz1 = (d.hi[2] - 1) / A.tz;
      const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
      if (bx < bx0 || bx > bx1 || by < by0 || by > by1 || bz < bz0 || bz > bz1) continue;
      double sum = 0.0;
      for (int w = 0; w < NT / 32; ++w) sum += wflux[s][w];
      const int64_t slotid = ((int64_t)(bz - bz0) * (by1 - by0 + 1) + (by - by0)) * (bx1 - bx0 + 1) + (bx - bx0);
      A.partial[d.poff + (int64_t)A.step * d.nblk + slotid] = sum;
    }
  }
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
  const int smem = smem_bytes(nstage);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, NT, smem);
  return e == cudaSuccess ? FDTD_OK : set_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
}

void launch_fwd_fused(const FwdArgs& a, const FwdMaps& m, cudaStream_t s) {
  const Geo& g = a.g;
  dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + a.tz - 1) / a.tz);
  if (a.nstage == 4) launch_pdl(k_fwd_fused<4>, grid, dim3(NT), smem_bytes(4), s, a, m);
  else launch_pdl(k_fwd_fused<3>, grid, dim3(NT), smem_bytes(3), s, a, m);
}

}  // namespace fdtd
