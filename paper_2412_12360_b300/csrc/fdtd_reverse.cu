// Reverse step of arXiv 2412.12360 Sec. 2.2 as two z-marching kernels, in place:
//
//   rev_E(n): the inverse E update E^n = E^{n+1} - src - S a curl_b(H^{n+1/2}) on the PML-free region R,
//             dL/da += S Ebar . curl_b(H^{n+1/2}) on the design box, and the transpose of the E update
//             for the adjoint: Hbar += sum of the E-update coefficients P of the neighbouring E points
//             (with the CPML memories psi-bar of E);
//   rev_H(n): the inverse H update H^{n-1/2} = H^{n+1/2} + S curl_f(E^n) on R, and the transpose of the
//             H update: Ebar += sum of the H-update coefficients Q of the neighbouring H points,
//             plus the adjoints of the detectors of step n-1 that read only E (E^n, held here), which
//             would otherwise take a launch of their own at the start of reverse step n-1.
//
// Each kernel reads only fields it does not write (rev_E reads H and Ebar and writes E and Hbar;
// rev_H reads E and Hbar and writes H and Ebar), so in-place updates are race-free. Blocks own a
// TX x TY column tile and march their z-chunk downwards, so the coefficient of the plane above is
// carried in registers. The tangential H recorded on the six boundary planes (Sec. 2.2) is written
// back into H by a copy kernel before each rev_E. With RevArgs::inverse = 0 (the checkpointing
// gradient, whose forward states are recomputed) the kernels leave the forward fields untouched and
// update only the adjoint fields and dL/da.
//
// The adjoint coefficients of one E point (component c, its transverse axes c1 = c+1, c2 = c+2):
//   u = S a Ebar_c (zero where E_c is held by a PEC wall),
//   P1 = u / kappa_c1 + c_c1 (psibar_c,c1 + u),   P2 = -u / kappa_c2 + c_c2 (psibar_c,c2 - u),
//   psibar_c,c1 <- b_c1 (psibar_c,c1 + u),       psibar_c,c2 <- b_c2 (psibar_c,c2 - u),
// and Hbar_h(p) += P1_{h+1}(p) - P1_{h+1}(p + e_{h+2}) + P2_{h+2}(p) - P2_{h+2}(p + e_{h+1}).
// Those of one H point mirror them with w = -S Hbar_h and the H tables, giving
//   Ebar_e(p) += Q1_{e+1}(p - e_{e+2}) - Q1_{e+1}(p) + Q2_{e+2}(p - e_{e+1}) - Q2_{e+2}(p).
// Off the layers 1/kappa = 1 and c = 0, so P and Q reduce to +-u and +-w: the kernels gather those
// plain values for every point and add, for each axis d whose layer holds the point or the
// neighbour along d, the correction sgn v (1/kappa_d - 1) + c_d (psibar + sgn v) of the coefficients
// along d (exactly 0 on the layer's inner edge).
#include <algorithm>

#include "../../include/fdtd.h"
#include "fdtd_internal.cuh"
#include "fdtd_tma.cuh"

namespace fdtd {

namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;

__device__ __forceinline__ int zx_of(const Geo& g, int y, int k, int s) { return (k * g.n[1] + y) * g.slab[0] + s; }
__device__ __forceinline__ int zy_of(const Geo& g, int x, int k, int s) { return (k * g.slab[1] + s) * g.nxp + x; }
__device__ __forceinline__ int zz_of(const Geo& g, int x, int y, int s) { return (s * g.n[1] + y) * g.nxp + x; }

// psi index of (x, y, k) for the derivative along axis D with slab index s
template <int D>
__device__ __forceinline__ int zd_of(const Geo& g, int x, int y, int k, int s) {
  return D == 0 ? zx_of(g, y, k, s) : (D == 1 ? zy_of(g, x, k, s) : zz_of(g, x, y, s));
}

// CPML part of one adjoint coefficient inside a layer: the coefficient is sv / kappa + c (psi + sv)
// (sv = sgn v), its plain value off the layers sv.
__device__ __forceinline__ float acorr(float sv, float ik, float c, float psi) { return sv * (ik - 1.f) + c * (psi + sv); }

__device__ __forceinline__ int box_offset(const int lo[3], const int hi[3], int x, int y, int k) {
  return ((k - lo[2]) * (hi[1] - lo[1]) + (y - lo[1])) * (hi[0] - lo[0]) + (x - lo[0]);
}

// ---------------------------------------------------------------------------------------------
// Plane staging. Both kernels march their z-chunk downwards and read every plane through a ring of
// NS shared-memory stages filled by TMA bulk tensor copies (one elected thread issues them; the
// block waits on one mbarrier per stage). Two box shapes are used: "own" boxes are the tile itself
// (TX x TY at (i0, j0)); "wide" boxes add one cell on one side in x and y (BW x BH), either on the
// high side (origin (i0, j0): the +x, +y neighbours) or on the low side (origin (i0-4, j0-1), 4 cells
// to the left so the copy's x coordinate stays 16-byte aligned: the -x, -y neighbours). Outside the
// grid the copies read 0, which is what the PEC walls and the zero adjoint give.
// ---------------------------------------------------------------------------------------------
constexpr int BW = TX + 4, BH = TY + 1;
// NS = stages of the ring: 4 (three blocks per SM) on grids that fill several waves of blocks, 3
// (four blocks per SM, so that the short z-chunks of small grids run side by side) otherwise
constexpr int round128(int b) { return (b + 127) / 128 * 128; }
constexpr uint32_t OWN3 = 3 * TX * TY * 4, WIDE3 = 3 * BW * BH * 4, WIDE1 = BW * BH * 4;

// rev_E stage: H (wide, low side), E (own), Ebar (wide, high side), Hbar (own), a (wide, high side)
constexpr int RE_H = 0, RE_E = RE_H + round128(WIDE3), RE_EB = RE_E + round128(OWN3),
              RE_HB = RE_EB + round128(WIDE3), RE_A = RE_HB + round128(OWN3), RE_STAGE = RE_A + round128(WIDE1);
constexpr uint32_t RE_TX = WIDE3 + OWN3 + WIDE3 + OWN3 + WIDE1;
// rev_H stage: E (wide, high side), H (own), Hbar (wide, low side), Ebar (own)
constexpr int RH_E = 0, RH_H = RH_E + round128(WIDE3), RH_HB = RH_H + round128(OWN3),
              RH_EB = RH_HB + round128(WIDE3), RH_STAGE = RH_EB + round128(OWN3);
constexpr uint32_t RH_TX = WIDE3 + OWN3 + WIDE3 + OWN3;

constexpr int re_smem(int ns) { return ns * RE_STAGE + ns * 8 + 128; }
constexpr int rh_smem(int ns) { return ns * RH_STAGE + ns * 8 + 128; }

typedef const float (*Own3)[TY][TX];
typedef const float (*Wide3)[BH][BW];
typedef const float (*Wide1)[BW];

// Stage ring of a downward march over planes ktop, ktop-1, ..., kbot: plane p is use number
// (ktop - p) / NS of stage (ktop - p) % NS.
template <int NS>
struct DownRing {
  unsigned char* base;
  uint64_t* bar;
  int stage_bytes, ktop;
  __device__ unsigned char* at(int p) const { return base + ((ktop - p) % NS) * stage_bytes; }
  __device__ uint64_t* bar_of(int p) const { return &bar[(ktop - p) % NS]; }
  __device__ bool wait(int p) const { return mbar_wait(bar_of(p), ((ktop - p) / NS) & 1); }
};

__device__ __forceinline__ unsigned char* align128(unsigned char* p) {
  return p + ((128 - (smem_addr(p) & 127)) & 127);
}

template <class Ring>
__device__ __forceinline__ void issue_rev_E(const RevMaps& M, const Ring& R, int i0, int j0, int p) {
  unsigned char* st = R.at(p);
  uint64_t* b = R.bar_of(p);
  mbar_arrive_expect(b, RE_TX);
  tma_load_box(st + RE_H, &M.h_low, i0 - 4, j0 - 1, p, 0, b);
  tma_load_box(st + RE_E, &M.e_own, i0, j0, p, 0, b);
  tma_load_box(st + RE_EB, &M.eb_high, i0, j0, p, 0, b);
  tma_load_box(st + RE_HB, &M.hb_own, i0, j0, p, 0, b);
  tma_load_box(st + RE_A, &M.a_high, i0, j0, p, 0, b);
}

template <class Ring>
__device__ __forceinline__ void issue_rev_H(const RevMaps& M, const Ring& R, int i0, int j0, int p) {
  unsigned char* st = R.at(p);
  uint64_t* b = R.bar_of(p);
  mbar_arrive_expect(b, RH_TX);
  tma_load_box(st + RH_E, &M.e_high, i0, j0, p, 0, b);
  tma_load_box(st + RH_H, &M.h_own, i0, j0, p, 0, b);
  tma_load_box(st + RH_HB, &M.hb_low, i0 - 4, j0 - 1, p, 0, b);
  tma_load_box(st + RH_EB, &M.eb_own, i0, j0, p, 0, b);
}

// ---------------------------------------------------------------------------------------------
// rev_E
// ---------------------------------------------------------------------------------------------
template <int NSTAGE>
__device__ __forceinline__ void revE_body(const RevArgs& A, const RevMaps& M, const int bx, const int by, const int bz) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = align128(smem_raw);

  const Geo& g = A.g;
  const Tables& T = A.T;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int i0 = bx * TX, j0 = by * TY;
  const int k0 = bz * A.tz;
  const int k1 = min(g.n[2], k0 + A.tz);
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int plane = (int)g.plane;
  const int i = i0 + tx, j = j0 + ty;
  const bool own = i < nx && j < ny;
  const int q0 = j * g.nxp + i;
  const float S = g.S;
  const int ktop = k1 - 1, kbot = max(k0 - 1, 0);  // planes staged: H(k-1) is read below the chunk
  const DownRing<NSTAGE> R{sm, reinterpret_cast<uint64_t*>(sm + NSTAGE * RE_STAGE), RE_STAGE, ktop};
  bool waited = true;

  pdl_wait();  // the fields come after the previous kernel of the stream
  if (tid == 0) {
    for (int b = 0; b < NSTAGE; ++b) mbar_init(&R.bar[b], 1);
    mbar_init_fence();
    for (int p = ktop; p >= max(ktop - NSTAGE + 1, kbot); --p) issue_rev_E(M, R, i0, j0, p);
  }
  __syncthreads();

  // CPML data (integer positions, the E tables) along x and y
  const int ic = min(i, nx - 1), jc = min(j, ny - 1);
  const float ikX0 = T.ik[0][0][ic], ikY0 = T.ik[1][0][jc];
  const int sX0 = T.sidx[0][ic], sY0 = T.sidx[1][jc];
  const bool hasX1 = i + 1 < nx, hasY1 = j + 1 < ny;
  const float ikX1 = T.ik[0][0][min(i + 1, nx - 1)], ikY1 = T.ik[1][0][min(j + 1, ny - 1)];
  const int sX1 = hasX1 ? T.sidx[0][i + 1] : -1, sY1 = hasY1 ? T.sidx[1][j + 1] : -1;

  // R membership of the own E components along x and y (E_c: half along c, integer along the others)
  const bool rxh = i >= g.rhalf_lo[0] && i <= g.rhalf_hi[0], rxi = i >= g.rint_lo[0] && i <= g.rint_hi[0];
  const bool ryh = j >= g.rhalf_lo[1] && j <= g.rhalf_hi[1], ryi = j >= g.rint_lo[1] && j <= g.rint_hi[1];
  const bool dxy = own && i >= A.dlo[0] && i < A.dhi[0] && j >= A.dlo[1] && j < A.dhi[1];
  unsigned src_xy = 0;
  for (int s = 0; s < A.nsrc; ++s)
    if (own && i >= A.src[s].lo[0] && i < A.src[s].hi[0] && j >= A.src[s].lo[1] && j < A.src[s].hi[1]) src_xy |= 1u << s;

  const PsiSet& Pi = A.pin;
  const PsiSet& Po = A.pout;

  // u_y, u_x of the own column at k1 (the plane above the chunk) and the z-layer corrections of
  // P1 of E_y and P2 of E_x there
  float uy_up = 0.f, ux_up = 0.f, d1y_up = 0.f, d2x_up = 0.f;
  if (own && k1 < nz) {
    const int q = k1 * plane + q0;
    const float Sa = S * A.a[q];
    ux_up = (j > 0) ? Sa * A.B.f[0][q] : 0.f;
    uy_up = (i > 0) ? Sa * A.B.f[1][q] : 0.f;
    const int sZ = T.sidx[2][k1];
    if (sZ >= 0) {
      const int zz = zz_of(g, i, j, sZ);
      const float ikZ = T.ik[2][0][k1], cZ = T.c[2][0][k1];
      d1y_up = acorr(uy_up, ikZ, cZ, Pi.p[1][2][zz]);
      d2x_up = acorr(-ux_up, ikZ, cZ, Pi.p[0][2][zz]);
    }
  }

  waited &= R.wait(ktop);
  int sZ1 = (k1 < nz) ? T.sidx[2][k1] : -1;  // slab index of the plane above
  for (int k = ktop; k >= k0; --k) {
    const int q = k * plane + q0;
    if (k - 1 >= kbot) waited &= R.wait(k - 1);
    __syncthreads();  // every thread is past plane k+1
    if (tid == 0 && k + 1 <= ktop && k + 1 - NSTAGE >= kbot) {
      async_proxy_fence();
      issue_rev_E(M, R, i0, j0, k + 1 - NSTAGE);
    }
    if (!own) continue;
    const unsigned char* st = R.at(k);
    const Wide3 Hs = reinterpret_cast<Wide3>(st + RE_H);
    const Own3 Es = reinterpret_cast<Own3>(st + RE_E);
    const Wide3 Bs = reinterpret_cast<Wide3>(st + RE_EB);
    const Own3 Gs = reinterpret_cast<Own3>(st + RE_HB);
    const Wide1 As = reinterpret_cast<Wide1>(st + RE_A);
    const float hx = Hs[0][ty + 1][tx + 4], hy = Hs[1][ty + 1][tx + 4], hz = Hs[2][ty + 1][tx + 4];
    float hxm = 0.f, hym = 0.f;
    if (k > 0) {
      const Wide3 Hm = reinterpret_cast<Wide3>(R.at(k - 1) + RE_H);
      hxm = Hm[0][ty + 1][tx + 4];
      hym = Hm[1][ty + 1][tx + 4];
    }
    const float bx = Bs[0][ty][tx], by = Bs[1][ty][tx], bz = Bs[2][ty][tx];
    const float Sa = S * As[ty][tx];
    const float ux = (j > 0 && k > 0) ? Sa * bx : 0.f;
    const float uy = (i > 0 && k > 0) ? Sa * by : 0.f;
    const float uz = (i > 0 && j > 0) ? Sa * bz : 0.f;
    // u of the +x neighbour (z and y) and of the +y neighbour (z and x); 0 beyond the grid
    const float Sax = S * As[ty][tx + 1], Say = S * As[ty + 1][tx];
    const float uz_x = (j > 0) ? Sax * Bs[2][ty][tx + 1] : 0.f, uy_x = (k > 0) ? Sax * Bs[1][ty][tx + 1] : 0.f;
    const float uz_y = (i > 0) ? Say * Bs[2][ty + 1][tx] : 0.f, ux_y = (k > 0) ? Say * Bs[0][ty + 1][tx] : 0.f;
    const float gx = Gs[0][ty][tx], gy = Gs[1][ty][tx], gz = Gs[2][ty][tx];
    float ex = Es[0][ty][tx], ey = Es[1][ty][tx], ez = Es[2][ty][tx];

    const float ikZ = T.ik[2][0][k];
    const int sZ = T.sidx[2][k];

    // adjoint gather into H-bar: the plain coefficients +-u of the own E point and of its +x, +y, +z
    // neighbours, then the CPML corrections axis by axis
    float hbx = (uy - uy_up) + (-uz + uz_y);
    float hby = (uz - uz_x) + (-ux + ux_up);
    float hbz = (ux - ux_y) + (-uy + uy_x);
    float cbx = 0.f, cby = 0.f, cbz = 0.f;
    if (sX0 >= 0 || sX1 >= 0) {  // along x: P1 of E_z (2,0) and P2 of E_y (1,0), own and +x
      float c1z = 0.f, c2y = 0.f, n1z = 0.f, n2y = 0.f;
      if (sX0 >= 0) {
        const int z = zx_of(g, j, k, sX0);
        const float cX = T.c[0][0][i], bX = T.b[0][0][i];
        const float p20 = Pi.p[2][0][z], p10 = Pi.p[1][0][z];
        c1z = acorr(uz, ikX0, cX, p20);
        c2y = acorr(-uy, ikX0, cX, p10);
        Po.p[2][0][z] = bX * (p20 + uz);
        Po.p[1][0][z] = bX * (p10 - uy);
      }
      if (sX1 >= 0) {
        const int z = zx_of(g, j, k, sX1);
        const float cX = T.c[0][0][i + 1];
        n1z = acorr(uz_x, ikX1, cX, Pi.p[2][0][z]);
        n2y = acorr(-uy_x, ikX1, cX, Pi.p[1][0][z]);
      }
      cby += c1z - n1z;
      cbz += c2y - n2y;
    }
    if (sY0 >= 0 || sY1 >= 0) {  // along y: P1 of E_x (0,1) and P2 of E_z (2,1), own and +y
      float c1x = 0.f, c2z = 0.f, n1x = 0.f, n2z = 0.f;
      if (sY0 >= 0) {
        const int z = zy_of(g, i, k, sY0);
        const float cY = T.c[1][0][j], bY = T.b[1][0][j];
        const float p01 = Pi.p[0][1][z], p21 = Pi.p[2][1][z];
        c1x = acorr(ux, ikY0, cY, p01);
        c2z = acorr(-uz, ikY0, cY, p21);
        Po.p[0][1][z] = bY * (p01 + ux);
        Po.p[2][1][z] = bY * (p21 - uz);
      }
      if (sY1 >= 0) {
        const int z = zy_of(g, i, k, sY1);
        const float cY = T.c[1][0][j + 1];
        n1x = acorr(ux_y, ikY1, cY, Pi.p[0][1][z]);
        n2z = acorr(-uz_y, ikY1, cY, Pi.p[2][1][z]);
      }
      cbx += c2z - n2z;
      cbz += c1x - n1x;
    }
    float d1y = 0.f, d2x = 0.f;  // along z: P1 of E_y (1,2) and P2 of E_x (0,2), own (below: carried)
    if (sZ >= 0 || sZ1 >= 0) {
      if (sZ >= 0) {
        const int z = zz_of(g, i, j, sZ);
        const float cZ = T.c[2][0][k], bZ = T.b[2][0][k];
        const float p12 = Pi.p[1][2][z], p02 = Pi.p[0][2][z];
        d1y = acorr(uy, ikZ, cZ, p12);
        d2x = acorr(-ux, ikZ, cZ, p02);
        Po.p[1][2][z] = bZ * (p12 + uy);
        Po.p[0][2][z] = bZ * (p02 - ux);
      }
      cbx += d1y - d1y_up;
      cby += d2x - d2x_up;
    }
    A.B.f[3][q] = gx + (hbx + cbx);
    A.B.f[4][q] = gy + (hby + cby);
    A.B.f[5][q] = gz + (hbz + cbz);
    uy_up = uy;
    ux_up = ux;
    d1y_up = d1y;
    d2x_up = d2x;
    sZ1 = sZ;

    // inverse E update on R (mirrors the forward arithmetic: the curl difference times 1/kappa = 1)
    const float dxa = hz - Hs[2][ty][tx + 4], dxb = hy - hym;       // E_x: along y, along z
    const float dya = hx - hxm, dyb = hz - Hs[2][ty + 1][tx + 3];   // E_y: along z, along x
    const float dza = hy - Hs[1][ty + 1][tx + 3], dzb = hx - Hs[0][ty][tx + 4];  // E_z: along x, along y
    const bool rzh = k >= g.rhalf_lo[2] && k <= g.rhalf_hi[2], rzi = k >= g.rint_lo[2] && k <= g.rint_hi[2];
    const bool inx = rxh && ryi && rzi && j > 0 && k > 0;
    const bool iny = rxi && ryh && rzi && i > 0 && k > 0;
    const bool inz = rxi && ryi && rzh && i > 0 && j > 0;
    if (src_xy) {
      unsigned src_k = 0;
      for (int s = 0; s < A.nsrc; ++s) src_k |= (k >= A.src[s].lo[2] && k < A.src[s].hi[2]) ? 1u << s : 0u;
      if (src_xy & src_k) {
        for (int s = 0; s < A.nsrc; ++s) {
          const SrcDev& sd = A.src[s];
          if (!(((src_xy & src_k) >> s) & 1u)) continue;
          const float v = sd.w[box_offset(sd.lo, sd.hi, i, j, k)] * sd.g[A.step];
          if (sd.comp == 0 && inx) ex -= v;
          else if (sd.comp == 1 && iny) ey -= v;
          else if (sd.comp == 2 && inz) ez -= v;
        }
      }
    }
    if (inx) ex -= Sa * (dxa * ikY0 - dxb * ikZ);
    if (iny) ey -= Sa * (dya * ikZ - dyb * ikX0);
    if (inz) ez -= Sa * (dza * ikX0 - dzb * ikY0);
    if (A.inverse) {
      A.F.f[0][q] = ex;
      A.F.f[1][q] = ey;
      A.F.f[2][q] = ez;
    }
    // dL/da on the design box (inside R: kappa = 1, psi = 0)
    if (dxy && k >= A.dlo[2] && k < A.dhi[2]) {
      float gs = 0.f;
      if (j > 0 && k > 0) gs += bx * (dxa - dxb);
      if (i > 0 && k > 0) gs += by * (dya - dyb);
      if (i > 0 && j > 0) gs += bz * (dza - dzb);
      const int m = ((k - A.dlo[2]) * (A.dhi[1] - A.dlo[1]) + (j - A.dlo[1])) * (A.dhi[0] - A.dlo[0]) + (i - A.dlo[0]);
      A.dLda[m] += (double)S * (double)gs;
    }
  }
  if (!waited) atomicOr(A.status, 1);
}

// ---------------------------------------------------------------------------------------------
// rev_H
// ---------------------------------------------------------------------------------------------
template <int NSTAGE>
__device__ __forceinline__ void revH_body(const RevArgs& A, const RevMaps& M, const int bx, const int by, const int bz) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = align128(smem_raw);

  const Geo& g = A.g;
  const Tables& T = A.T;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int i0 = bx * TX, j0 = by * TY;
  const int k0 = bz * A.tz;
  const int k1 = min(g.n[2], k0 + A.tz);
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int plane = (int)g.plane;
  const int i = i0 + tx, j = j0 + ty;
  const bool own = i < nx && j < ny;
  const int q0 = j * g.nxp + i;
  const float S = g.S;
  const int ktop = k1 - 1, kbot = max(k0 - 1, 0);  // planes staged: Hbar(k-1) is read below the chunk
  const DownRing<NSTAGE> R{sm, reinterpret_cast<uint64_t*>(sm + NSTAGE * RH_STAGE), RH_STAGE, ktop};
  bool waited = true;

  pdl_wait();  // the fields come after the previous kernel of the stream
  if (tid == 0) {
    for (int b = 0; b < NSTAGE; ++b) mbar_init(&R.bar[b], 1);
    mbar_init_fence();
    for (int p = ktop; p >= max(ktop - NSTAGE + 1, kbot); --p) issue_rev_H(M, R, i0, j0, p);
  }
  __syncthreads();

  // CPML data (half positions, the H tables) along x and y, at the own column and at -x, -y
  const int ic = min(i, nx - 1), jc = min(j, ny - 1);
  const float ikX0 = T.ik[0][1][ic], ikY0 = T.ik[1][1][jc];
  const int sX0 = T.sidx[0][ic], sY0 = T.sidx[1][jc];
  const bool hasXm = i > 0, hasYm = j > 0;
  const float ikXm = T.ik[0][1][max(i - 1, 0)], ikYm = T.ik[1][1][max(j - 1, 0)];
  const int sXm = hasXm ? T.sidx[0][i - 1] : -1, sYm = hasYm ? T.sidx[1][j - 1] : -1;

  // R membership of the own H components along x and y (H_c: integer along c, half along the others)
  const bool rxh = i >= g.rhalf_lo[0] && i <= g.rhalf_hi[0], rxi = i >= g.rint_lo[0] && i <= g.rint_hi[0];
  const bool ryh = j >= g.rhalf_lo[1] && j <= g.rhalf_hi[1], ryi = j >= g.rint_lo[1] && j <= g.rint_hi[1];

  const PsiSet& Pi = A.pin;
  const PsiSet& Po = A.pout;
  const bool lay_xy = (sX0 & sXm & sY0 & sYm) >= 0;  // this column or its -x/-y neighbour is in a layer
  unsigned det_xy = 0;  // folded detectors whose box holds this column
  if (A.det_step >= 0)
    for (int s = 0; s < A.ndet; ++s)
      if (own && i >= A.det[s].lo[0] && i < A.det[s].hi[0] && j >= A.det[s].lo[1] && j < A.det[s].hi[1])
        det_xy |= 1u << s;

  // E_x, E_y of the own column at k1 (the plane above the chunk)
  float ex_up = 0.f, ey_up = 0.f;
  if (own && k1 < nz) {
    ex_up = A.F.f[0][k1 * plane + q0];
    ey_up = A.F.f[1][k1 * plane + q0];
  }

  waited &= R.wait(ktop);
  for (int k = ktop; k >= k0; --k) {
    const int q = k * plane + q0;
    if (k - 1 >= kbot) waited &= R.wait(k - 1);
    __syncthreads();  // every thread is past plane k+1
    if (tid == 0 && k + 1 <= ktop && k + 1 - NSTAGE >= kbot) {
      async_proxy_fence();
      issue_rev_H(M, R, i0, j0, k + 1 - NSTAGE);
    }
    if (!own) continue;
    const unsigned char* st = R.at(k);
    const Wide3 Es = reinterpret_cast<Wide3>(st + RH_E);
    const Own3 Hs = reinterpret_cast<Own3>(st + RH_H);
    const Wide3 Bs = reinterpret_cast<Wide3>(st + RH_HB);
    const Own3 Gs = reinterpret_cast<Own3>(st + RH_EB);
    const float ex = Es[0][ty][tx], ey = Es[1][ty][tx], ez = Es[2][ty][tx];
    const float hx = Hs[0][ty][tx], hy = Hs[1][ty][tx], hz = Hs[2][ty][tx];
    const float bx = Bs[0][ty + 1][tx + 4], by = Bs[1][ty + 1][tx + 4], bz = Bs[2][ty + 1][tx + 4];
    const float ebx = Gs[0][ty][tx], eby = Gs[1][ty][tx], ebz = Gs[2][ty][tx];
    float bxm = 0.f, bym = 0.f;
    if (k > 0) {
      const Wide3 Bm = reinterpret_cast<Wide3>(R.at(k - 1) + RH_HB);
      bxm = Bm[0][ty + 1][tx + 4];
      bym = Bm[1][ty + 1][tx + 4];
    }
    const float wx = -S * bx, wy = -S * by, wz = -S * bz;
    // w of the -x neighbour (z and y) and of the -y neighbour (z and x); 0 beyond the grid
    const float wz_x = -S * Bs[2][ty + 1][tx + 3], wy_x = -S * Bs[1][ty + 1][tx + 3];
    const float wz_y = -S * Bs[2][ty][tx + 4], wx_y = -S * Bs[0][ty][tx + 4];

    const float ikZ = T.ik[2][1][k];
    const int sZ = T.sidx[2][k];

    // inverse H update on R (E beyond index N - 1 is the PEC wall: zero)
    const float ez_y = Es[2][ty + 1][tx], ex_y = Es[0][ty + 1][tx];
    const float ey_x = Es[1][ty][tx + 1], ez_x = Es[2][ty][tx + 1];
    const bool rzh = k >= g.rhalf_lo[2] && k <= g.rhalf_hi[2], rzi = k >= g.rint_lo[2] && k <= g.rint_hi[2];
    if (A.inverse) {
      if (rxi && ryh && rzh) A.F.f[3][q] = hx + S * ((ez_y - ez) * ikY0 - (ey_up - ey) * ikZ);
      if (rxh && ryi && rzh) A.F.f[4][q] = hy + S * ((ex_up - ex) * ikZ - (ez_x - ez) * ikX0);
      if (rxh && ryh && rzi) A.F.f[5][q] = hz + S * ((ey_x - ey) * ikX0 - (ex_y - ex) * ikY0);
    }
    ex_up = ex;
    ey_up = ey;

    // adjoint gather into E-bar: the plain coefficients +-w of the own H point and of its -x, -y, -z
    // neighbours, then the CPML corrections axis by axis
    const float wy_m = k > 0 ? -S * bym : 0.f, wx_m = k > 0 ? -S * bxm : 0.f;  // w at (i, j, k-1)
    const int sZm = k > 0 ? T.sidx[2][k - 1] : -1;
    float nbx, nby, nbz;  // the new E-bar
    if (!lay_xy && sZ < 0 && sZm < 0) {  // no layer along any axis at this point or its neighbours
      nbx = ebx + ((wy_m - wy) + (-wz_y + wz));
      nby = eby + ((wz_x - wz) + (-wx_m + wx));
      nbz = ebz + ((wx_y - wx) + (-wy_x + wy));
    } else {
      float cex = 0.f, cey = 0.f, cez = 0.f;
      if (sX0 >= 0 || sXm >= 0) {  // along x: Q1 of H_z (2,0) and Q2 of H_y (1,0), own and -x
        float e1z = 0.f, e2y = 0.f, n1z = 0.f, n2y = 0.f;
        if (sX0 >= 0) {
          const int z = zx_of(g, j, k, sX0);
          const float cX = T.c[0][1][i], bX = T.b[0][1][i];
          const float p20 = Pi.p[2][0][z], p10 = Pi.p[1][0][z];
          e1z = acorr(wz, ikX0, cX, p20);
          e2y = acorr(-wy, ikX0, cX, p10);
          Po.p[2][0][z] = bX * (p20 + wz);
          Po.p[1][0][z] = bX * (p10 - wy);
        }
        if (sXm >= 0) {
          const int z = zx_of(g, j, k, sXm);
          const float cX = T.c[0][1][i - 1];
          n1z = acorr(wz_x, ikXm, cX, Pi.p[2][0][z]);
          n2y = acorr(-wy_x, ikXm, cX, Pi.p[1][0][z]);
        }
        cey += n1z - e1z;
        cez += n2y - e2y;
      }
      if (sY0 >= 0 || sYm >= 0) {  // along y: Q1 of H_x (0,1) and Q2 of H_z (2,1), own and -y
        float e1x = 0.f, e2z = 0.f, n1x = 0.f, n2z = 0.f;
        if (sY0 >= 0) {
          const int z = zy_of(g, i, k, sY0);
          const float cY = T.c[1][1][j], bY = T.b[1][1][j];
          const float p01 = Pi.p[0][1][z], p21 = Pi.p[2][1][z];
          e1x = acorr(wx, ikY0, cY, p01);
          e2z = acorr(-wz, ikY0, cY, p21);
          Po.p[0][1][z] = bY * (p01 + wx);
          Po.p[2][1][z] = bY * (p21 - wz);
        }
        if (sYm >= 0) {
          const int z = zy_of(g, i, k, sYm);
          const float cY = T.c[1][1][j - 1];
          n1x = acorr(wx_y, ikYm, cY, Pi.p[0][1][z]);
          n2z = acorr(-wz_y, ikYm, cY, Pi.p[2][1][z]);
        }
        cex += n2z - e2z;
        cez += n1x - e1x;
      }
      if (sZ >= 0 || sZm >= 0) {  // along z: Q1 of H_y (1,2) and Q2 of H_x (0,2), own and -z
        float e1y = 0.f, e2x = 0.f, m1y = 0.f, m2x = 0.f;
        if (sZ >= 0) {
          const int z = zz_of(g, i, j, sZ);
          const float cZ = T.c[2][1][k], bZ = T.b[2][1][k];
          const float p12 = Pi.p[1][2][z], p02 = Pi.p[0][2][z];
          e1y = acorr(wy, ikZ, cZ, p12);
          e2x = acorr(-wx, ikZ, cZ, p02);
          Po.p[1][2][z] = bZ * (p12 + wy);
          Po.p[0][2][z] = bZ * (p02 - wx);
        }
        if (sZm >= 0) {
          const int z = zz_of(g, i, j, sZm);
          const float ikZm = T.ik[2][1][k - 1], cZ = T.c[2][1][k - 1];
          m1y = acorr(wy_m, ikZm, cZ, Pi.p[1][2][z]);
          m2x = acorr(-wx_m, ikZm, cZ, Pi.p[0][2][z]);
        }
        cex += m1y - e1y;
        cey += m2x - e2x;
      }
      nbx = ebx + (((wy_m - wy) + (-wz_y + wz)) + cex);
      nby = eby + (((wz_x - wz) + (-wx_m + wx)) + cey);
      nbz = ebz + (((wx_y - wx) + (-wy_x + wy)) + cez);
    }
    if (det_xy) {  // folded detector adjoints, one after the other in detector order
      for (int s = 0; s < A.ndet; ++s) {
        const DetDev& d = A.det[s];
        if (!((det_xy >> s) & 1u) || k < d.lo[2] || k >= d.hi[2]) continue;
        if (d.kind == FDTD_DET_POINT_SERIES) {
          const float v = (float)A.gy[d.off + A.det_step];
          if (d.comp == 0) nbx += v;
          else if (d.comp == 1) nby += v;
          else nbz += v;
        } else {  // |E|^2 summed over the steps: dL/dE = 2 g E
          const double w = 2.0 * A.gy[d.off + box_offset(d.lo, d.hi, i, j, k)];
          nbx += (float)(w * (double)ex);
          nby += (float)(w * (double)ey);
          nbz += (float)(w * (double)ez);
        }
      }
    }
    // E components on the PEC walls keep E-bar = 0
    if (j > 0 && k > 0) A.B.f[0][q] = nbx;
    if (i > 0 && k > 0) A.B.f[1][q] = nby;
    if (i > 0 && j > 0) A.B.f[2][q] = nbz;
  }
  if (!waited) atomicOr(A.status, 1);
}

template <int NSTAGE>
__global__ void __launch_bounds__(NT, NSTAGE == 3 ? 4 : 3) k_rev_E(const __grid_constant__ RevArgs A, const __grid_constant__ RevMaps M) {
  revE_body<NSTAGE>(A, M, blockIdx.x, blockIdx.y, blockIdx.z);
}
template <int NSTAGE>
__global__ void __launch_bounds__(NT, NSTAGE == 3 ? 4 : 3) k_rev_H(const __grid_constant__ RevArgs A, const __grid_constant__ RevMaps M) {
  revH_body<NSTAGE>(A, M, blockIdx.x, blockIdx.y, blockIdx.z);
}
// Several requests in one launch (the flat grid of GroupGrid).
template <int NSTAGE>
__global__ void __launch_bounds__(NT, NSTAGE == 3 ? 4 : 3) k_rev_E_group(const __grid_constant__ RevGroup G) {
  int bx, by, bz;
  const int r = group_locate(G.grid, bx, by, bz);
  revE_body<NSTAGE>(G.a[r], G.m[r], bx, by, bz);
}
template <int NSTAGE>
__global__ void __launch_bounds__(NT, NSTAGE == 3 ? 4 : 3) k_rev_H_group(const __grid_constant__ RevGroup G) {
  int bx, by, bz;
  const int r = group_locate(G.grid, bx, by, bz);
  revH_body<NSTAGE>(G.a[r], G.m[r], bx, by, bz);
}

}  // namespace

void launch_rev_group(RevGroup& G, int which, cudaStream_t s) {
  const int total = group_fill(G.grid, G.n, [&](int r, int* nb) {
    const Geo& g = G.a[r].g;
    nb[0] = (g.n[0] + TX - 1) / TX;
    nb[1] = (g.n[1] + TY - 1) / TY;
    nb[2] = (g.n[2] + G.a[r].tz - 1) / G.a[r].tz;
  });
  if (total == 0) return;
  const int ns = G.a[0].nstage;
  if (which == 0) {
    if (ns == 3) launch_pdl(k_rev_E_group<3>, dim3(total), dim3(NT), re_smem(3), s, G);
    else launch_pdl(k_rev_E_group<4>, dim3(total), dim3(NT), re_smem(4), s, G);
  } else {
    if (ns == 3) launch_pdl(k_rev_H_group<3>, dim3(total), dim3(NT), rh_smem(3), s, G);
    else launch_pdl(k_rev_H_group<4>, dim3(total), dim3(NT), rh_smem(4), s, G);
  }
}

int rev_tile_x() { return TX; }
int rev_tile_y() { return TY; }

MapBox rev_box_own() { return {TX, TY}; }
MapBox rev_box_wide() { return {BW, BH}; }

int prepare_rev(int nstage, int* blocks_per_sm) {
  auto ke = nstage == 3 ? k_rev_E<3> : k_rev_E<4>;
  auto kh = nstage == 3 ? k_rev_H<3> : k_rev_H<4>;
  auto kge = nstage == 3 ? k_rev_E_group<3> : k_rev_E_group<4>;
  auto kgh = nstage == 3 ? k_rev_H_group<3> : k_rev_H_group<4>;
  cudaError_t e = cudaFuncSetAttribute(ke, cudaFuncAttributeMaxDynamicSharedMemorySize, re_smem(nstage));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kh, cudaFuncAttributeMaxDynamicSharedMemorySize, rh_smem(nstage));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kge, cudaFuncAttributeMaxDynamicSharedMemorySize, re_smem(nstage));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kgh, cudaFuncAttributeMaxDynamicSharedMemorySize, rh_smem(nstage));
  int be = 0, bh = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&be, ke, NT, re_smem(nstage));
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bh, kh, NT, rh_smem(nstage));
  *blocks_per_sm = std::min(be, bh);
  return e == cudaSuccess ? FDTD_OK : set_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
}

void launch_rev_E(const RevArgs& a, const RevMaps& m, cudaStream_t s) {
  const Geo& g = a.g;
  dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + a.tz - 1) / a.tz);
  if (a.nstage == 3) launch_pdl(k_rev_E<3>, grid, dim3(NT), re_smem(3), s, a, m);
  else launch_pdl(k_rev_E<4>, grid, dim3(NT), re_smem(4), s, a, m);
}

void launch_rev_H(const RevArgs& a, const RevMaps& m, cudaStream_t s) {
  const Geo& g = a.g;
  dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + a.tz - 1) / a.tz);
  if (a.nstage == 3) launch_pdl(k_rev_H<3>, grid, dim3(NT), rh_smem(3), s, a, m);
  else launch_pdl(k_rev_H<4>, grid, dim3(NT), rh_smem(4), s, a, m);
}

}  // namespace fdtd
