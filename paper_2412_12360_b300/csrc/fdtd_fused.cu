// Fused forward step of arXiv 2412.12360 Sec. 2.1: the H update (Eq. 1) and the E update (Eq. 2) of
// one time step in a single sweep over the grid, with the CPML memories, the soft sources, the
// detectors and the boundary-face record (Sec. 2.2) as epilogues of the same sweep.
//
// Each block owns a TX x TY column tile and marches a chunk of TZ z-planes. Per plane it stages
// E^n of the tile plus a one-cell halo in shared memory (planes k and k+1 in flight), computes
// H^{n+1/2} for its cells and, redundantly, for the halo column x = i0-1 and row y = j0-1 that its
// E update reads, then computes E^{n+1}. Fields are double-buffered (read `cur`, write `nxt`) so
// neighbouring tiles never see a half-updated field; every cell is read and written once per step
// from HBM (52 bytes per cell) and the halos come from L1/L2.
//
// The march is software-pipelined: while plane k is computed, the loads of E^n for plane k+2 and of
// H^{n-1/2} and a for plane k+1 are already in flight. Everything that depends only on x and y (CPML
// coefficients, slab indices, source, detector and face membership) is computed once per thread;
// what depends on z once per plane. Every cell takes the plain Yee update; cells in a CPML layer add
// the correction (1/kappa - 1) d + psi per curl term, which is exactly 0 off the layers and on their
// inner edge, so the PML-free region R is updated by the plain formula the inverse step mirrors.
#include "fdtd_internal.cuh"

namespace fdtd {

namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int SX = TX + 2, SY = TY + 2;  // staged E tile with a one-cell halo
constexpr int HX = TX + 1, HY = TY + 1;  // new H with the low halo

// CPML correction of one curl term inside a layer: the update uses d / kappa + psi_new where the plain
// Yee update uses d, so the correction is (1/kappa - 1) d + psi_new with psi_new = b psi_old + c d
// (read from pin[z], written to pout[z] when STORE). Off the layers (s < 0) it is 0; on the layer's
// inner edge (depth 0) 1/kappa = 1, b = 1, c = 0 and psi stays 0, so it is 0 there too.
template <bool STORE>
__device__ __forceinline__ float corr(float d, float ik, int s, const float* __restrict__ bt,
                                      const float* __restrict__ ct, int pos, const float* pin, float* pout, int z) {
  if (s < 0) return 0.f;
  const float v = bt[pos] * pin[z] + ct[pos] * d;
  if (STORE) pout[z] = v;
  return (ik - 1.f) * d + v;
}

// psi index of the point (x, y, k), slab index s, for the derivative along x, y or z
__device__ __forceinline__ int zx_of(const Geo& g, int y, int k, int s) { return (k * g.n[1] + y) * g.slab[0] + s; }
__device__ __forceinline__ int zy_of(const Geo& g, int x, int k, int s) { return (k * g.slab[1] + s) * g.nxp + x; }
__device__ __forceinline__ int zz_of(const Geo& g, int x, int y, int s) { return (s * g.n[1] + y) * g.nxp + x; }

__device__ __forceinline__ float pick3(int c, float a, float b, float d) { return c == 0 ? a : (c == 1 ? b : d); }

// Write this cell's H into face segment s of the record if (i, j, k) lies on it.
__device__ __noinline__ void face_write(const FwdArgs& A, int s, int i, int j, int k, float hx, float hy, float hz) {
  const FaceSeg& sg = A.faces.seg[s];
  const int p[3] = {i, j, k};
  const int a1 = (sg.axis + 1) % 3, a2 = (sg.axis + 2) % 3;
  if (p[sg.axis] != sg.idx) return;
  const int u = p[a1] - sg.lo1, v = p[a2] - sg.lo2;
  if (u < 0 || u >= sg.n1 || v < 0 || v >= sg.n2) return;
  A.rec[sg.off + (int64_t)v * sg.n1 + u] = sg.comp == 0 ? hx : (sg.comp == 1 ? hy : hz);
}

__device__ __forceinline__ int box_offset(const int lo[3], const int hi[3], int x, int y, int k) {
  return ((k - lo[2]) * (hi[1] - lo[1]) + (y - lo[1])) * (hi[0] - lo[0]) + (x - lo[0]);
}

// Staging of one E plane (tile plus a one-cell halo) into shared memory: every thread loads its own
// cell (row ty+1, column tx+1: aligned, coalesced rows); warp 0 loads the halo row y = j0-1, warp 1 the
// row y = j0+TY, and warp 2 the halo columns x = i0-1 (lanes 0..TY+1) and x = i0+TX (lanes 16..17+TY),
// corners included.
struct Stage {
  int own_off, role_off;  // in-plane offsets of the own cell and of this thread's halo point
  bool own_ok, role_ok;   // inside the grid
  int role_ry, role_rx;   // where the halo point goes in the staged tile (role_ry < 0: no halo point)
};

__device__ __forceinline__ void load_stage(const Geo& g, const Fields& F, const Stage& st, int k, float r[2][3]) {
  const bool kin = k < g.n[2];
  const int base = k * (int)g.plane;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    r[0][c] = (kin && st.own_ok) ? F.f[c][base + st.own_off] : 0.f;
    r[1][c] = (kin && st.role_ok) ? F.f[c][base + st.role_off] : 0.f;
  }
}

__device__ __forceinline__ void store_stage(float (*dst)[SY][SX], const Stage& st, const float r[2][3], int tx, int ty) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dst[c][ty + 1][tx + 1] = r[0][c];
    if (st.role_ry >= 0) dst[c][st.role_ry][st.role_rx] = r[1][c];
  }
}

__global__ void __launch_bounds__(NT, 3) k_fwd_fused(FwdArgs A) {
  __shared__ float sE[2][3][SY][SX];
  __shared__ float sH[3][HY][HX];
  __shared__ double sred[NT];

  const Geo& g = A.g;
  const Tables& T = A.T;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * A.tz;
  const int k1 = min(g.n[2], k0 + A.tz);
  const int nx = g.n[0], ny = g.n[1];
  const int plane = (int)g.plane;
  const int i = i0 + tx, j = j0 + ty;
  const bool own = i < nx && j < ny;
  const int q0 = j * g.nxp + i;
  const float S = g.S;
  const int rx = tx + 1, ry = ty + 1;

  Stage st;
  st.own_ok = own;
  st.own_off = q0;
  st.role_ry = -1;
  st.role_rx = 0;
  st.role_ok = false;
  st.role_off = 0;
  {
    int x = 0, y = 0;
    if (ty == 0) {  // halo row y = j0 - 1
      x = i0 + tx; y = j0 - 1; st.role_ry = 0; st.role_rx = tx + 1;
    } else if (ty == 1) {  // halo row y = j0 + TY
      x = i0 + tx; y = j0 + TY; st.role_ry = TY + 1; st.role_rx = tx + 1;
    } else if (ty == 2 && tx < SY) {  // halo column x = i0 - 1, rows j0-1 .. j0+TY
      x = i0 - 1; y = j0 - 1 + tx; st.role_ry = tx; st.role_rx = 0;
    } else if (ty == 2 && tx >= 16 && tx < 16 + SY) {  // halo column x = i0 + TX
      x = i0 + TX; y = j0 - 1 + (tx - 16); st.role_ry = tx - 16; st.role_rx = TX + 1;
    }
    st.role_ok = st.role_ry >= 0 && x >= 0 && x < nx && y >= 0 && y < ny;
    st.role_off = y * g.nxp + x;
  }

  // halo H: warp 3 computes the row y = j0-1 (Hx, Hz), warp 4 lanes 0..TY-1 the column x = i0-1 (Hy, Hz)
  const bool hrow = ty == 3 && j0 > 0 && i < nx;
  const bool hcol = ty == 4 && tx < TY && i0 > 0 && (j0 + tx) < ny;
  const int xh = hcol ? i0 - 1 : min(i, nx - 1);
  const int yh = hcol ? j0 + tx : max(j0 - 1, 0);
  const int hrx = hcol ? 0 : tx + 1, hry = hcol ? tx + 1 : 0;  // staged position of the halo point
  const int qh0 = yh * g.nxp + xh;

  // CPML data along x and y, fixed for the whole march (H tables at half, E tables at integer positions)
  const int ic = min(i, nx - 1), jc = min(j, ny - 1);
  const float ikXh = T.ik[0][1][ic], ikXe = T.ik[0][0][ic], ikYh = T.ik[1][1][jc], ikYe = T.ik[1][0][jc];
  const int sX = T.sidx[0][ic], sY = T.sidx[1][jc];
  const float ikXhh = T.ik[0][1][xh], ikYhh = T.ik[1][1][yh];  // at the halo point
  const int sXh = T.sidx[0][xh], sYh = T.sidx[1][yh];

  // membership of this column in the source and detector boxes (bit s), and face segments
  unsigned src_xy = 0, det_xy = 0;
  for (int s = 0; s < A.nsrc; ++s) {
    const SrcDev& sd = A.src[s];
    if (own && i >= sd.lo[0] && i < sd.hi[0] && j >= sd.lo[1] && j < sd.hi[1]) src_xy |= 1u << s;
  }
  for (int s = 0; s < A.ndet; ++s) {
    const DetDev& d = A.det[s];
    if (own && i >= d.lo[0] && i < d.hi[0] && j >= d.lo[1] && j < d.hi[1]) det_xy |= 1u << s;
  }
  // (a column lies on at most one x- or y-face line, i.e. two segments; z-faces are at most two
  // planes, each with an Hx and an Hy segment). Only segment numbers are kept; offsets are computed
  // when a face value is written.
  int fseg = -1;              // x/y face: segment numbers a | b << 8
  int fz0 = -1, fz1 = -1;     // z-face planes through this column
  int fzseg = 0;              // their segments: plane 0 (x, y), plane 1 (x, y), 8 bits each
  if (A.rec && own) {
    int na = 0;
    for (int s = 0; s < A.faces.nseg; ++s) {
      const FaceSeg& sg = A.faces.seg[s];
      if ((sg.axis == 0 && i == sg.idx && j >= sg.lo1 && j < sg.lo1 + sg.n1) ||
          (sg.axis == 1 && j == sg.idx && i >= sg.lo2 && i < sg.lo2 + sg.n2)) {
        fseg = (na == 0) ? s : ((fseg & 0xff) | (s << 8));
        ++na;
      } else if (sg.axis == 2 && i >= sg.lo1 && i < sg.lo1 + sg.n1 && j >= sg.lo2 && j < sg.lo2 + sg.n2) {
        const int pl = (fz0 < 0 || fz0 == sg.idx) ? 0 : 1;
        if (pl == 0) fz0 = sg.idx; else fz1 = sg.idx;
        fzseg |= s << (8 * (2 * pl + sg.comp));
      }
    }
  }

  double facc[kMaxDet];
#pragma unroll
  for (int q = 0; q < kMaxDet; ++q) facc[q] = 0.0;

  const PsiSet& PHi = A.psiH_cur;
  const PsiSet& PHo = A.psiH_nxt;
  const PsiSet& PEi = A.psiE_cur;
  const PsiSet& PEo = A.psiE_nxt;
  const Fields& C = A.cur;
  const Fields& N = A.nxt;

  float pe[2][3];
  float hxm = 0.f, hym = 0.f;
  int cur = 0;
  if (k0 > 0) {
    // H^{n+1/2} at (i, j, k0-1), read by the first plane's E update (its owner stores it)
    const int km = k0 - 1;
    load_stage(g, C, st, km, pe);
    store_stage(sE[0], st, pe, tx, ty);
    load_stage(g, C, st, k0, pe);
    store_stage(sE[1], st, pe, tx, ty);
    __syncthreads();
    if (own) {
      const int q = km * plane + q0;
      const float(*a0)[SY][SX] = sE[0];
      const float(*a1)[SY][SX] = sE[1];
      const float ikZh = T.ik[2][1][km];
      const int sZ = T.sidx[2][km];
      const float dzy = a0[2][ry + 1][rx] - a0[2][ry][rx], dyz = a1[1][ry][rx] - a0[1][ry][rx];
      const float dxz = a1[0][ry][rx] - a0[0][ry][rx], dzx = a0[2][ry][rx + 1] - a0[2][ry][rx];
      float cx = dzy - dyz, cy = dxz - dzx;
      if ((sX & sY & sZ) >= 0) {
        const int zx = sX >= 0 ? zx_of(g, j, km, sX) : 0, zy = sY >= 0 ? zy_of(g, i, km, sY) : 0;
        const int zz = sZ >= 0 ? zz_of(g, i, j, sZ) : 0;
        cx += corr<false>(dzy, ikYh, sY, T.b[1][1], T.c[1][1], j, PHi.p[0][1], nullptr, zy) -
              corr<false>(dyz, ikZh, sZ, T.b[2][1], T.c[2][1], km, PHi.p[0][2], nullptr, zz);
        cy += corr<false>(dxz, ikZh, sZ, T.b[2][1], T.c[2][1], km, PHi.p[1][2], nullptr, zz) -
              corr<false>(dzx, ikXh, sX, T.b[0][1], T.c[0][1], i, PHi.p[1][0], nullptr, zx);
      }
      hxm = C.f[3][q] - S * cx;
      hym = C.f[4][q] - S * cy;
    }
    cur = 1;
    __syncthreads();
  } else {
    load_stage(g, C, st, k0, pe);
    store_stage(sE[0], st, pe, tx, ty);
  }
  // prefetch: E^n of plane k0+1, and H^{n-1/2}, a of plane k0 (own and halo point)
  load_stage(g, C, st, k0 + 1, pe);
  float nhx = 0.f, nhy = 0.f, nhz = 0.f, na = 0.f, nh1 = 0.f, nh2 = 0.f;
  if (own) {
    const int q = k0 * plane + q0;
    nhx = C.f[3][q];
    nhy = C.f[4][q];
    nhz = C.f[5][q];
    na = A.a[q];
  }
  if (hrow || hcol) {
    const int q = k0 * plane + qh0;
    nh1 = hrow ? C.f[3][q] : C.f[4][q];
    nh2 = C.f[5][q];
  }

  for (int k = k0; k < k1; ++k) {
    const int q = k * plane + q0;
    store_stage(sE[cur ^ 1], st, pe, tx, ty);
    const float hox = nhx, hoy = nhy, hoz = nhz, av = na, ho1 = nh1, ho2 = nh2;
    if (k + 1 < k1) {  // prefetch for the next plane
      load_stage(g, C, st, k + 2, pe);
      if (own) {
        nhx = C.f[3][q + plane];
        nhy = C.f[4][q + plane];
        nhz = C.f[5][q + plane];
        na = A.a[q + plane];
      }
      if (hrow || hcol) {
        const int qn = (k + 1) * plane + qh0;
        nh1 = hrow ? C.f[3][qn] : C.f[4][qn];
        nh2 = C.f[5][qn];
      }
    }
    const float ikZh = T.ik[2][1][k], ikZe = T.ik[2][0][k];
    const int sZ = T.sidx[2][k];
    unsigned src_k = 0, det_k = 0;  // sources and detectors whose z-range holds this plane
    for (int s = 0; s < A.nsrc; ++s) src_k |= (k >= A.src[s].lo[2] && k < A.src[s].hi[2]) ? 1u << s : 0u;
    for (int s = 0; s < A.ndet; ++s) det_k |= (k >= A.det[s].lo[2] && k < A.det[s].hi[2]) ? 1u << s : 0u;
    __syncthreads();
    const float(*ek)[SY][SX] = sE[cur];
    const float(*ek1)[SY][SX] = sE[cur ^ 1];
    const bool lay = (sX & sY & sZ) >= 0;  // some axis of this cell is in a layer (-1 = all bits set)
    const int zx = sX >= 0 ? zx_of(g, j, k, sX) : 0;
    const int zy = sY >= 0 ? zy_of(g, i, k, sY) : 0;
    const int zz = sZ >= 0 ? zz_of(g, i, j, sZ) : 0;

    // (b) H^{n+1/2} on plane k: own cell (plain Yee update plus the CPML correction in the layers)
    float hx = 0.f, hy = 0.f, hz = 0.f;
    if (own) {
      const float dzy = ek[2][ry + 1][rx] - ek[2][ry][rx], dyz = ek1[1][ry][rx] - ek[1][ry][rx];
      const float dxz = ek1[0][ry][rx] - ek[0][ry][rx], dzx = ek[2][ry][rx + 1] - ek[2][ry][rx];
      const float dyx = ek[1][ry][rx + 1] - ek[1][ry][rx], dxy = ek[0][ry + 1][rx] - ek[0][ry][rx];
      float cx = dzy - dyz, cy = dxz - dzx, cz = dyx - dxy;
      if (lay) {
        cx += corr<true>(dzy, ikYh, sY, T.b[1][1], T.c[1][1], j, PHi.p[0][1], PHo.p[0][1], zy) -
              corr<true>(dyz, ikZh, sZ, T.b[2][1], T.c[2][1], k, PHi.p[0][2], PHo.p[0][2], zz);
        cy += corr<true>(dxz, ikZh, sZ, T.b[2][1], T.c[2][1], k, PHi.p[1][2], PHo.p[1][2], zz) -
              corr<true>(dzx, ikXh, sX, T.b[0][1], T.c[0][1], i, PHi.p[1][0], PHo.p[1][0], zx);
        cz += corr<true>(dyx, ikXh, sX, T.b[0][1], T.c[0][1], i, PHi.p[2][0], PHo.p[2][0], zx) -
              corr<true>(dxy, ikYh, sY, T.b[1][1], T.c[1][1], j, PHi.p[2][1], PHo.p[2][1], zy);
      }
      hx = hox - S * cx;
      hy = hoy - S * cy;
      hz = hoz - S * cz;
      sH[0][ry][rx] = hx;
      sH[1][ry][rx] = hy;
      sH[2][ry][rx] = hz;
      N.f[3][q] = hx;
      N.f[4][q] = hy;
      N.f[5][q] = hz;
    }
    // the low halo: (i, j0-1) gives Hx, Hz; (i0-1, j0+r) gives Hy, Hz
    if (hrow || hcol) {
      const int r = hry, c = hrx;
      const bool hl = (sXh & sYh & sZ) >= 0;
      const int hzx = sXh >= 0 ? zx_of(g, yh, k, sXh) : 0, hzy = sYh >= 0 ? zy_of(g, xh, k, sYh) : 0;
      const int hzz = sZ >= 0 ? zz_of(g, xh, yh, sZ) : 0;
      const float dyx = ek[1][r][c + 1] - ek[1][r][c], dxy = ek[0][r + 1][c] - ek[0][r][c];
      float cz = dyx - dxy;
      if (hl)
        cz += corr<false>(dyx, ikXhh, sXh, T.b[0][1], T.c[0][1], xh, PHi.p[2][0], nullptr, hzx) -
              corr<false>(dxy, ikYhh, sYh, T.b[1][1], T.c[1][1], yh, PHi.p[2][1], nullptr, hzy);
      sH[2][r][c] = ho2 - S * cz;
      if (hrow) {  // Hx
        const float dzy = ek[2][r + 1][c] - ek[2][r][c], dyz = ek1[1][r][c] - ek[1][r][c];
        float cx = dzy - dyz;
        if (hl)
          cx += corr<false>(dzy, ikYhh, sYh, T.b[1][1], T.c[1][1], yh, PHi.p[0][1], nullptr, hzy) -
                corr<false>(dyz, ikZh, sZ, T.b[2][1], T.c[2][1], k, PHi.p[0][2], nullptr, hzz);
        sH[0][r][c] = ho1 - S * cx;
      } else {  // Hy
        const float dxz = ek1[0][r][c] - ek[0][r][c], dzx = ek[2][r][c + 1] - ek[2][r][c];
        float cy = dxz - dzx;
        if (hl)
          cy += corr<false>(dxz, ikZh, sZ, T.b[2][1], T.c[2][1], k, PHi.p[1][2], nullptr, hzz) -
                corr<false>(dzx, ikXhh, sXh, T.b[0][1], T.c[0][1], xh, PHi.p[1][0], nullptr, hzx);
        sH[1][r][c] = ho1 - S * cy;
      }
    }
    if (fseg >= 0) face_write(A, fseg & 0xff, i, j, k, hx, hy, hz);
    if (fseg > 0xff) face_write(A, fseg >> 8, i, j, k, hx, hy, hz);
    if (k == fz0 || k == fz1) {
      const int sh = (k == fz0) ? 0 : 16;
      face_write(A, (fzseg >> sh) & 0xff, i, j, k, hx, hy, hz);
      face_write(A, (fzseg >> (sh + 8)) & 0xff, i, j, k, hx, hy, hz);
    }
    __syncthreads();

    // (c) E^{n+1} on plane k at the own cell (tangential E on a PEC wall at index 0 is held), then
    // sources and detectors
    if (own) {
      const float Sa = S * av;
      float ex = ek[0][ry][rx], ey = ek[1][ry][rx], ez = ek[2][ry][rx];
      const float d1x = hz - sH[2][ry - 1][rx], d2x = hy - hym;   // E_x: along y, along z
      const float d1y = hx - hxm, d2y = hz - sH[2][ry][rx - 1];   // E_y: along z, along x
      const float d1z = hy - sH[1][ry][rx - 1], d2z = hx - sH[0][ry - 1][rx];  // E_z: along x, along y
      float cx = d1x - d2x, cy = d1y - d2y, cz = d1z - d2z;
      if (lay) {
        if (j > 0 && k > 0)
          cx += corr<true>(d1x, ikYe, sY, T.b[1][0], T.c[1][0], j, PEi.p[0][1], PEo.p[0][1], zy) -
                corr<true>(d2x, ikZe, sZ, T.b[2][0], T.c[2][0], k, PEi.p[0][2], PEo.p[0][2], zz);
        if (i > 0 && k > 0)
          cy += corr<true>(d1y, ikZe, sZ, T.b[2][0], T.c[2][0], k, PEi.p[1][2], PEo.p[1][2], zz) -
                corr<true>(d2y, ikXe, sX, T.b[0][0], T.c[0][0], i, PEi.p[1][0], PEo.p[1][0], zx);
        if (i > 0 && j > 0)
          cz += corr<true>(d1z, ikXe, sX, T.b[0][0], T.c[0][0], i, PEi.p[2][0], PEo.p[2][0], zx) -
                corr<true>(d2z, ikYe, sY, T.b[1][0], T.c[1][0], j, PEi.p[2][1], PEo.p[2][1], zy);
      }
      if (j > 0 && k > 0) ex += Sa * cx;
      if (i > 0 && k > 0) ey += Sa * cy;
      if (i > 0 && j > 0) ez += Sa * cz;
      if (src_xy & src_k) {
        for (int s = 0; s < A.nsrc; ++s) {
          const SrcDev& sd = A.src[s];
          if (!(((src_xy & src_k) >> s) & 1u)) continue;
          const float v = sd.w[box_offset(sd.lo, sd.hi, i, j, k)] * sd.g[A.step];
          if (sd.comp == 0) ex += v;
          else if (sd.comp == 1) ey += v;
          else ez += v;
        }
      }
      N.f[0][q] = ex;
      N.f[1][q] = ey;
      N.f[2][q] = ez;
      if (det_xy & det_k) {
#pragma unroll
        for (int s = 0; s < kMaxDet; ++s) {
          if (s >= A.ndet) break;
          const DetDev& d = A.det[s];
          if (!(((det_xy & det_k) >> s) & 1u)) continue;
          if (d.kind == 0) {
            A.det_out[d.off + A.step] = (double)(d.comp < 3 ? pick3(d.comp, ex, ey, ez) : pick3(d.comp - 3, hx, hy, hz));
          } else if (d.kind == 1) {
            A.det_out[d.off + box_offset(d.lo, d.hi, i, j, k)] += (double)ex * ex + (double)ey * ey + (double)ez * ez;
          } else {
            const int a1 = (d.axis + 1) % 3, a2 = (d.axis + 2) % 3;
            facc[s] += (double)pick3(a1, ex, ey, ez) * (double)pick3(a2, hx, hy, hz) -
                       (double)pick3(a2, ex, ey, ez) * (double)pick3(a1, hx, hy, hz);
          }
        }
      }
    }
    hxm = hx;
    hym = hy;
    cur ^= 1;
  }

  // flux detectors: fixed-order block reduction into this block's slot
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
    __syncthreads();
    sred[tid] = facc[s];
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
      if (tid < w) sred[tid] += sred[tid + w];
      __syncthreads();
    }
    if (tid == 0) {
      const int64_t slotid = ((int64_t)(bz - bz0) * (by1 - by0 + 1) + (by - by0)) * (bx1 - bx0 + 1) + (bx - bx0);
      A.partial[d.poff + (int64_t)A.step * d.nblk + slotid] = sred[0];
    }
  }
}

}  // namespace

int fused_tile_x() { return TX; }
int fused_tile_y() { return TY; }

void launch_fwd_fused(const FwdArgs& a, cudaStream_t s) {
  const Geo& g = a.g;
  dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + a.tz - 1) / a.tz);
  k_fwd_fused<<<grid, NT, 0, s>>>(a);
}

}  // namespace fdtd
