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
// what depends on z once per plane. A cell off the layers pays a multiply by 1/kappa = 1 (exact) and
// a few untaken branches for the CPML.
#include "fdtd_internal.cuh"

namespace fdtd {

namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int SX = TX + 2, SY = TY + 2;  // staged E tile with a one-cell halo
constexpr int HX = TX + 1, HY = TY + 1;  // new H with the low halo

// One curl term: difference / kappa plus the updated CPML memory (b, c at table position `pos`, memory
// read from pin[z], written to pout[z] when STORE). Off the layers (s < 0) it is d * 1 exactly.
template <bool STORE>
__device__ __forceinline__ float cterm(float d, float ik, int s, const float* __restrict__ bt,
                                       const float* __restrict__ ct, int pos, const float* pin, float* pout, int z) {
  float t = d * ik;
  if (s >= 0) {
    const float v = bt[pos] * pin[z] + ct[pos] * d;
    if (STORE) pout[z] = v;
    t += v;
  }
  return t;
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

// The four staging positions of a thread: rows ty and TY + ty (ty < 2), columns tx and TX + tx (tx < 2)
// of the (TY + 2) x (TX + 2) tile whose corner is (i0 - 1, j0 - 1).
struct Stage {
  int off[4];
  bool ok[4];
};

__device__ __forceinline__ void load_plane(const Geo& g, const Fields& F, const Stage& st, int k, float r[3][4]) {
  const bool kin = k < g.n[2];
  const int base = k * (int)g.plane;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int u = 0; u < 4; ++u) r[c][u] = (kin && st.ok[u]) ? F.f[c][base + st.off[u]] : 0.f;
}

__device__ __forceinline__ void store_plane(float (*dst)[SY][SX], const float r[3][4], int tx, int ty) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dst[c][ty][tx] = r[c][0];
    if (tx < 2) dst[c][ty][TX + tx] = r[c][1];
    if (ty < 2) {
      dst[c][TY + ty][tx] = r[c][2];
      if (tx < 2) dst[c][TY + ty][TX + tx] = r[c][3];
    }
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
  {
    const int xa = i0 - 1 + tx, xb = i0 + TX - 1 + tx, ya = j0 - 1 + ty, yb = j0 + TY - 1 + ty;
    const bool oxa = xa >= 0 && xa < nx, oxb = tx < 2 && xb < nx;
    const bool oya = ya >= 0 && ya < ny, oyb = ty < 2 && yb < ny;
    st.ok[0] = oya && oxa;
    st.ok[1] = oya && oxb;
    st.ok[2] = oyb && oxa;
    st.ok[3] = oyb && oxb;
    st.off[0] = ya * g.nxp + xa;
    st.off[1] = ya * g.nxp + xb;
    st.off[2] = yb * g.nxp + xa;
    st.off[3] = yb * g.nxp + xb;
  }

  // halo work: warp 0 takes the row y = j0-1 (Hx, Hz), threads TX .. TX+TY-1 the column x = i0-1 (Hy, Hz)
  const bool hrow = tid < TX && j0 > 0 && i < nx;
  const int hr = tid - TX;
  const bool hcol = tid >= TX && tid < TX + TY && i0 > 0 && (j0 + hr) < ny;
  const int xh = hcol ? i0 - 1 : min(i, nx - 1);            // x of this thread's halo point
  const int yh = hcol ? j0 + hr : max(j0 - 1, 0);           // y of this thread's halo point
  const int qh0 = yh * g.nxp + xh;

  // CPML data along x and y, fixed for the whole march
  const int ic = min(i, nx - 1), jc = min(j, ny - 1);
  const float ikXh = T.ik[0][1][ic], ikXe = T.ik[0][0][ic], ikYh = T.ik[1][1][jc], ikYe = T.ik[1][0][jc];
  const int sX = T.sidx[0][ic], sY = T.sidx[1][jc];
  const float ikXhh = T.ik[0][1][xh], ikYhh = T.ik[1][1][yh];  // at the halo point
  const int sXh = T.sidx[0][xh], sYh = T.sidx[1][yh];

  // membership of this column in the source and detector boxes (bit s), and in the x/y face planes
  unsigned src_xy = 0, det_xy = 0;
  for (int s = 0; s < A.nsrc; ++s) {
    const SrcDev& sd = A.src[s];
    if (own && i >= sd.lo[0] && i < sd.hi[0] && j >= sd.lo[1] && j < sd.hi[1]) src_xy |= 1u << s;
  }
  for (int s = 0; s < A.ndet; ++s) {
    const DetDev& d = A.det[s];
    if (own && i >= d.lo[0] && i < d.hi[0] && j >= d.lo[1] && j < d.hi[1]) det_xy |= 1u << s;
  }
  // boundary-face record: a column on an x- or y-face writes its H there for the planes in range; a
  // z-face plane is written by every column in range. Offsets into one step's record:
  //   x-face (comp y, z): off + (k - lo2) * n1 + (j - lo1);   y-face (comp z, x): off + (i - lo2) * n1 + (k - lo1)
  //   z-face (comp x, y): off + (j - lo2) * n1 + (i - lo1)
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

  float pe[3][4];
  float hxm = 0.f, hym = 0.f;
  int cur = 0;
  if (k0 > 0) {
    // H^{n+1/2} at (i, j, k0-1), read by the first plane's E update (its owner stores it)
    const int km = k0 - 1;
    load_plane(g, C, st, km, pe);
    store_plane(sE[0], pe, tx, ty);
    load_plane(g, C, st, k0, pe);
    store_plane(sE[1], pe, tx, ty);
    __syncthreads();
    if (own) {
      const int q = km * plane + q0;
      const float(*a0)[SY][SX] = sE[0];
      const float(*a1)[SY][SX] = sE[1];
      const float ikZh = T.ik[2][1][km];
      const int sZ = T.sidx[2][km];
      const int zx = sX >= 0 ? zx_of(g, j, km, sX) : 0, zy = sY >= 0 ? zy_of(g, i, km, sY) : 0;
      const int zz = sZ >= 0 ? zz_of(g, i, j, sZ) : 0;
      hxm = C.f[3][q] - S * (cterm<false>(a0[2][ry + 1][rx] - a0[2][ry][rx], ikYh, sY, T.b[1][1], T.c[1][1], j, PHi.p[0][1], nullptr, zy) -
                             cterm<false>(a1[1][ry][rx] - a0[1][ry][rx], ikZh, sZ, T.b[2][1], T.c[2][1], km, PHi.p[0][2], nullptr, zz));
      hym = C.f[4][q] - S * (cterm<false>(a1[0][ry][rx] - a0[0][ry][rx], ikZh, sZ, T.b[2][1], T.c[2][1], km, PHi.p[1][2], nullptr, zz) -
                             cterm<false>(a0[2][ry][rx + 1] - a0[2][ry][rx], ikXh, sX, T.b[0][1], T.c[0][1], i, PHi.p[1][0], nullptr, zx));
    }
    cur = 1;
    __syncthreads();
  } else {
    load_plane(g, C, st, k0, pe);
    store_plane(sE[0], pe, tx, ty);
  }
  // prefetch: E^n of plane k0+1, and H^{n-1/2}, a of plane k0 (own and halo point)
  load_plane(g, C, st, k0 + 1, pe);
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
    store_plane(sE[cur ^ 1], pe, tx, ty);
    const float hox = nhx, hoy = nhy, hoz = nhz, av = na, ho1 = nh1, ho2 = nh2;
    if (k + 1 < k1) {  // prefetch for the next plane
      load_plane(g, C, st, k + 2, pe);
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

    // (b) H^{n+1/2} on plane k: own cell and the low halo
    const int zx = sX >= 0 ? zx_of(g, j, k, sX) : 0;
    const int zy = sY >= 0 ? zy_of(g, i, k, sY) : 0;
    const int zz = sZ >= 0 ? zz_of(g, i, j, sZ) : 0;
    float hx = 0.f, hy = 0.f, hz = 0.f;
    const bool lay = (sX & sY & sZ) >= 0;  // some axis is in a layer (slab indices are -1 off them, all bits set)
    if (own && !lay) {  // off the layers 1/kappa = 1 exactly: the plain Yee update
      hx = hox - S * ((ek[2][ry + 1][rx] - ek[2][ry][rx]) - (ek1[1][ry][rx] - ek[1][ry][rx]));
      hy = hoy - S * ((ek1[0][ry][rx] - ek[0][ry][rx]) - (ek[2][ry][rx + 1] - ek[2][ry][rx]));
      hz = hoz - S * ((ek[1][ry][rx + 1] - ek[1][ry][rx]) - (ek[0][ry + 1][rx] - ek[0][ry][rx]));
    } else if (own) {
      hx = hox - S * (cterm<true>(ek[2][ry + 1][rx] - ek[2][ry][rx], ikYh, sY, T.b[1][1], T.c[1][1], j, PHi.p[0][1], PHo.p[0][1], zy) -
                      cterm<true>(ek1[1][ry][rx] - ek[1][ry][rx], ikZh, sZ, T.b[2][1], T.c[2][1], k, PHi.p[0][2], PHo.p[0][2], zz));
      hy = hoy - S * (cterm<true>(ek1[0][ry][rx] - ek[0][ry][rx], ikZh, sZ, T.b[2][1], T.c[2][1], k, PHi.p[1][2], PHo.p[1][2], zz) -
                      cterm<true>(ek[2][ry][rx + 1] - ek[2][ry][rx], ikXh, sX, T.b[0][1], T.c[0][1], i, PHi.p[1][0], PHo.p[1][0], zx));
      hz = hoz - S * (cterm<true>(ek[1][ry][rx + 1] - ek[1][ry][rx], ikXh, sX, T.b[0][1], T.c[0][1], i, PHi.p[2][0], PHo.p[2][0], zx) -
                      cterm<true>(ek[0][ry + 1][rx] - ek[0][ry][rx], ikYh, sY, T.b[1][1], T.c[1][1], j, PHi.p[2][1], PHo.p[2][1], zy));
    }
    if (own) {
      sH[0][ry][rx] = hx;
      sH[1][ry][rx] = hy;
      sH[2][ry][rx] = hz;
      N.f[3][q] = hx;
      N.f[4][q] = hy;
      N.f[5][q] = hz;
    }
    if (hrow) {  // (i, j0 - 1): staged at row 0, column tid + 1
      const int c = tid + 1;
      const int hzy = sYh >= 0 ? zy_of(g, xh, k, sYh) : 0, hzz = sZ >= 0 ? zz_of(g, xh, yh, sZ) : 0;
      const int hzx = sXh >= 0 ? zx_of(g, yh, k, sXh) : 0;
      sH[0][0][c] = ho1 - S * (cterm<false>(ek[2][1][c] - ek[2][0][c], ikYhh, sYh, T.b[1][1], T.c[1][1], yh, PHi.p[0][1], nullptr, hzy) -
                               cterm<false>(ek1[1][0][c] - ek[1][0][c], ikZh, sZ, T.b[2][1], T.c[2][1], k, PHi.p[0][2], nullptr, hzz));
      sH[2][0][c] = ho2 - S * (cterm<false>(ek[1][0][c + 1] - ek[1][0][c], ikXhh, sXh, T.b[0][1], T.c[0][1], xh, PHi.p[2][0], nullptr, hzx) -
                               cterm<false>(ek[0][1][c] - ek[0][0][c], ikYhh, sYh, T.b[1][1], T.c[1][1], yh, PHi.p[2][1], nullptr, hzy));
    }
    if (hcol) {  // (i0 - 1, j0 + hr): staged at row hr + 1, column 0
      const int r = hr + 1;
      const int hzy = sYh >= 0 ? zy_of(g, xh, k, sYh) : 0, hzz = sZ >= 0 ? zz_of(g, xh, yh, sZ) : 0;
      const int hzx = sXh >= 0 ? zx_of(g, yh, k, sXh) : 0;
      sH[1][r][0] = ho1 - S * (cterm<false>(ek1[0][r][0] - ek[0][r][0], ikZh, sZ, T.b[2][1], T.c[2][1], k, PHi.p[1][2], nullptr, hzz) -
                               cterm<false>(ek[2][r][1] - ek[2][r][0], ikXhh, sXh, T.b[0][1], T.c[0][1], xh, PHi.p[1][0], nullptr, hzx));
      sH[2][r][0] = ho2 - S * (cterm<false>(ek[1][r][1] - ek[1][r][0], ikXhh, sXh, T.b[0][1], T.c[0][1], xh, PHi.p[2][0], nullptr, hzx) -
                               cterm<false>(ek[0][r + 1][0] - ek[0][r][0], ikYhh, sYh, T.b[1][1], T.c[1][1], yh, PHi.p[2][1], nullptr, hzy));
    }
    if (fseg >= 0) face_write(A, fseg & 0xff, i, j, k, hx, hy, hz);
    if (fseg >= 0) face_write(A, fseg >> 8, i, j, k, hx, hy, hz);
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
      if (!lay && i > 0 && j > 0 && k > 0) {
        ex += Sa * ((hz - sH[2][ry - 1][rx]) - (hy - hym));
        ey += Sa * ((hx - hxm) - (hz - sH[2][ry][rx - 1]));
        ez += Sa * ((hy - sH[1][ry][rx - 1]) - (hx - sH[0][ry - 1][rx]));
      } else {
      if (j > 0 && k > 0)
        ex += Sa * (cterm<true>(hz - sH[2][ry - 1][rx], ikYe, sY, T.b[1][0], T.c[1][0], j, PEi.p[0][1], PEo.p[0][1], zy) -
                    cterm<true>(hy - hym, ikZe, sZ, T.b[2][0], T.c[2][0], k, PEi.p[0][2], PEo.p[0][2], zz));
      if (i > 0 && k > 0)
        ey += Sa * (cterm<true>(hx - hxm, ikZe, sZ, T.b[2][0], T.c[2][0], k, PEi.p[1][2], PEo.p[1][2], zz) -
                    cterm<true>(hz - sH[2][ry][rx - 1], ikXe, sX, T.b[0][0], T.c[0][0], i, PEi.p[1][0], PEo.p[1][0], zx));
      if (i > 0 && j > 0)
        ez += Sa * (cterm<true>(hy - sH[1][ry][rx - 1], ikXe, sX, T.b[0][0], T.c[0][0], i, PEi.p[2][0], PEo.p[2][0], zx) -
                    cterm<true>(hx - sH[0][ry - 1][rx], ikYe, sY, T.b[1][0], T.c[1][0], j, PEi.p[2][1], PEo.p[2][1], zy));
      }
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
