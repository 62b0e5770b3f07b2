// Fused adjoint step of arXiv 2412.12360 Sec. 2.2: the reverse-mode (transposed) E and H updates of one
// time step in a single sweep over the grid, with the CPML memories' adjoints, on adjoint fields that
// are double-buffered (read `cur`, write `nxt`).
//
// The forward step is H' = H - S curl_f(E) (with psi_H), E' = E + S a curl_b(H') (with psi_E). Its
// transpose, for the adjoint fields (Ebar, Hbar) of (E', H'), is
//   (A) Hbar_new = Hbar + [transpose of the E update] applied to u = S a Ebar   (with psi-bar_E),
//   (B) Ebar_new = Ebar + [transpose of the H update] applied to w = -S Hbar_new (with psi-bar_H),
// where, for an E point of component c and a transverse axis d, the coefficient of the E update along
// d is P = sv / kappa_d + c_d (psibar + sv) with sv = +-u_c (plain value +-u off the layers), the
// memory update psibar <- b_d (psibar + sv), and Hbar_h(p) gathers P1_{h+1}(p) - P1_{h+1}(p + e_{h+2})
// + P2_{h+2}(p) - P2_{h+2}(p + e_{h+1}); (B) mirrors it with w, the H tables and the -x/-y/-z
// neighbours: Ebar_e(p) += Q1_{e+1}(p - e_{e+2}) - Q1_{e+1}(p) + Q2_{e+2}(p - e_{e+1}) - Q2_{e+2}(p).
// Off the layers and on their inner edge the CPML part of P and Q is exactly 0, so each coefficient is
// the plain +-u (or +-w) plus, for each layer axis, the correction sv (1/kappa - 1) + c (psibar + sv).
// Tangential E held by a PEC wall (index 0) has Ebar = 0 and u = 0.
//
// (B) reads Hbar_new at p - x, p - y and p - z, so a block owns a TX x TY column tile and marches its
// z-chunk UPWARDS, as the forward kernel does: per plane it computes Hbar_new for its cells and,
// redundantly, for the column x = i0 - 1 and the row y = j0 - 1, then Ebar_new; Hbar_new of the plane
// below stays in registers, and the chunk's first plane recomputes the one below the chunk. (A) reads u
// at p + x, p + y and p + z, so the staged Ebar and a boxes carry a one-cell halo on both sides and
// the plane above is staged too. Hbar_new of a cell is computed by one function whether the cell is
// the block's own or the halo of a neighbouring tile, so the result does not depend on the tiling.
//
// The adjoints of detectors that read only E after a step (points on E components, |E|^2 boxes) of
// step det_step are added to Ebar_new here, from E of that step in the primal buffer `prim`.
// Each thread updates two x-adjacent cells.
//
// Tiles that touch an x or y layer run a second copy of the plane loop. There, each thread copies the
// x/y psi-bar values of its own cells (and the halo threads those of their halo cells) into private
// shared-memory slots one phase before they are used (cp.async), and a neighbour's coefficient is
// taken from the thread that computed it for its own cell (warp shuffles along x and between the two
// rows of a warp) wherever that thread is in the same warp. Every coefficient is still computed by the
// same function from the same values, so the bits are those of the direct form.
#include "../../include/fdtd.h"
#include "fdtd_internal.cuh"
#include "fdtd_tma.cuh"

namespace fdtd {

namespace {

constexpr int TX = 32, TY = 16, NT = 256;
constexpr int LX = TX / 2;
static_assert(NT == LX * TY && LX == 16, "one thread per cell pair, two tile rows per warp");

// staged boxes, all with origin (i0 - 4, j0 - 1) (x coordinate 16-byte aligned): Ebar and a over the
// tile with both halos, Hbar over the tile with the low halo. Cell (x, y) sits at [y - j0 + 1][x - i0 + 4].
constexpr int BW = TX + 8, BH = TY + 2;   // Ebar, a
constexpr int GW = TX + 4, GH = TY + 1;   // Hbar
constexpr int XO = 4;
constexpr uint32_t EB_BYTES = 3 * BW * BH * 4, HB_BYTES = 3 * GW * GH * 4, A_BYTES = BW * BH * 4;
constexpr uint32_t STAGE_TX = EB_BYTES + HB_BYTES + A_BYTES;
constexpr int round128(int b) { return (b + 127) / 128 * 128; }
constexpr int EB_OFF = 0, HB_OFF = round128(EB_BYTES), A_OFF = HB_OFF + round128(HB_BYTES);
constexpr int STAGE_BYTES = round128(A_OFF + A_BYTES);
// Hbar_new of a plane with the low halo: [3][NY][NX], row 0 = y j0 - 1, column 1 = x i0 - 1, own cell
// (x, y) at [y - j0 + 1][x - i0 + 2] (column 0 pads, so that every pair starts at an even column)
constexpr int NX = TX + 2, NY = TY + 1;
static_assert(BW % 2 == 0 && GW % 2 == 0 && NX % 2 == 0 && XO % 2 == 0, "float2 pairs");
static_assert((BW * BH) % 2 == 0 && (GW * GH) % 2 == 0 && (NX * NY) % 2 == 0, "float2 pairs");
constexpr int MAXTZ = 256;
constexpr int SH_OFF = 0;                                          // [2][3][NY][NX]
constexpr int PF_OFF = SH_OFF + round128(2 * 3 * NY * NX * 4);     // per-plane flags [MAXTZ]

typedef const float (*Box3)[BH][BW];
typedef const float (*Box1)[BW];
typedef const float (*GBox3)[GH][GW];

template <bool B>
struct Flag {
  static constexpr bool value = B;
};

__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }

__device__ __forceinline__ void cp8(float2* dst, const float2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ int box_offset(const int lo[3], const int hi[3], int x, int y, int k) {
  return ((k - lo[2]) * (hi[1] - lo[1]) + (y - lo[1])) * (hi[0] - lo[0]) + (x - lo[0]);
}

// This kernel keeps the two psi-bar memories of one axis side by side, one float2 per position (axis
// x: the y then the z component; axis y: x then z; axis z: x then y), in the space a PsiSet gives that
// axis's two arrays, so a cell's pair of memories is one 8-byte access. (The arrays are the adjoint
// step's own: zeroed before the sweep and read by no other kernel.)
__device__ __forceinline__ float2* psi2(const PsiSet& P, int d) {
  return reinterpret_cast<float2*>(P.p[d == 0 ? 1 : 0][d]);
}

// psi index of (x, y, k) for the derivative along x, y or z, slab index s
__device__ __forceinline__ int zx_of(const Geo& g, int y, int k, int s) { return (k * g.n[1] + y) * g.slab[0] + s; }
__device__ __forceinline__ int zy_of(const Geo& g, int x, int k, int s) { return (k * g.slab[1] + s) * g.nxp + x; }
__device__ __forceinline__ int zz_of(const Geo& g, int x, int y, int s) { return (s * g.n[1] + y) * g.nxp + x; }

// CPML part of one adjoint coefficient inside a layer: sv (1/kappa - 1) + c (psibar + sv), with
// km1 = 1/kappa - 1 from the tables, as one fused multiply-add (explicit, so that every evaluation of a
// coefficient rounds the same way and gives the same bits)
__device__ __forceinline__ float acorr(float sv, float km1, float c, float psi) {
  return __fmaf_rn(sv, km1, __fmul_rn(c, __fadd_rn(psi, sv)));
}
// the memory update psibar <- b (psibar + sv)
__device__ __forceinline__ float amem(float sv, float b, float psi) { return __fmul_rn(b, __fadd_rn(psi, sv)); }

struct Ring {
  unsigned char* base;
  uint64_t* bar;
  int kb;  // first plane staged (the ring is filled upwards from it)
  int ns;
  __device__ int slot(int p) const { return (p - kb) % ns; }
  __device__ uint32_t parity(int p) const { return ((p - kb) / ns) & 1; }
  __device__ Box3 Eb(int p) const { return reinterpret_cast<Box3>(base + slot(p) * STAGE_BYTES + EB_OFF); }
  __device__ GBox3 Hb(int p) const { return reinterpret_cast<GBox3>(base + slot(p) * STAGE_BYTES + HB_OFF); }
  __device__ Box1 Av(int p) const { return reinterpret_cast<Box1>(base + slot(p) * STAGE_BYTES + A_OFF); }
  __device__ bool wait(int p) const { return mbar_wait(&bar[slot(p)], parity(p)); }
  __device__ void issue(const AdjMaps& M, int i0, int j0, int p) const {
    unsigned char* st = base + slot(p) * STAGE_BYTES;
    uint64_t* b = &bar[slot(p)];
    mbar_arrive_expect(b, STAGE_TX);
    tma_load_box(st + EB_OFF, &M.eb, i0 - XO, j0 - 1, p, 0, b);
    tma_load_box(st + HB_OFF, &M.hb, i0 - XO, j0 - 1, p, 0, b);
    tma_load_box(st + A_OFF, &M.a, i0 - XO, j0 - 1, p, 0, b);
  }
};

// u_c = S a Ebar_c, zero where E_c is held by a PEC wall (index 0 along an axis transverse to c);
// beyond the grid the staged values are 0. Rounded as (S a) Ebar everywhere.
__device__ __forceinline__ float u_val(float Sa, float e, bool held) { return held ? 0.f : __fmul_rn(Sa, e); }

// The u values (A) reads at one cell p: its own three, those of the +x, +y and +z neighbours that its
// Hbar components gather.
struct UA {
  float ux, uy, uz, uz_x, uy_x, uz_y, ux_y, uy_z, ux_z;
};

// u values of the x-adjacent cell pair (x, y), (x + 1, y) at box position (bx, by) (bx even) of plane k,
// Eu/Au plane k + 1 (null beyond the grid): the staged planes are read as float2 pairs and the u of
// cell 1 serves as the +x neighbour of cell 0.
__device__ __forceinline__ void pair_u(float S, int x, int y, int k, int bx, int by, Box3 E, Box1 Av, Box3 Eu, Box1 Au,
                                       UA u[2]) {
  const float2 e0 = ld2(&E[0][by][bx]), e1 = ld2(&E[1][by][bx]), e2 = ld2(&E[2][by][bx]);
  const float2 av = ld2(&Av[by][bx]);
  const float sa[3] = {__fmul_rn(S, av.x), __fmul_rn(S, av.y), __fmul_rn(S, Av[by][bx + 2])};
  const float2 ex1 = ld2(&E[0][by + 1][bx]), ez1 = ld2(&E[2][by + 1][bx]);
  const float2 ay = ld2(&Av[by + 1][bx]);
  const float say[2] = {__fmul_rn(S, ay.x), __fmul_rn(S, ay.y)};
  float2 eyu = make_float2(0.f, 0.f), exu = make_float2(0.f, 0.f), au = make_float2(0.f, 0.f);
  if (Eu) {
    eyu = ld2(&Eu[1][by][bx]);
    exu = ld2(&Eu[0][by][bx]);
    au = ld2(&Au[by][bx]);
  }
  const float sau[2] = {__fmul_rn(S, au.x), __fmul_rn(S, au.y)};
  const float ey2 = E[1][by][bx + 2], ez2 = E[2][by][bx + 2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int xc = x + c;
    u[c].ux = u_val(sa[c], c ? e0.y : e0.x, y == 0 || k == 0);
    u[c].uy = u_val(sa[c], c ? e1.y : e1.x, xc == 0 || k == 0);
    u[c].uz = u_val(sa[c], c ? e2.y : e2.x, xc == 0 || y == 0);
    u[c].uz_y = u_val(say[c], c ? ez1.y : ez1.x, xc == 0);
    u[c].ux_y = u_val(say[c], c ? ex1.y : ex1.x, k == 0);
    u[c].uy_z = u_val(sau[c], c ? eyu.y : eyu.x, xc == 0);
    u[c].ux_z = u_val(sau[c], c ? exu.y : exu.x, y == 0);
  }
  u[0].uz_x = u[1].uz;  // the +x neighbour of cell 0 is cell 1 (x + 1 > 0: the same masks)
  u[0].uy_x = u[1].uy;
  u[1].uz_x = u_val(sa[2], ez2, y == 0);
  u[1].uy_x = u_val(sa[2], ey2, k == 0);
}

// u values of one cell at box position (bx, by) of plane k (the halo column)
__device__ __forceinline__ void cell_u(float S, int x, int y, int k, int bx, int by, Box3 E, Box1 Av, Box3 Eu, Box1 Au,
                                       UA& u) {
  const float sa = __fmul_rn(S, Av[by][bx]), sax = __fmul_rn(S, Av[by][bx + 1]), say = __fmul_rn(S, Av[by + 1][bx]);
  u.ux = u_val(sa, E[0][by][bx], y == 0 || k == 0);
  u.uy = u_val(sa, E[1][by][bx], x == 0 || k == 0);
  u.uz = u_val(sa, E[2][by][bx], x == 0 || y == 0);
  u.uz_x = u_val(sax, E[2][by][bx + 1], y == 0);
  u.uy_x = u_val(sax, E[1][by][bx + 1], k == 0);
  u.uz_y = u_val(say, E[2][by + 1][bx], x == 0);
  u.ux_y = u_val(say, E[0][by + 1][bx], k == 0);
  u.uy_z = u.ux_z = 0.f;
  if (Eu) {
    const float sau = __fmul_rn(S, Au[by][bx]);
    u.uy_z = u_val(sau, Eu[1][by][bx], x == 0);
    u.ux_z = u_val(sau, Eu[0][by][bx], y == 0);
  }
}

// CPML coefficients of one position along an axis (integer positions for E, half positions for H):
// b, c and ik = 1/kappa - 1
struct Coef {
  float b, c, ik;
};

// Tables of the tile's x positions i0 - 1 .. i0 + TX and y positions j0 - 1 .. j0 + TY in shared memory:
// rows b, c, 1/kappa at integer positions, then at half positions
constexpr int TABX = TX + 2, TABY = TY + 2;

template <int W>
__device__ __forceinline__ Coef coef_at(const float (*tab)[W], int row0, int col) {
  return Coef{tab[row0][col], tab[row0 + 1][col], tab[row0 + 2][col]};
}

// Slab indices along x and y of a cell and of the neighbours the phases read (-1 off the layers)
struct Slabs {
  int sX, sX1, sXm, sY, sY1, sYm;
};

__device__ __forceinline__ Slabs slabs_of(const Geo& g, int x, int y) {
  const int nx = g.n[0], ny = g.n[1];
  Slabs s;
  s.sX = slab_of_pos(x, nx, g.pml[0], g.pml[1]);
  s.sX1 = x + 1 < nx ? slab_of_pos(x + 1, nx, g.pml[0], g.pml[1]) : -1;
  s.sXm = x > 0 ? slab_of_pos(x - 1, nx, g.pml[0], g.pml[1]) : -1;
  s.sY = slab_of_pos(y, ny, g.pml[2], g.pml[3]);
  s.sY1 = y + 1 < ny ? slab_of_pos(y + 1, ny, g.pml[2], g.pml[3]) : -1;
  s.sYm = y > 0 ? slab_of_pos(y - 1, ny, g.pml[2], g.pml[3]) : -1;
  return s;
}

// z-axis CPML data of one plane: slab index and the integer (E) and half (H) position coefficients
struct ZPlane {
  int s;
  Coef e, h;
};

__device__ __forceinline__ ZPlane zplane(const Geo& g, const Tables& T, int k) {
  ZPlane z;
  z.s = (k >= 0 && k < g.n[2]) ? slab_of_pos(k, g.n[2], g.pml[4], g.pml[5]) : -1;
  z.e = Coef{0.f, 0.f, 0.f};
  z.h = Coef{0.f, 0.f, 0.f};
  if (z.s >= 0) {
    z.e = Coef{T.b[2][0][k], T.c[2][0][k], __fsub_rn(T.ik[2][0][k], 1.f)};
    z.h = Coef{T.b[2][1][k], T.c[2][1][k], __fsub_rn(T.ik[2][1][k], 1.f)};
  }
  return z;
}

// The CPML coefficients of one cell along x or y, as (A) and (B) gather them: the pair (P1, P2) of the
// two E components transverse to the axis (A), or (Q1, Q2) of the two H components (B). A cell's
// coefficient is computed by these functions alone, whether for the cell itself (STORE: also its
// psi-bar memory update) or as the neighbour of another cell, so every evaluation gives the same bits.
struct CP {
  float a, b;
};
__device__ __forceinline__ CP cp0() { return CP{0.f, 0.f}; }

// (A) along x at (x, y, k), slab s: P1 of E_z from uz, P2 of E_y from -uy
// (psi-bar values given: p20, p10 the memories of E_z and E_y along x)
template <bool STORE>
__device__ __forceinline__ CP cpa_xv(const AdjArgs& A, const float (*tabX)[TABX], int y, int k, int cx, int s, float uz,
                                     float uy, float p20, float p10) {
  const Coef cf = coef_at(tabX, 0, cx);
  if (STORE) {
    const int z = zx_of(A.g, y, k, s);
    psi2(A.poutE, 0)[z] = make_float2(amem(-uy, cf.b, p10), amem(uz, cf.b, p20));
  }
  return CP{acorr(uz, cf.ik, cf.c, p20), acorr(-uy, cf.ik, cf.c, p10)};
}
template <bool STORE>
__device__ __forceinline__ CP cpa_x(const AdjArgs& A, const float (*tabX)[TABX], int y, int k, int cx, int s, float uz,
                                    float uy) {
  const int z = zx_of(A.g, y, k, s);
  const float2 v = psi2(A.pinE, 0)[z];
  return cpa_xv<STORE>(A, tabX, y, k, cx, s, uz, uy, v.y, v.x);
}
// (A) along y: P1 of E_x from ux, P2 of E_z from -uz
template <bool STORE>
__device__ __forceinline__ CP cpa_yv(const AdjArgs& A, const float (*tabY)[TABY], int x, int k, int cy, int s, float ux,
                                     float uz, float p01, float p21) {
  const Coef cf = coef_at(tabY, 0, cy);
  if (STORE) {
    const int z = zy_of(A.g, x, k, s);
    psi2(A.poutE, 1)[z] = make_float2(amem(ux, cf.b, p01), amem(-uz, cf.b, p21));
  }
  return CP{acorr(ux, cf.ik, cf.c, p01), acorr(-uz, cf.ik, cf.c, p21)};
}
template <bool STORE>
__device__ __forceinline__ CP cpa_y(const AdjArgs& A, const float (*tabY)[TABY], int x, int k, int cy, int s, float ux,
                                    float uz) {
  const int z = zy_of(A.g, x, k, s);
  const float2 v = psi2(A.pinE, 1)[z];
  return cpa_yv<STORE>(A, tabY, x, k, cy, s, ux, uz, v.x, v.y);
}
// (B) along x: Q1 of H_z from wz, Q2 of H_y from -wy (half-position tables)
template <bool STORE>
__device__ __forceinline__ CP cpb_xv(const AdjArgs& A, const float (*tabX)[TABX], int y, int k, int cx, int s, float wz,
                                     float wy, float p20, float p10) {
  const Coef cf = coef_at(tabX, 3, cx);
  if (STORE) {
    const int z = zx_of(A.g, y, k, s);
    psi2(A.poutH, 0)[z] = make_float2(amem(-wy, cf.b, p10), amem(wz, cf.b, p20));
  }
  return CP{acorr(wz, cf.ik, cf.c, p20), acorr(-wy, cf.ik, cf.c, p10)};
}
template <bool STORE>
__device__ __forceinline__ CP cpb_x(const AdjArgs& A, const float (*tabX)[TABX], int y, int k, int cx, int s, float wz,
                                    float wy) {
  const int z = zx_of(A.g, y, k, s);
  const float2 v = psi2(A.pinH, 0)[z];
  return cpb_xv<STORE>(A, tabX, y, k, cx, s, wz, wy, v.y, v.x);
}
// (B) along y: Q1 of H_x from wx, Q2 of H_z from -wz
template <bool STORE>
__device__ __forceinline__ CP cpb_yv(const AdjArgs& A, const float (*tabY)[TABY], int x, int k, int cy, int s, float wx,
                                     float wz, float p01, float p21) {
  const Coef cf = coef_at(tabY, 3, cy);
  if (STORE) {
    const int z = zy_of(A.g, x, k, s);
    psi2(A.poutH, 1)[z] = make_float2(amem(wx, cf.b, p01), amem(-wz, cf.b, p21));
  }
  return CP{acorr(wx, cf.ik, cf.c, p01), acorr(-wz, cf.ik, cf.c, p21)};
}
template <bool STORE>
__device__ __forceinline__ CP cpb_y(const AdjArgs& A, const float (*tabY)[TABY], int x, int k, int cy, int s, float wx,
                                    float wz) {
  const int z = zy_of(A.g, x, k, s);
  const float2 v = psi2(A.pinH, 1)[z];
  return cpb_yv<STORE>(A, tabY, x, k, cy, s, wx, wz, v.x, v.y);
}

// (A) along z at (x, y): the own and +z terms into cbx, cby
template <bool STORE>
__device__ __forceinline__ void za_terms(const AdjArgs& A, int x, int y, const UA& u, const ZPlane& zk, const ZPlane& zu,
                                         float& cbx, float& cby) {
  if (zk.s >= 0 || zu.s >= 0) {  // P1 of E_y (1, 2) and P2 of E_x (0, 2), own and at +z
    const Geo& g = A.g;
    const PsiSet& Pi = A.pinE;
    const PsiSet& Po = A.poutE;
    float d1y = 0.f, d2x = 0.f, m1y = 0.f, m2x = 0.f;
    if (zk.s >= 0) {
      const int z = zz_of(g, x, y, zk.s);
      const float2 v = psi2(Pi, 2)[z];
      const float p12 = v.y, p02 = v.x;
      d1y = acorr(u.uy, zk.e.ik, zk.e.c, p12);
      d2x = acorr(-u.ux, zk.e.ik, zk.e.c, p02);
      if (STORE) psi2(Po, 2)[z] = make_float2(amem(-u.ux, zk.e.b, p02), amem(u.uy, zk.e.b, p12));
    }
    if (zu.s >= 0) {
      const int z = zz_of(g, x, y, zu.s);
      const float2 v = psi2(Pi, 2)[z];
      m1y = acorr(u.uy_z, zu.e.ik, zu.e.c, v.y);
      m2x = acorr(-u.ux_z, zu.e.ik, zu.e.c, v.x);
    }
    cbx = __fadd_rn(cbx, __fsub_rn(d1y, m1y));
    cby = __fadd_rn(cby, __fsub_rn(d2x, m2x));
  }
}

// (A) output from the CPML sums: Hbar_new components in WANT from the u values and the old Hbar
template <int WANT>
__device__ __forceinline__ void a_out(const UA& u, float g0, float g1, float g2, float cbx, float cby, float cbz,
                                      float out[3]) {
  if (WANT & 1) out[0] = __fadd_rn(g0, __fadd_rn(__fadd_rn(__fsub_rn(u.uy, u.uy_z), __fsub_rn(u.uz_y, u.uz)), cbx));
  if (WANT & 2) out[1] = __fadd_rn(g1, __fadd_rn(__fadd_rn(__fsub_rn(u.uz, u.uz_x), __fsub_rn(u.ux_z, u.ux)), cby));
  if (WANT & 4) out[2] = __fadd_rn(g2, __fadd_rn(__fadd_rn(__fsub_rn(u.ux, u.ux_y), __fsub_rn(u.uy_x, u.uy)), cbz));
}

// (A) at one cell: Hbar_new components in WANT (bit h) from the u values and the old Hbar (g0..g2);
// (cx, cy) the cell's columns in the x and y tables, zk / zu the z data of planes k and k + 1.
// STORE: write this cell's psi-bar_E memories (own cells only). XY: x/y layers may be present.
template <int WANT, bool STORE, bool XY>
__device__ __forceinline__ void phase_a(const AdjArgs& A, const float (*tabX)[TABX], const float (*tabY)[TABY], int x,
                                        int y, int k, int cx, int cy, const Slabs& sl, const UA& u, float g0,
                                        float g1, float g2, const ZPlane& zk, const ZPlane& zu, float out[3]) {
  float cbx = 0.f, cby = 0.f, cbz = 0.f;
  if constexpr (XY) {
    if (sl.sX >= 0 || sl.sX1 >= 0) {  // along x: own and at +x
      const CP o = sl.sX >= 0 ? cpa_x<STORE>(A, tabX, y, k, cx, sl.sX, u.uz, u.uy) : cp0();
      const CP n = sl.sX1 >= 0 ? cpa_x<false>(A, tabX, y, k, cx + 1, sl.sX1, u.uz_x, u.uy_x) : cp0();
      cby = __fadd_rn(cby, __fsub_rn(o.a, n.a));
      cbz = __fadd_rn(cbz, __fsub_rn(o.b, n.b));
    }
    if (sl.sY >= 0 || sl.sY1 >= 0) {  // along y: own and at +y
      const CP o = sl.sY >= 0 ? cpa_y<STORE>(A, tabY, x, k, cy, sl.sY, u.ux, u.uz) : cp0();
      const CP n = sl.sY1 >= 0 ? cpa_y<false>(A, tabY, x, k, cy + 1, sl.sY1, u.ux_y, u.uz_y) : cp0();
      cbx = __fadd_rn(cbx, __fsub_rn(o.b, n.b));
      cbz = __fadd_rn(cbz, __fsub_rn(o.a, n.a));
    }
  }
  za_terms<STORE>(A, x, y, u, zk, zu, cbx, cby);
  a_out<WANT>(u, g0, g1, g2, cbx, cby, cbz, out);
}

// The x/y CPML memories one (A) evaluation reads: at the cell and at its +x and +y neighbours.
struct PsiXY {
  float xo20, xo10, xn20, xn10, yo01, yo21, yn01, yn21;
};

// phase_a (no psi-bar stores) with the x/y memories given rather than loaded
template <int WANT>
__device__ __forceinline__ void phase_a_given(const AdjArgs& A, const float (*tabX)[TABX], const float (*tabY)[TABY],
                                              int x, int y, int k, int cx, int cy, const Slabs& sl, const UA& u,
                                              float g0, float g1, float g2, const PsiXY& p, const ZPlane& zk,
                                              const ZPlane& zu, float out[3]) {
  float cbx = 0.f, cby = 0.f, cbz = 0.f;
  if (sl.sX >= 0 || sl.sX1 >= 0) {
    const CP o = sl.sX >= 0 ? cpa_xv<false>(A, tabX, y, k, cx, sl.sX, u.uz, u.uy, p.xo20, p.xo10) : cp0();
    const CP n = sl.sX1 >= 0 ? cpa_xv<false>(A, tabX, y, k, cx + 1, sl.sX1, u.uz_x, u.uy_x, p.xn20, p.xn10) : cp0();
    cby = __fadd_rn(cby, __fsub_rn(o.a, n.a));
    cbz = __fadd_rn(cbz, __fsub_rn(o.b, n.b));
  }
  if (sl.sY >= 0 || sl.sY1 >= 0) {
    const CP o = sl.sY >= 0 ? cpa_yv<false>(A, tabY, x, k, cy, sl.sY, u.ux, u.uz, p.yo01, p.yo21) : cp0();
    const CP n = sl.sY1 >= 0 ? cpa_yv<false>(A, tabY, x, k, cy + 1, sl.sY1, u.ux_y, u.uz_y, p.yn01, p.yn21) : cp0();
    cbx = __fadd_rn(cbx, __fsub_rn(o.b, n.b));
    cbz = __fadd_rn(cbz, __fsub_rn(o.a, n.a));
  }
  za_terms<false>(A, x, y, u, zk, zu, cbx, cby);
  a_out<WANT>(u, g0, g1, g2, cbx, cby, cbz, out);
}

// shared memory besides the Hbar_new tiles: the x and y tables
constexpr int TXT_OFF = round128(PF_OFF + MAXTZ);                  // [6][TABX]
constexpr int TYT_OFF = TXT_OFF + 6 * TABX * 4;                    // [6][TABY]
// x/y CPML memories of the own cells, copied ahead by each thread for itself (cp.async) one phase
// before they are used: psi-bar_E (for (A)) and psi-bar_H (for (B)), as the float2 pairs of psi2, slot
// 2 c for cell c's x pair and 2 c + 1 for its y pair
constexpr int NPS = 8;
constexpr int PSE_OFF = round128(TYT_OFF + 6 * TABY * 4);          // [NPS / 2][NT] float2
constexpr int PSH_OFF = PSE_OFF + NPS * NT * 4;                    // [NPS / 2][NT] float2
// the same for the low halo row (lane lx: cell c of its pair at 4 c + (x pair, x pair at +x, y pair, y
// pair at +y)) and column (lane lx: its cell at 0..3 likewise)
constexpr int PHR_OFF = PSH_OFF + NPS * NT * 4;                    // [8][LX] float2
constexpr int PHC_OFF = PHR_OFF + 16 * LX * 4;                     // [4][LX] float2
constexpr int BAR2_OFF = round128(PHC_OFF + 8 * LX * 4);
constexpr int RING2_OFF = round128(BAR2_OFF + 4 * 8);
constexpr int smem_total(int ns) { return RING2_OFF + ns * STAGE_BYTES + 128; }

// The adjoint step of one request for the block at tile (bx, by), z-chunk bz.
// PATH 0: a block runs the plane loop its tile needs (both loops compiled in); 1: the plain loop only;
// 2: the x/y CPML loop only (the caller maps the block to a tile that needs it)
template <int NSTAGE, int PATH>
__device__ __forceinline__ void adj_body(const AdjArgs& A, const AdjMaps& M, const int bx, const int by, const int bz) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
  float(*sHn)[3][NY][NX] = reinterpret_cast<float(*)[3][NY][NX]>(sm + SH_OFF);
  unsigned char* pflag = sm + PF_OFF;
  float(*tabX)[TABX] = reinterpret_cast<float(*)[TABX]>(sm + TXT_OFF);
  float(*tabY)[TABY] = reinterpret_cast<float(*)[TABY]>(sm + TYT_OFF);
  // slots of float2 pairs (one axis's two memories): own cell c at 2 c + (0: x, 1: y); halo cell c at
  // 4 c + (x own, x at +x, y own, y at +y)
  float2(*sPE)[NT] = reinterpret_cast<float2(*)[NT]>(sm + PSE_OFF);
  float2(*sPH)[NT] = reinterpret_cast<float2(*)[NT]>(sm + PSH_OFF);
  float2(*sHR)[LX] = reinterpret_cast<float2(*)[LX]>(sm + PHR_OFF);
  float2(*sHC)[LX] = reinterpret_cast<float2(*)[LX]>(sm + PHC_OFF);

  const Geo& g = A.g;
  const Tables& T = A.T;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int lx = lane & (LX - 1), ty = 2 * warp + (lane >> 4);
  const int i0 = bx * TX, j0 = by * TY;
  const int k0 = bz * A.tz;
  const int k1 = min(g.n[2], k0 + A.tz);
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int plane = (int)g.plane;
  const int i = i0 + 2 * lx, j = j0 + ty;
  const bool own0 = i < nx && j < ny, own1 = i + 1 < nx && j < ny;
  const int q0 = j * g.nxp + i;
  const float S = g.S;
  const int kb = k0 > 0 ? k0 - 1 : 0;           // planes staged: kb .. klast
  const int klast = k1 < nz ? k1 : k1 - 1;
  const Ring R{sm + RING2_OFF, reinterpret_cast<uint64_t*>(sm + BAR2_OFF), kb, NSTAGE};
  const int bx0 = 2 * lx + XO, by0 = ty + 1;    // own cell 0 in the staged boxes
  const int rx = 2 * lx + 2, ry = ty + 1;        // own cell 0 in the Hbar_new tile
  const int cx0 = 2 * lx + 1, cy0 = ty + 1;      // own cell 0 in the x and y tables
  bool waited = true;

  if (tid == 0) {
    for (int b = 0; b < NSTAGE; ++b) mbar_init(&R.bar[b], 1);
    mbar_init_fence();
  }
  // CPML tables of the tile's positions (clamped into the grid; entries beyond it are not used)
  for (int t = tid; t < 6 * (TABX + TABY); t += NT) {
    const bool isx = t < 6 * TABX;
    const int u = isx ? t : t - 6 * TABX;
    const int row = isx ? u / TABX : u / TABY, col = isx ? u % TABX : u % TABY;
    const int ax = isx ? 0 : 1;
    const int pos = min(max((isx ? i0 : j0) - 1 + col, 0), g.n[ax] - 1);
    const int hf = row / 3, w = row % 3;
    const float* src = w == 0 ? T.b[ax][hf] : (w == 1 ? T.c[ax][hf] : T.ik[ax][hf]);
    const float v = src[pos];
    (isx ? tabX[row] : tabY[row])[col] = w == 2 ? __fsub_rn(v, 1.f) : v;  // 1/kappa - 1
  }
  {
    // per-plane flags: bit 1 a folded detector meets the tile at that plane
    const int xa = i0, xb = min(i0 + TX, nx), ya = j0, yb = min(j0 + TY, ny);
    for (int p = tid; p < k1 - k0; p += NT) {
      const int k = k0 + p;
      int f = 0;
      if (A.det_step >= 0)
        for (int s = 0; s < A.ndet; ++s) {
          const DetDev& d = A.det[s];
          if (k >= d.lo[2] && k < d.hi[2] && d.lo[0] < xb && d.hi[0] > xa && d.lo[1] < yb && d.hi[1] > ya) f |= 2;
        }
      pflag[p] = (unsigned char)f;
    }
  }
  pdl_wait();
  if (tid == 0)
    for (int p = kb; p <= min(kb + NSTAGE - 1, klast); ++p) R.issue(M, i0, j0, p);
  __syncthreads();

  // halo roles: warp 3 lanes 0..15 the row y = j0 - 1 at the pair (i, i + 1) (Hbar_x, Hbar_z); warp 4
  // lanes 0..15 the column x = i0 - 1 at y = j0 + lx (Hbar_y, Hbar_z)
  const bool hrow = warp == 3 && lane < LX && j0 > 0 && i < nx;
  const bool hrow1 = hrow && i + 1 < nx;
  const int yc = j0 + lx;
  const bool hcol = warp == 4 && lane < LX && i0 > 0 && yc < ny;
  // whether the tile, its halos or their +x/+y neighbours reach an x or y layer (uniform over the
  // block): if not, only planes at a z layer have CPML work
  const bool tile_xy = i0 - 1 < g.pml[0] || i0 + TX >= nx - g.pml[1] - 1 || j0 - 1 < g.pml[2] ||
                       j0 + TY >= ny - g.pml[3] - 1;
  unsigned det_xy = 0;  // folded detectors whose box holds this pair's row and one of its cells
  if (A.det_step >= 0)
    for (int s = 0; s < A.ndet; ++s)
      if (own0 && j >= A.det[s].lo[1] && j < A.det[s].hi[1] && i + 1 >= A.det[s].lo[0] && i < A.det[s].hi[0])
        det_xy |= 1u << s;
  // slab indices of the own pair and the halo cells (constant over the march)
  const Slabs sl0 = slabs_of(g, min(i, nx - 1), min(j, ny - 1)), sl1 = slabs_of(g, min(i + 1, nx - 1), min(j, ny - 1));
  const Slabs slr0 = slabs_of(g, min(i, nx - 1), max(j0 - 1, 0)), slr1 = slabs_of(g, min(i + 1, nx - 1), max(j0 - 1, 0));
  const Slabs slc = slabs_of(g, max(i0 - 1, 0), min(yc, ny - 1));

  auto march = [&](auto xy_tag) {
    constexpr bool XY = decltype(xy_tag)::value;
    // copies of the own cells' x/y CPML memories of plane kk (psi-bar_E for (A), psi-bar_H for (B))
    // into this thread's slots, one commit group each (tiles with x/y layers only)
    auto fetch_slots = [&](const PsiSet& P, float2 (*slot)[NT], int kk, bool halo) {
      const float2* px = psi2(P, 0);
      const float2* py = psi2(P, 1);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!(c == 0 ? own0 : own1)) continue;
        const Slabs& sl = c ? sl1 : sl0;
        if (sl.sX >= 0) cp8(&slot[2 * c][tid], px + zx_of(g, j, kk, sl.sX));
        if (sl.sY >= 0) cp8(&slot[2 * c + 1][tid], py + zy_of(g, i + c, kk, sl.sY));
      }
      // (A) of the halo row and column reads the memories at the halo cell and its +x, +y neighbours
      auto fetch_halo = [&](float2 (*hs)[LX], int m0, int x, int y, const Slabs& sl) {
        if (sl.sX >= 0) cp8(&hs[m0][lx], px + zx_of(g, y, kk, sl.sX));
        if (sl.sX1 >= 0) cp8(&hs[m0 + 1][lx], px + zx_of(g, y, kk, sl.sX1));
        if (sl.sY >= 0) cp8(&hs[m0 + 2][lx], py + zy_of(g, x, kk, sl.sY));
        if (sl.sY1 >= 0) cp8(&hs[m0 + 3][lx], py + zy_of(g, x, kk, sl.sY1));
      };
      if (halo && hrow) {
        fetch_halo(sHR, 0, i, j0 - 1, slr0);
        if (hrow1) fetch_halo(sHR, 4, i + 1, j0 - 1, slr1);
      }
      if (halo && hcol) fetch_halo(sHC, 0, i0 - 1, yc, slc);
      cp_commit();
    };
    // Hbar_new (x and y components) of the own pair at the plane below the one being updated
    float hxm[2] = {0.f, 0.f}, hym[2] = {0.f, 0.f};
    waited &= R.wait(kb);
    ZPlane zm = zplane(g, T, k0 - 1), zk = zplane(g, T, k0), zu;
    if (k0 > 0) {
      // plane k0 - 1 (its owner stores it; this block recomputes it from the staged planes)
      const int km = k0 - 1;
      waited &= R.wait(k0);
      if (own0) {
        UA u[2];
        pair_u(S, i, j, km, bx0, by0, R.Eb(km), R.Av(km), R.Eb(k0), R.Av(k0), u);
        const GBox3 G = R.Hb(km);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (c == 1 && !own1) continue;
          float o[3];
          phase_a<3, false, XY>(A, tabX, tabY, i + c, j, km, cx0 + c, cy0, c ? sl1 : sl0, u[c], G[0][by0][bx0 + c],
                                G[1][by0][bx0 + c], G[2][by0][bx0 + c], zm, zk, o);
          hxm[c] = o[0];
          hym[c] = o[1];
        }
      }
      __syncthreads();  // every thread is done with plane k0 - 1
      if (tid == 0 && km + NSTAGE <= klast) {
        async_proxy_fence();
        R.issue(M, i0, j0, km + NSTAGE);
      }
    }

    if constexpr (XY) {
      fetch_slots(A.pinE, sPE, k0, true);
      fetch_slots(A.pinH, sPH, k0, false);
    }
    for (int k = k0; k < k1; ++k) {
      const int it = k - k0;
      const int q = k * plane + q0;
      const int pf = pflag[it];
      const bool up = k + 1 < nz;
      zu = zplane(g, T, up ? k + 1 : -1);
      if (up) waited &= R.wait(k + 1);  // plane k was waited for before
      const Box3 Ek = R.Eb(k);
      const Box1 Ak = R.Av(k);
      const Box3 Eu = up ? R.Eb(k + 1) : nullptr;
      const Box1 Au = up ? R.Av(k + 1) : nullptr;
      const GBox3 Gk = R.Hb(k);
      float(*sH)[NY][NX] = sHn[it & 1];

      // (A) Hbar_new of the own pair, and Ebar of the pair (kept for (B))
      float hn[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
      float2 eo[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      if constexpr (XY) {
        // x/y layers: the own cells' coefficients first; a +x or +y neighbour's coefficient is then
        // taken from the thread that owns it (+x of cell 1: the next lane's cell 0; +y of the warp's
        // first row: the lane 16 above), and computed here only where that owner is in another warp
        // or tile (the tile row's last pair, the warp's second row)
        UA u[2];
        CP ox[2] = {cp0(), cp0()}, oy[2] = {cp0(), cp0()};
        cp_wait_all_but_one();  // this plane's psi-bar_E slots (its psi-bar_H copies may still be in flight)
        if (own0) {
          pair_u(S, i, j, k, bx0, by0, Ek, Ak, Eu, Au, u);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            if (c == 1 && !own1) continue;
            const Slabs& sl = c ? sl1 : sl0;
            if (sl.sX >= 0)
              ox[c] = cpa_xv<true>(A, tabX, j, k, cx0 + c, sl.sX, u[c].uz, u[c].uy, sPE[2 * c][tid].y, sPE[2 * c][tid].x);
            if (sl.sY >= 0)
              oy[c] = cpa_yv<true>(A, tabY, i + c, k, cy0, sl.sY, u[c].ux, u[c].uz, sPE[2 * c + 1][tid].x,
                                   sPE[2 * c + 1][tid].y);
          }
        }
        CP nx1, ny[2];
        nx1.a = __shfl_down_sync(0xffffffffu, ox[0].a, 1, LX);
        nx1.b = __shfl_down_sync(0xffffffffu, ox[0].b, 1, LX);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          ny[c].a = __shfl_down_sync(0xffffffffu, oy[c].a, LX);
          ny[c].b = __shfl_down_sync(0xffffffffu, oy[c].b, LX);
        }
        if (own0) {
          const float2 g0 = ld2(&Gk[0][by0][bx0]), g1 = ld2(&Gk[1][by0][bx0]), g2 = ld2(&Gk[2][by0][bx0]);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            if (c == 1 && !own1) continue;
            const Slabs& sl = c ? sl1 : sl0;
            float cbx = 0.f, cby = 0.f, cbz = 0.f;
            if (sl.sX >= 0 || sl.sX1 >= 0) {
              const CP n = c == 0 ? ox[1]  // cell 1 (0 beyond the grid)
                                  : (lx < LX - 1 ? nx1
                                                 : (sl.sX1 >= 0 ? cpa_x<false>(A, tabX, j, k, cx0 + 2, sl.sX1, u[1].uz_x,
                                                                               u[1].uy_x)
                                                                : cp0()));
              cby = __fadd_rn(cby, __fsub_rn(ox[c].a, n.a));
              cbz = __fadd_rn(cbz, __fsub_rn(ox[c].b, n.b));
            }
            if (sl.sY >= 0 || sl.sY1 >= 0) {
              const CP n = lane < LX ? ny[c]
                                     : (sl.sY1 >= 0 ? cpa_y<false>(A, tabY, i + c, k, cy0 + 1, sl.sY1, u[c].ux_y,
                                                                   u[c].uz_y)
                                                    : cp0());
              cbx = __fadd_rn(cbx, __fsub_rn(oy[c].b, n.b));
              cbz = __fadd_rn(cbz, __fsub_rn(oy[c].a, n.a));
            }
            za_terms<true>(A, i + c, j, u[c], zk, zu, cbx, cby);
            a_out<7>(u[c], c ? g0.y : g0.x, c ? g1.y : g1.x, c ? g2.y : g2.x, cbx, cby, cbz, hn[c]);
          }
#pragma unroll
          for (int e = 0; e < 3; ++e) eo[e] = ld2(&Ek[e][by0][bx0]);
          st2(&A.nxt.f[3][q], hn[0][0], hn[1][0]);
          st2(&A.nxt.f[4][q], hn[0][1], hn[1][1]);
          st2(&A.nxt.f[5][q], hn[0][2], hn[1][2]);
        }
      } else if (own0) {
        UA u[2];
        pair_u(S, i, j, k, bx0, by0, Ek, Ak, Eu, Au, u);
        const float2 g0 = ld2(&Gk[0][by0][bx0]), g1 = ld2(&Gk[1][by0][bx0]), g2 = ld2(&Gk[2][by0][bx0]);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (c == 1 && !own1) continue;
          phase_a<7, true, false>(A, tabX, tabY, i + c, j, k, cx0 + c, cy0, c ? sl1 : sl0, u[c], c ? g0.y : g0.x,
                                  c ? g1.y : g1.x, c ? g2.y : g2.x, zk, zu, hn[c]);
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) eo[e] = ld2(&Ek[e][by0][bx0]);
        st2(&A.nxt.f[3][q], hn[0][0], hn[1][0]);
        st2(&A.nxt.f[4][q], hn[0][1], hn[1][1]);
        st2(&A.nxt.f[5][q], hn[0][2], hn[1][2]);
      }
#pragma unroll
      for (int h = 0; h < 3; ++h) st2(&sH[h][ry][rx], hn[0][h], hn[1][h]);
      // the low halo row (i, j0 - 1), (i + 1, j0 - 1): Hbar_x, Hbar_z
      if (warp == 3 && lane < LX) {
        float r0[2] = {0.f, 0.f}, r2[2] = {0.f, 0.f};
        if (hrow) {
          UA u[2];
          pair_u(S, i, j0 - 1, k, bx0, 0, Ek, Ak, Eu, Au, u);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            if (c == 1 && !hrow1) continue;
            float o[3];
            if constexpr (XY) {
              const float2 hx = sHR[4 * c][lx], hxn = sHR[4 * c + 1][lx];
              const float2 hy = sHR[4 * c + 2][lx], hyn = sHR[4 * c + 3][lx];
              const PsiXY ps{hx.y, hx.x, hxn.y, hxn.x, hy.x, hy.y, hyn.x, hyn.y};
              phase_a_given<5>(A, tabX, tabY, i + c, j0 - 1, k, cx0 + c, 0, c ? slr1 : slr0, u[c], Gk[0][0][bx0 + c],
                               0.f, Gk[2][0][bx0 + c], ps, zk, zu, o);
            } else {
              phase_a<5, false, false>(A, tabX, tabY, i + c, j0 - 1, k, cx0 + c, 0, c ? slr1 : slr0, u[c],
                                       Gk[0][0][bx0 + c], 0.f, Gk[2][0][bx0 + c], zk, zu, o);
            }
            r0[c] = o[0];
            r2[c] = o[2];
          }
        }
        st2(&sH[0][0][rx], r0[0], r0[1]);
        st2(&sH[2][0][rx], r2[0], r2[1]);
      }
      // the low halo column (i0 - 1, j0 + lx): Hbar_y, Hbar_z
      if (warp == 4 && lane < LX) {
        float o[3] = {0.f, 0.f, 0.f};
        if (hcol) {
          UA u;
          cell_u(S, i0 - 1, yc, k, XO - 1, lx + 1, Ek, Ak, Eu, Au, u);
          if constexpr (XY) {
            const float2 hx = sHC[0][lx], hxn = sHC[1][lx], hy = sHC[2][lx], hyn = sHC[3][lx];
            const PsiXY ps{hx.y, hx.x, hxn.y, hxn.x, hy.x, hy.y, hyn.x, hyn.y};
            phase_a_given<6>(A, tabX, tabY, i0 - 1, yc, k, 0, lx + 1, slc, u, 0.f, Gk[1][lx + 1][XO - 1],
                             Gk[2][lx + 1][XO - 1], ps, zk, zu, o);
          } else {
            phase_a<6, false, false>(A, tabX, tabY, i0 - 1, yc, k, 0, lx + 1, slc, u, 0.f, Gk[1][lx + 1][XO - 1],
                                     Gk[2][lx + 1][XO - 1], zk, zu, o);
          }
        }
        sH[1][lx + 1][1] = o[1];
        sH[2][lx + 1][1] = o[2];
      }
      if constexpr (XY) {  // the next plane's psi-bar_E, into the slots (A) has just read
        if (k + 1 < k1) fetch_slots(A.pinE, sPE, k + 1, true);
        else cp_commit();
      }
      __syncthreads();  // the Hbar_new tile is complete; every thread is done with plane k's stage
      if (tid == 0 && k + NSTAGE <= klast) {
        async_proxy_fence();
        R.issue(M, i0, j0, k + NSTAGE);
      }

      // (B) Ebar_new of the own pair from Hbar_new of this plane (tile and halo) and of the plane below.
      // x/y layers: the own cells' coefficients first, a -x or -y neighbour's taken from the thread that
      // owns it (-x of cell 0: the previous lane's cell 1; -y of the warp's second row: the lane 16
      // below) or computed here where that owner is in another warp or tile
      CP bxo[2] = {cp0(), cp0()}, byo[2] = {cp0(), cp0()}, bxp = cp0(), byp[2] = {cp0(), cp0()};
      if constexpr (XY) {
        cp_wait_all_but_one();  // this plane's psi-bar_H slots (the next plane's psi-bar_E may be in flight)
        if (own0) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            if (c == 1 && !own1) continue;
            const Slabs& sl = c ? sl1 : sl0;
            const float wx = __fmul_rn(-S, hn[c][0]), wy = __fmul_rn(-S, hn[c][1]), wz = __fmul_rn(-S, hn[c][2]);
            if (sl.sX >= 0)
              bxo[c] = cpb_xv<true>(A, tabX, j, k, cx0 + c, sl.sX, wz, wy, sPH[2 * c][tid].y, sPH[2 * c][tid].x);
            if (sl.sY >= 0)
              byo[c] = cpb_yv<true>(A, tabY, i + c, k, cy0, sl.sY, wx, wz, sPH[2 * c + 1][tid].x, sPH[2 * c + 1][tid].y);
          }
        }
        if (k + 1 < k1) fetch_slots(A.pinH, sPH, k + 1, false);
        else cp_commit();
        bxp.a = __shfl_up_sync(0xffffffffu, bxo[1].a, 1, LX);
        bxp.b = __shfl_up_sync(0xffffffffu, bxo[1].b, 1, LX);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          byp[c].a = __shfl_up_sync(0xffffffffu, byo[c].a, LX);
          byp[c].b = __shfl_up_sync(0xffffffffu, byo[c].b, LX);
        }
      }
      if (own0) {
        const float2 hzs = ld2(&sH[2][ry - 1][rx]), hxs = ld2(&sH[0][ry - 1][rx]);  // at y - 1
        const float hyl = sH[1][ry][rx - 1], hzl = sH[2][ry][rx - 1];             // at x - 1 of cell 0
        float nb[2][3];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int x = i + c;
          const Slabs& sl = c ? sl1 : sl0;
          const int cx = cx0 + c;
          // Hbar_new at the cell and at its -x, -y, -z neighbours (the plane below the grid holds 0)
          const float hx = hn[c][0], hy = hn[c][1], hz = hn[c][2];
          const float hz_x = c ? hn[0][2] : hzl, hy_x = c ? hn[0][1] : hyl;
          const float hz_y = c ? hzs.y : hzs.x, hx_y = c ? hxs.y : hxs.x;
          const float hy_m = k > 0 ? hym[c] : 0.f, hx_m = k > 0 ? hxm[c] : 0.f;
          // w = -S Hbar_new, for the CPML terms
          const float wx = __fmul_rn(-S, hx), wy = __fmul_rn(-S, hy), wz = __fmul_rn(-S, hz);
          const float wz_x = __fmul_rn(-S, hz_x), wy_x = __fmul_rn(-S, hy_x);
          const float wz_y = __fmul_rn(-S, hz_y), wx_y = __fmul_rn(-S, hx_y);
          const float wy_m = __fmul_rn(-S, hy_m), wx_m = __fmul_rn(-S, hx_m);
          float cex = 0.f, cey = 0.f, cez = 0.f;
          const PsiSet& Pi = A.pinH;
          const PsiSet& Po = A.poutH;
          const bool ok = c == 0 || own1;
          if constexpr (XY) {
            if (ok && (sl.sX >= 0 || sl.sXm >= 0)) {  // along x: Q1 of H_z, Q2 of H_y, own and -x
              const CP n = c == 1 ? bxo[0]  // cell 0
                                  : (lx > 0 ? bxp
                                            : (sl.sXm >= 0 ? cpb_x<false>(A, tabX, j, k, cx - 1, sl.sXm, wz_x, wy_x)
                                                           : cp0()));
              cey = __fadd_rn(cey, __fsub_rn(n.a, bxo[c].a));
              cez = __fadd_rn(cez, __fsub_rn(n.b, bxo[c].b));
            }
            if (ok && (sl.sY >= 0 || sl.sYm >= 0)) {  // along y: Q1 of H_x, Q2 of H_z, own and -y
              const CP n = lane >= LX ? byp[c]
                                      : (sl.sYm >= 0 ? cpb_y<false>(A, tabY, x, k, cy0 - 1, sl.sYm, wx_y, wz_y)
                                                     : cp0());
              cex = __fadd_rn(cex, __fsub_rn(n.b, byo[c].b));
              cez = __fadd_rn(cez, __fsub_rn(n.a, byo[c].a));
            }
          }
          if (ok && (zk.s >= 0 || zm.s >= 0)) {  // along z: Q1 of H_y (1, 2), Q2 of H_x (0, 2), own and -z
            float e1y = 0.f, e2x = 0.f, m1y = 0.f, m2x = 0.f;
            if (zk.s >= 0) {
              const int z = zz_of(g, x, j, zk.s);
              const float2 v = psi2(Pi, 2)[z];
              const float p12 = v.y, p02 = v.x;
              e1y = acorr(wy, zk.h.ik, zk.h.c, p12);
              e2x = acorr(-wx, zk.h.ik, zk.h.c, p02);
              psi2(Po, 2)[z] = make_float2(amem(-wx, zk.h.b, p02), amem(wy, zk.h.b, p12));
            }
            if (zm.s >= 0) {
              const int z = zz_of(g, x, j, zm.s);
              const float2 v = psi2(Pi, 2)[z];
              m1y = acorr(wy_m, zm.h.ik, zm.h.c, v.y);
              m2x = acorr(-wx_m, zm.h.ik, zm.h.c, v.x);
            }
            cex = __fadd_rn(cex, __fsub_rn(m1y, e1y));
            cey = __fadd_rn(cey, __fsub_rn(m2x, e2x));
          }
          // the plain gather of the w values, -S (the H-update coefficient) applied once per component
          const float px = __fmul_rn(-S, __fadd_rn(__fsub_rn(hy_m, hy), __fsub_rn(hz, hz_y)));
          const float py = __fmul_rn(-S, __fadd_rn(__fsub_rn(hz_x, hz), __fsub_rn(hx, hx_m)));
          const float pz = __fmul_rn(-S, __fadd_rn(__fsub_rn(hx_y, hx), __fsub_rn(hy, hy_x)));
          nb[c][0] = __fadd_rn(c ? eo[0].y : eo[0].x, __fadd_rn(px, cex));
          nb[c][1] = __fadd_rn(c ? eo[1].y : eo[1].x, __fadd_rn(py, cey));
          nb[c][2] = __fadd_rn(c ? eo[2].y : eo[2].x, __fadd_rn(pz, cez));
        }
        if ((pf & 2) && det_xy) {  // folded detector adjoints, one after the other in detector order
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int x = i + c;
            if (c == 1 && !own1) continue;
            for (int s = 0; s < A.ndet; ++s) {
              const DetDev& d = A.det[s];
              if (!((det_xy >> s) & 1u) || k < d.lo[2] || k >= d.hi[2] || x < d.lo[0] || x >= d.hi[0]) continue;
              if (d.kind == FDTD_DET_POINT_SERIES) {
                const float v = (float)A.gy[d.off + A.det_step];
                if (d.comp == 0) nb[c][0] += v;
                else if (d.comp == 1) nb[c][1] += v;
                else nb[c][2] += v;
              } else {  // |E|^2 summed over the steps: dL/dE = 2 g E
                const double w = 2.0 * A.gy[d.off + box_offset(d.lo, d.hi, x, j, k)];
                const int64_t qq = (int64_t)q + c;
                nb[c][0] += (float)(w * (double)A.prim.f[0][qq]);
                nb[c][1] += (float)(w * (double)A.prim.f[1][qq]);
                nb[c][2] += (float)(w * (double)A.prim.f[2][qq]);
              }
            }
          }
        }
        // E components held by a PEC wall keep Ebar = 0; the pair's second cell beyond the grid is 0
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int x = i + c;
          const bool in = c == 0 || own1;
          if (!(in && j > 0 && k > 0)) nb[c][0] = 0.f;
          if (!(in && x > 0 && k > 0)) nb[c][1] = 0.f;
          if (!(in && x > 0 && j > 0)) nb[c][2] = 0.f;
        }
        st2(&A.nxt.f[0][q], nb[0][0], nb[1][0]);
        st2(&A.nxt.f[1][q], nb[0][1], nb[1][1]);
        st2(&A.nxt.f[2][q], nb[0][2], nb[1][2]);
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        hxm[c] = hn[c][0];
        hym[c] = hn[c][1];
      }
      zm = zk;
      zk = zu;
    }
  };
  if constexpr (PATH == 1) {
    march(Flag<false>{});
  } else if constexpr (PATH == 2) {
    march(Flag<true>{});
  } else {
    if (tile_xy) march(Flag<true>{});
    else march(Flag<false>{});
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // no slot copy outlives the block
  if (!waited) atomicOr(A.status, kStatusTimeout);
}

template <int NSTAGE>
__global__ void __launch_bounds__(NT, 2) k_adj_fused(const __grid_constant__ AdjArgs A, const __grid_constant__ AdjMaps M) {
  adj_body<NSTAGE, 0>(A, M, blockIdx.x, blockIdx.y, blockIdx.z);
}

// The plain tiles of a split step: the rectangle of tile columns [xl, ntx - xh) and rows [yl, nty - yh).
template <int NSTAGE>
__global__ void __launch_bounds__(NT, 2) k_adj_plain(const __grid_constant__ AdjArgs A, const __grid_constant__ AdjMaps M) {
  adj_body<NSTAGE, 1>(A, M, A.xl + (int)blockIdx.x, A.yl + (int)blockIdx.y, blockIdx.z);
}

// The x/y CPML tiles of a split step, blockIdx.x numbering the frame: the first yl rows whole, then the
// last yh rows whole, then the xl first and xh last columns of the rows between; blockIdx.y the z-chunk.
template <int NSTAGE>
__global__ void __launch_bounds__(NT, 2) k_adj_frame(const __grid_constant__ AdjArgs A, const __grid_constant__ AdjMaps M) {
  const int ntx = (A.g.n[0] + TX - 1) / TX, nty = (A.g.n[1] + TY - 1) / TY;
  int t = blockIdx.x, bx, by;
  if (t < A.yl * ntx) {
    by = t / ntx;
    bx = t % ntx;
  } else if ((t -= A.yl * ntx) < A.yh * ntx) {
    by = nty - A.yh + t / ntx;
    bx = t % ntx;
  } else {
    t -= A.yh * ntx;
    const int w = A.xl + A.xh;
    by = A.yl + t / w;
    const int r = t % w;
    bx = r < A.xl ? r : ntx - A.xh + (r - A.xl);
  }
  adj_body<NSTAGE, 2>(A, M, bx, by, blockIdx.y);
}

// Several requests in one launch (see k_fwd_fused_group).
template <int NSTAGE>
__global__ void __launch_bounds__(NT, 2) k_adj_fused_group(const __grid_constant__ AdjGroup G) {
  int bx, by, bz;
  const int r = group_locate(G.grid, bx, by, bz);
  adj_body<NSTAGE, 0>(G.a[r], G.m[r], bx, by, bz);
}

}  // namespace

void launch_adj_group(AdjGroup& G, cudaStream_t s) {
  const int total = group_fill(G.grid, G.n, [&](int r, int* nb) {
    const Geo& g = G.a[r].g;
    nb[0] = (g.n[0] + TX - 1) / TX;
    nb[1] = (g.n[1] + TY - 1) / TY;
    nb[2] = (g.n[2] + G.a[r].tz - 1) / G.a[r].tz;
  });
  if (total == 0) return;
  if (G.a[0].nstage == 4) launch_pdl(k_adj_fused_group<4>, dim3(total), dim3(NT), smem_total(4), s, G);
  else launch_pdl(k_adj_fused_group<3>, dim3(total), dim3(NT), smem_total(3), s, G);
}

MapBox adj_box_e() { return {BW, BH}; }
MapBox adj_box_h() { return {GW, GH}; }

int prepare_adj(int nstage, int* blocks_per_sm) {
  auto k = nstage == 4 ? k_adj_fused<4> : k_adj_fused<3>;
  auto kg = nstage == 4 ? k_adj_fused_group<4> : k_adj_fused_group<3>;
  auto kp = nstage == 4 ? k_adj_plain<4> : k_adj_plain<3>;
  auto kf = nstage == 4 ? k_adj_frame<4> : k_adj_frame<3>;
  const int smem = smem_total(nstage);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kg, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, NT, smem);
  return e == cudaSuccess ? FDTD_OK : set_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
}

int adj_max_tz() { return MAXTZ; }

int adj_tiles_x(const Geo& g) { return (g.n[0] + TX - 1) / TX; }
int adj_tiles_y(const Geo& g) { return (g.n[1] + TY - 1) / TY; }

// Whether tile column bx (axis 0) or row by (axis 1) needs the x/y CPML path: the tile, its halo or
// their neighbours reach a layer (the test the plane loop makes per block).
bool adj_tile_xy(const Geo& g, int axis, int b) {
  const int t = axis == 0 ? TX : TY, o = b * t, n = g.n[axis];
  return o - 1 < g.pml[2 * axis] || o + t >= n - g.pml[2 * axis + 1] - 1;
}

int launch_adj(const AdjArgs& a, const AdjMaps& m, cudaStream_t s, cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join) {
  const Geo& g = a.g;
  const int ntx = adj_tiles_x(g), nty = adj_tiles_y(g);
  if (!a.split) {
    dim3 grid(ntx, nty, (g.n[2] + a.tz - 1) / a.tz);
    if (a.nstage == 4) launch_pdl(k_adj_fused<4>, grid, dim3(NT), smem_total(4), s, a, m);
    else launch_pdl(k_adj_fused<3>, grid, dim3(NT), smem_total(3), s, a, m);
    return 1;
  }
  const int frame = (a.yl + a.yh) * ntx + (nty - a.yl - a.yh) * (a.xl + a.xh);
  dim3 gf(frame, (g.n[2] + a.tz_xy - 1) / a.tz_xy);
  dim3 gp(ntx - a.xl - a.xh, nty - a.yl - a.yh, (g.n[2] + a.tz - 1) / a.tz);
  AdjArgs af = a;
  af.tz = a.tz_xy;
  // with a second stream the two launches run side by side (they write disjoint tiles of the same
  // buffers): s2 waits for s's work so far, then s waits for s2's launch
  cudaStream_t sf = s;
  if (s2) {
    cudaEventRecord(fork, s);
    cudaStreamWaitEvent(s2, fork, 0);
    sf = s2;
  }
  if (a.nstage == 4) {
    launch_pdl(k_adj_frame<4>, gf, dim3(NT), smem_total(4), sf, af, m);
    launch_pdl(k_adj_plain<4>, gp, dim3(NT), smem_total(4), s, a, m);
  } else {
    launch_pdl(k_adj_frame<3>, gf, dim3(NT), smem_total(3), sf, af, m);
    launch_pdl(k_adj_plain<3>, gp, dim3(NT), smem_total(3), s, a, m);
  }
  if (s2) {
    cudaEventRecord(join, s2);
    cudaStreamWaitEvent(s, join, 0);
  }
  return 2;
}

}  // namespace fdtd
