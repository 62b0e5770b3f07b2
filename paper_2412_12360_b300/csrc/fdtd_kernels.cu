// Reference-structured CUDA kernels of libfdtd: one thread per cell, every step of the hot path as its
// own kernel. They define the arithmetic that the fused kernels (fdtd_fused.cu) reproduce, and they
// serve the small, launch-bound grids and the auxiliary copies.
//
// Forward (arXiv 2412.12360 Sec. 2.1, Eqs. 1-2): H^{n+1/2} = H^{n-1/2} - S curl E^n and
// E^{n+1} = E^n + S a curl H^{n+1/2}, each curl difference divided by kappa and corrected by the CPML
// memory psi <- b psi + c * difference inside the layers.
// Reverse (Sec. 2.2): the inverse update step on the PML-free region R, and the transpose of every
// forward statement for the adjoint fields, written in gather form so that each thread owns its outputs.
#include "fdtd_internal.cuh"

namespace fdtd {

namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ bool e_updated(int C, const int p[3]) {
  return p[(C + 1) % 3] != 0 && p[(C + 2) % 3] != 0;
}

// component lies in R (E: half along its own axis, integer along the others; H: the opposite)
__device__ __forceinline__ bool in_R(const Geo& g, int C, bool is_h, const int p[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const bool half = is_h ? (d != C) : (d == C);
    const int lo = half ? g.rhalf_lo[d] : g.rint_lo[d];
    const int hi = half ? g.rhalf_hi[d] : g.rint_hi[d];
    if (p[d] < lo || p[d] > hi) return false;
  }
  return true;
}

__device__ __forceinline__ bool cell_of(const Geo& g, int p[3]) {
  p[0] = blockIdx.x * BX + threadIdx.x;
  p[1] = blockIdx.y * BY + threadIdx.y;
  p[2] = blockIdx.z;
  return p[0] < g.n[0] && p[1] < g.n[1];
}

// ---------------------------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------------------------
template <int C>
__device__ __forceinline__ void h_update(const Geo& g, const Fields& F, const PsiSet& P, const Tables& T,
                                         const int p[3], int64_t q, const int64_t st[3]) {
  constexpr int C1 = (C + 1) % 3, C2 = (C + 2) % 3;
  const float* Ea = F.f[C2];  // differenced along C1
  const float* Eb = F.f[C1];  // differenced along C2
  const float ea1 = (p[C1] + 1 < g.n[C1]) ? Ea[q + st[C1]] : 0.f;
  const float eb2 = (p[C2] + 1 < g.n[C2]) ? Eb[q + st[C2]] : 0.f;
  const float d1 = ea1 - Ea[q];
  const float d2 = eb2 - Eb[q];
  float t1 = d1 * T.ik[C1][1][p[C1]];
  float t2 = d2 * T.ik[C2][1][p[C2]];
  const int s1 = slab_index(g, C1, p[C1]);
  if (s1 >= 0) {
    float* ps = P.p[C][C1] + psi_index(g, C1, p[0], p[1], p[2], s1);
    const float v = T.b[C1][1][p[C1]] * *ps + T.c[C1][1][p[C1]] * d1;
    *ps = v;
    t1 += v;
  }
  const int s2 = slab_index(g, C2, p[C2]);
  if (s2 >= 0) {
    float* ps = P.p[C][C2] + psi_index(g, C2, p[0], p[1], p[2], s2);
    const float v = T.b[C2][1][p[C2]] * *ps + T.c[C2][1][p[C2]] * d2;
    *ps = v;
    t2 += v;
  }
  F.f[3 + C][q] -= g.S * (t1 - t2);
}

__global__ void k_update_H(Geo g, Fields F, PsiSet P, Tables T) {
  int p[3];
  if (!cell_of(g, p)) return;
  const int64_t q = cell_index(g, p[0], p[1], p[2]);
  const int64_t st[3] = {1, g.nxp, g.plane};
  h_update<0>(g, F, P, T, p, q, st);
  h_update<1>(g, F, P, T, p, q, st);
  h_update<2>(g, F, P, T, p, q, st);
}

template <int C>
__device__ __forceinline__ void e_update(const Geo& g, const Fields& F, const PsiSet& P, const Tables& T,
                                         const float* a, const int p[3], int64_t q, const int64_t st[3]) {
  constexpr int C1 = (C + 1) % 3, C2 = (C + 2) % 3;
  if (!e_updated(C, p)) return;
  const float* Ha = F.f[3 + C2];  // differenced along C1
  const float* Hb = F.f[3 + C1];  // differenced along C2
  const float d1 = Ha[q] - Ha[q - st[C1]];
  const float d2 = Hb[q] - Hb[q - st[C2]];
  float t1 = d1 * T.ik[C1][0][p[C1]];
  float t2 = d2 * T.ik[C2][0][p[C2]];
  const int s1 = slab_index(g, C1, p[C1]);
  if (s1 >= 0) {
    float* ps = P.p[C][C1] + psi_index(g, C1, p[0], p[1], p[2], s1);
    const float v = T.b[C1][0][p[C1]] * *ps + T.c[C1][0][p[C1]] * d1;
    *ps = v;
    t1 += v;
  }
  const int s2 = slab_index(g, C2, p[C2]);
  if (s2 >= 0) {
    float* ps = P.p[C][C2] + psi_index(g, C2, p[0], p[1], p[2], s2);
    const float v = T.b[C2][0][p[C2]] * *ps + T.c[C2][0][p[C2]] * d2;
    *ps = v;
    t2 += v;
  }
  const float Sa = g.S * a[q];
  F.f[C][q] += Sa * (t1 - t2);
}

__global__ void k_update_E(Geo g, Fields F, PsiSet P, Tables T, const float* __restrict__ a) {
  int p[3];
  if (!cell_of(g, p)) return;
  const int64_t q = cell_index(g, p[0], p[1], p[2]);
  const int64_t st[3] = {1, g.nxp, g.plane};
  e_update<0>(g, F, P, T, a, p, q, st);
  e_update<1>(g, F, P, T, a, p, q, st);
  e_update<2>(g, F, P, T, a, p, q, st);
}

__device__ __forceinline__ bool box_cell(const int lo[3], const int hi[3], int64_t m, int p[3]) {
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1];
  p[0] = lo[0] + int(m % bx);
  const int64_t r = m / bx;
  p[1] = lo[1] + int(r % by);
  p[2] = lo[2] + int(r / by);
  return p[2] < hi[2];
}

__device__ __forceinline__ int64_t box_count(const int lo[3], const int hi[3]) {
  return (int64_t)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
}

__global__ void k_source(Geo g, Fields F, SrcDev src, int step, float sign, int only_R) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= box_count(src.lo, src.hi)) return;
  int p[3];
  box_cell(src.lo, src.hi, m, p);
  if (only_R && !in_R(g, src.comp, false, p)) return;
  const float v = src.w[m] * src.g[step];
  float* e = F.f[src.comp] + cell_index(g, p[0], p[1], p[2]);
  *e += sign * v;
}

__global__ void k_det_point(Geo g, Fields F, DetDev d, int step, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    out[d.off + step] = (double)F.f[d.comp][cell_index(g, d.lo[0], d.lo[1], d.lo[2])];
}

__global__ void k_det_e2(Geo g, Fields F, DetDev d, double* out) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= box_count(d.lo, d.hi)) return;
  int p[3];
  box_cell(d.lo, d.hi, m, p);
  const int64_t q = cell_index(g, p[0], p[1], p[2]);
  const double ex = F.f[0][q], ey = F.f[1][q], ez = F.f[2][q];
  out[d.off + m] += ex * ex + ey * ey + ez * ez;
}

constexpr int kFluxThreads = 256;

__global__ void __launch_bounds__(kFluxThreads) k_det_flux(Geo g, Fields F, DetDev d, int step, double* partial) {
  __shared__ double sh[kFluxThreads];
  const int64_t M = box_count(d.lo, d.hi);
  const int64_t chunk = (M + gridDim.x - 1) / gridDim.x;
  const int64_t m0 = blockIdx.x * chunk, m1 = min(M, m0 + chunk);
  const int a1 = (d.axis + 1) % 3, a2 = (d.axis + 2) % 3;
  double acc = 0.0;
  for (int64_t m = m0 + threadIdx.x; m < m1; m += blockDim.x) {
    int p[3];
    box_cell(d.lo, d.hi, m, p);
    const int64_t q = cell_index(g, p[0], p[1], p[2]);
    acc += (double)F.f[a1][q] * (double)F.f[3 + a2][q] - (double)F.f[a2][q] * (double)F.f[3 + a1][q];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kFluxThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[d.poff + (int64_t)step * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void k_flux_finalize(DetDev d, int nsteps, const double* partial, double* out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nsteps) return;
  double s = 0.0;
  for (int b = 0; b < d.nblk; ++b) s += partial[d.poff + (int64_t)n * d.nblk + b];
  out[d.off + n] = s;
}

__global__ void k_face_copy(Geo g, Fields F, FaceSet fs, float* rec, int to_record) {
  const FaceSeg& sg = fs.seg[blockIdx.y];
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)sg.n1 * sg.n2) return;
  const int e1 = (sg.axis + 1) % 3, e2 = (sg.axis + 2) % 3;
  int p[3];
  p[sg.axis] = sg.idx;
  p[e1] = sg.lo1 + int(t % sg.n1);
  p[e2] = sg.lo2 + int(t / sg.n1);
  float* h = F.f[3 + sg.comp] + cell_index(g, p[0], p[1], p[2]);
  if (to_record) rec[sg.off + t] = *h;
  else *h = rec[sg.off + t];
}

// ---------------------------------------------------------------------------------------------
// reverse: detector adjoint (the transpose of the sampling at step n)
// ---------------------------------------------------------------------------------------------
__global__ void k_det_adjoint(Geo g, Fields F, Fields A, DetDev d, int step, const double* __restrict__ gy) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (d.kind == 0) {
    if (m != 0) return;
    int p[3] = {d.lo[0], d.lo[1], d.lo[2]};
    if (d.comp < 3 && !e_updated(d.comp, p)) return;
    A.f[d.comp][cell_index(g, p[0], p[1], p[2])] += (float)gy[d.off + step];
    return;
  }
  if (m >= box_count(d.lo, d.hi)) return;
  int p[3];
  box_cell(d.lo, d.hi, m, p);
  const int64_t q = cell_index(g, p[0], p[1], p[2]);
  if (d.kind == 1) {
    const double w = 2.0 * gy[d.off + m];
    for (int c = 0; c < 3; ++c)
      if (e_updated(c, p)) A.f[c][q] += (float)(w * (double)F.f[c][q]);
  } else {
    const int a1 = (d.axis + 1) % 3, a2 = (d.axis + 2) % 3;
    const double gn = gy[d.off + step];
    if (e_updated(a1, p)) A.f[a1][q] += (float)(gn * (double)F.f[3 + a2][q]);
    if (e_updated(a2, p)) A.f[a2][q] -= (float)(gn * (double)F.f[3 + a1][q]);
    A.f[3 + a2][q] += (float)(gn * (double)F.f[a1][q]);
    A.f[3 + a1][q] -= (float)(gn * (double)F.f[a2][q]);
  }
}

// ---------------------------------------------------------------------------------------------
// reverse: E part. Transpose of the E update (gather into H-bar), the inverse E update on R, and
// dL/da on the design box.
// ---------------------------------------------------------------------------------------------
struct PQ {
  float c1, c2;  // coefficients on the difference along C1 and along C2
};

// Adjoint coefficients of the E_C update at cell p (zero outside the grid or where E_C is held).
template <int C>
__device__ __forceinline__ PQ e_coef(const Geo& g, const Fields& A, const PsiSet& Pold, const Tables& T,
                                     const float* a, const int p[3]) {
  constexpr int C1 = (C + 1) % 3, C2 = (C + 2) % 3;
  PQ r = {0.f, 0.f};
  if (p[0] >= g.n[0] || p[1] >= g.n[1] || p[2] >= g.n[2] || !e_updated(C, p)) return r;
  const int64_t q = cell_index(g, p[0], p[1], p[2]);
  const float u = (g.S * a[q]) * A.f[C][q];
  r.c1 = u * T.ik[C1][0][p[C1]];
  r.c2 = -u * T.ik[C2][0][p[C2]];
  const int s1 = slab_index(g, C1, p[C1]);
  if (s1 >= 0) r.c1 += T.c[C1][0][p[C1]] * (Pold.p[C][C1][psi_index(g, C1, p[0], p[1], p[2], s1)] + u);
  const int s2 = slab_index(g, C2, p[C2]);
  if (s2 >= 0) r.c2 += T.c[C2][0][p[C2]] * (Pold.p[C][C2][psi_index(g, C2, p[0], p[1], p[2], s2)] - u);
  return r;
}

template <int C>
__device__ __forceinline__ void e_psi_adjoint(const Geo& g, const Fields& A, const PsiSet& Pold, const PsiSet& Pnew,
                                              const Tables& T, const float* a, const int p[3], int64_t q) {
  constexpr int C1 = (C + 1) % 3, C2 = (C + 2) % 3;
  const int s1 = slab_index(g, C1, p[C1]);
  const int s2 = slab_index(g, C2, p[C2]);
  if (s1 < 0 && s2 < 0) return;
  const float u = e_updated(C, p) ? (g.S * a[q]) * A.f[C][q] : 0.f;
  if (s1 >= 0) {
    const int64_t z = psi_index(g, C1, p[0], p[1], p[2], s1);
    Pnew.p[C][C1][z] = T.b[C1][0][p[C1]] * (Pold.p[C][C1][z] + u);
  }
  if (s2 >= 0) {
    const int64_t z = psi_index(g, C2, p[0], p[1], p[2], s2);
    Pnew.p[C][C2][z] = T.b[C2][0][p[C2]] * (Pold.p[C][C2][z] - u);
  }
}

// curl of H at E_C (plain differences; kappa and psi applied by the caller)
template <int C>
__device__ __forceinline__ void e_diffs(const Fields& F, int64_t q, const int64_t st[3], float& d1, float& d2) {
  constexpr int C1 = (C + 1) % 3, C2 = (C + 2) % 3;
  d1 = F.f[3 + C2][q] - F.f[3 + C2][q - st[C1]];
  d2 = F.f[3 + C1][q] - F.f[3 + C1][q - st[C2]];
}

__global__ void k_rev_E(Geo g, Fields F, Fields A, PsiSet Pold, PsiSet Pnew, Tables T, const float* __restrict__ a,
                        int dlo0, int dlo1, int dlo2, int dhi0, int dhi1, int dhi2, double* dLda) {
  int p[3];
  if (!cell_of(g, p)) return;
  const int64_t q = cell_index(g, p[0], p[1], p[2]);
  const int64_t st[3] = {1, g.nxp, g.plane};

  // (1) dL/da and the inverse E update (reads H^{n+1/2}, which this kernel does not write)
  const bool design = p[0] >= dlo0 && p[0] < dhi0 && p[1] >= dlo1 && p[1] < dhi1 && p[2] >= dlo2 && p[2] < dhi2;
  const float Sa = g.S * a[q];
  float gsum = 0.f;
#pragma unroll
  for (int C = 0; C < 3; ++C) {
    if (!e_updated(C, p)) continue;
    const bool r = in_R(g, C, false, p);
    if (!design && !r) continue;
    float d1, d2;
    if (C == 0) e_diffs<0>(F, q, st, d1, d2);
    else if (C == 1) e_diffs<1>(F, q, st, d1, d2);
    else e_diffs<2>(F, q, st, d1, d2);
    const int C1 = (C + 1) % 3, C2 = (C + 2) % 3;
    if (design) gsum += A.f[C][q] * (d1 - d2);  // kappa = 1 and psi = 0 inside R
    if (r) F.f[C][q] -= Sa * (d1 * T.ik[C1][0][p[C1]] - d2 * T.ik[C2][0][p[C2]]);
  }
  if (design) {
    const int64_t m = ((int64_t)(p[2] - dlo2) * (dhi1 - dlo1) + (p[1] - dlo1)) * (dhi0 - dlo0) + (p[0] - dlo0);
    dLda[m] += (double)g.S * (double)gsum;
  }

  // (2) H-bar += transpose of the E update: gather the coefficients of neighbouring E points
  int px[3] = {p[0] + 1, p[1], p[2]};
  int py[3] = {p[0], p[1] + 1, p[2]};
  int pz[3] = {p[0], p[1], p[2] + 1};
  const PQ ex0 = e_coef<0>(g, A, Pold, T, a, p), ey0 = e_coef<1>(g, A, Pold, T, a, p), ez0 = e_coef<2>(g, A, Pold, T, a, p);
  const PQ ex_y = e_coef<0>(g, A, Pold, T, a, py);
  const PQ ey_x = e_coef<1>(g, A, Pold, T, a, px), ey_z = e_coef<1>(g, A, Pold, T, a, pz);
  const PQ ez_x = e_coef<2>(g, A, Pold, T, a, px), ez_y = e_coef<2>(g, A, Pold, T, a, py);
  const PQ ex_z = e_coef<0>(g, A, Pold, T, a, pz);
  // Hx enters E_y (diff along z, coefficient c1) and E_z (diff along y, coefficient c2)
  A.f[3][q] += (ey0.c1 - ey_z.c1) + (ez0.c2 - ez_y.c2);
  // Hy enters E_z (along x, c1) and E_x (along z, c2)
  A.f[4][q] += (ez0.c1 - ez_x.c1) + (ex0.c2 - ex_z.c2);
  // Hz enters E_x (along y, c1) and E_y (along x, c2)
  A.f[5][q] += (ex0.c1 - ex_y.c1) + (ey0.c2 - ey_x.c2);

  // (3) psi-bar of E at this cell, into the other buffer
  e_psi_adjoint<0>(g, A, Pold, Pnew, T, a, p, q);
  e_psi_adjoint<1>(g, A, Pold, Pnew, T, a, p, q);
  e_psi_adjoint<2>(g, A, Pold, Pnew, T, a, p, q);
}

// ---------------------------------------------------------------------------------------------
// reverse: H part. Inverse H update on R and the transpose of the H update (gather into E-bar).
// ---------------------------------------------------------------------------------------------
template <int C>
__device__ __forceinline__ PQ h_coef(const Geo& g, const Fields& A, const PsiSet& Pold, const Tables& T,
                                     const int p[3]) {
  constexpr int C1 = (C + 1) % 3, C2 = (C + 2) % 3;
  PQ r = {0.f, 0.f};
  if (p[0] < 0 || p[1] < 0 || p[2] < 0) return r;
  const int64_t q = cell_index(g, p[0], p[1], p[2]);
  const float w = -g.S * A.f[3 + C][q];
  r.c1 = w * T.ik[C1][1][p[C1]];
  r.c2 = -w * T.ik[C2][1][p[C2]];
  const int s1 = slab_index(g, C1, p[C1]);
  if (s1 >= 0) r.c1 += T.c[C1][1][p[C1]] * (Pold.p[C][C1][psi_index(g, C1, p[0], p[1], p[2], s1)] + w);
  const int s2 = slab_index(g, C2, p[C2]);
  if (s2 >= 0) r.c2 += T.c[C2][1][p[C2]] * (Pold.p[C][C2][psi_index(g, C2, p[0], p[1], p[2], s2)] - w);
  return r;
}

template <int C>
__device__ __forceinline__ void h_psi_adjoint(const Geo& g, const Fields& A, const PsiSet& Pold, const PsiSet& Pnew,
                                              const Tables& T, const int p[3], int64_t q) {
  constexpr int C1 = (C + 1) % 3, C2 = (C + 2) % 3;
  const int s1 = slab_index(g, C1, p[C1]);
  const int s2 = slab_index(g, C2, p[C2]);
  if (s1 < 0 && s2 < 0) return;
  const float w = -g.S * A.f[3 + C][q];
  if (s1 >= 0) {
    const int64_t z = psi_index(g, C1, p[0], p[1], p[2], s1);
    Pnew.p[C][C1][z] = T.b[C1][1][p[C1]] * (Pold.p[C][C1][z] + w);
  }
  if (s2 >= 0) {
    const int64_t z = psi_index(g, C2, p[0], p[1], p[2], s2);
    Pnew.p[C][C2][z] = T.b[C2][1][p[C2]] * (Pold.p[C][C2][z] - w);
  }
}

template <int C>
__device__ __forceinline__ void h_inverse(const Geo& g, const Fields& F, const Tables& T, const int p[3], int64_t q,
                                          const int64_t st[3]) {
  constexpr int C1 = (C + 1) % 3, C2 = (C + 2) % 3;
  if (!in_R(g, C, true, p)) return;
  const float* Ea = F.f[C2];
  const float* Eb = F.f[C1];
  const float ea1 = (p[C1] + 1 < g.n[C1]) ? Ea[q + st[C1]] : 0.f;
  const float eb2 = (p[C2] + 1 < g.n[C2]) ? Eb[q + st[C2]] : 0.f;
  const float d1 = ea1 - Ea[q];
  const float d2 = eb2 - Eb[q];
  F.f[3 + C][q] += g.S * (d1 * T.ik[C1][1][p[C1]] - d2 * T.ik[C2][1][p[C2]]);
}

__global__ void k_rev_H(Geo g, Fields F, Fields A, PsiSet Pold, PsiSet Pnew, Tables T) {
  int p[3];
  if (!cell_of(g, p)) return;
  const int64_t q = cell_index(g, p[0], p[1], p[2]);
  const int64_t st[3] = {1, g.nxp, g.plane};

  // (1) inverse H update on R (reads E^n, which this kernel does not write)
  h_inverse<0>(g, F, T, p, q, st);
  h_inverse<1>(g, F, T, p, q, st);
  h_inverse<2>(g, F, T, p, q, st);

  // (2) E-bar += transpose of the H update
  int mx[3] = {p[0] - 1, p[1], p[2]};
  int my[3] = {p[0], p[1] - 1, p[2]};
  int mz[3] = {p[0], p[1], p[2] - 1};
  const PQ hx0 = h_coef<0>(g, A, Pold, T, p), hy0 = h_coef<1>(g, A, Pold, T, p), hz0 = h_coef<2>(g, A, Pold, T, p);
  // Ex enters Hy (diff along z, c1) and Hz (diff along y, c2)
  if (e_updated(0, p)) {
    const PQ hy_z = h_coef<1>(g, A, Pold, T, mz), hz_y = h_coef<2>(g, A, Pold, T, my);
    A.f[0][q] += (hy_z.c1 - hy0.c1) + (hz_y.c2 - hz0.c2);
  }
  // Ey enters Hz (along x, c1) and Hx (along z, c2)
  if (e_updated(1, p)) {
    const PQ hz_x = h_coef<2>(g, A, Pold, T, mx), hx_z = h_coef<0>(g, A, Pold, T, mz);
    A.f[1][q] += (hz_x.c1 - hz0.c1) + (hx_z.c2 - hx0.c2);
  }
  // Ez enters Hx (along y, c1) and Hy (along x, c2)
  if (e_updated(2, p)) {
    const PQ hx_y = h_coef<0>(g, A, Pold, T, my), hy_x = h_coef<1>(g, A, Pold, T, mx);
    A.f[2][q] += (hx_y.c1 - hx0.c1) + (hy_x.c2 - hy0.c2);
  }

  // (3) psi-bar of H at this cell
  h_psi_adjoint<0>(g, A, Pold, Pnew, T, p, q);
  h_psi_adjoint<1>(g, A, Pold, Pnew, T, p, q);
  h_psi_adjoint<2>(g, A, Pold, Pnew, T, p, q);
}

__global__ void k_set_density(Geo g, float* a, int lo0, int lo1, int lo2, int hi0, int hi1, int hi2,
                              const float* rho, float eps_lo, float deps) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int bx = hi0 - lo0, by = hi1 - lo1;
  if (m >= (int64_t)bx * by * (hi2 - lo2)) return;
  const int i = lo0 + int(m % bx), j = lo1 + int((m / bx) % by), k = lo2 + int(m / ((int64_t)bx * by));
  const float eps = eps_lo + deps * rho[m];          // float, as the scene inputs are built
  a[cell_index(g, i, j, k)] = (float)(1.0 / (double)eps);
}

__global__ void k_grad_finalize(Geo g, const float* __restrict__ a, int dlo0, int dlo1, int dlo2, int dhi0,
                                int dhi1, int dhi2, const double* dLda, float* out, double scale) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int bx = dhi0 - dlo0, by = dhi1 - dlo1;
  const int64_t M = (int64_t)bx * by * (dhi2 - dlo2);
  if (m >= M) return;
  const int i = dlo0 + int(m % bx), j = dlo1 + int((m / bx) % by), k = dlo2 + int(m / ((int64_t)bx * by));
  const double av = a[cell_index(g, i, j, k)];
  out[m] = (float)(-av * av * dLda[m] * scale);  // a = 1/eps, da/deps = -a^2; scale = deps/drho or 1
}

__global__ void k_pack(Geo g, Fields F, float* out6, int unpack) {
  int p[3];
  if (!cell_of(g, p)) return;
  const int64_t q = cell_index(g, p[0], p[1], p[2]);
  const int64_t N = (int64_t)g.n[0] * g.n[1] * g.n[2];
  const int64_t u = ((int64_t)p[2] * g.n[1] + p[1]) * g.n[0] + p[0];
  for (int f = 0; f < 6; ++f) {
    if (unpack) F.f[f][q] = out6[f * N + u];
    else out6[f * N + u] = F.f[f][q];
  }
}

__global__ void k_set_box(Geo g, float* a, int lo0, int lo1, int lo2, int hi0, int hi1, int hi2, const float* box) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int bx = hi0 - lo0, by = hi1 - lo1;
  if (m >= (int64_t)bx * by * (hi2 - lo2)) return;
  const int i = lo0 + int(m % bx), j = lo1 + int((m / bx) % by), k = lo2 + int(m / ((int64_t)bx * by));
  a[cell_index(g, i, j, k)] = box[m];
}

dim3 cell_grid(const Geo& g) { return dim3((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY, g.n[2]); }

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_update_H(const Geo& g, const Fields& F, const PsiSet& psiH, const Tables& T, cudaStream_t s) {
  k_update_H<<<cell_grid(g), dim3(BX, BY), 0, s>>>(g, F, psiH, T);
}

void launch_update_E(const Geo& g, const Fields& F, const PsiSet& psiE, const Tables& T, const float* a,
                     cudaStream_t s) {
  k_update_E<<<cell_grid(g), dim3(BX, BY), 0, s>>>(g, F, psiE, T, a);
}

void launch_source(const Geo& g, const Fields& F, const SrcDev& src, int step, float sign, int only_R,
                   cudaStream_t s) {
  const int64_t n = (int64_t)(src.hi[0] - src.lo[0]) * (src.hi[1] - src.lo[1]) * (src.hi[2] - src.lo[2]);
  if (n <= 0) return;
  k_source<<<blocks_for(n, 256), 256, 0, s>>>(g, F, src, step, sign, only_R);
}

void launch_detector_sample(const Geo& g, const Fields& F, const DetDev& d, int step, double* out,
                            double* partial, cudaStream_t s) {
  const int64_t n = (int64_t)(d.hi[0] - d.lo[0]) * (d.hi[1] - d.lo[1]) * (d.hi[2] - d.lo[2]);
  if (d.kind == 0) k_det_point<<<1, 32, 0, s>>>(g, F, d, step, out);
  else if (d.kind == 1) k_det_e2<<<blocks_for(n, 256), 256, 0, s>>>(g, F, d, out);
  else k_det_flux<<<d.nblk, kFluxThreads, 0, s>>>(g, F, d, step, partial);
}

void launch_flux_finalize(const DetDev& d, int nsteps, const double* partial, double* out, cudaStream_t s) {
  if (nsteps <= 0) return;
  k_flux_finalize<<<blocks_for(nsteps, 128), 128, 0, s>>>(d, nsteps, partial, out);
}

void launch_face_copy(const Geo& g, const Fields& F, const FaceSet& fs, float* rec, int to_record,
                      cudaStream_t s) {
  if (fs.nseg == 0) return;
  int64_t mx = 0;
  for (int i = 0; i < fs.nseg; ++i) mx = mx > (int64_t)fs.seg[i].n1 * fs.seg[i].n2 ? mx : (int64_t)fs.seg[i].n1 * fs.seg[i].n2;
  k_face_copy<<<dim3(blocks_for(mx, 256), fs.nseg), 256, 0, s>>>(g, F, fs, rec, to_record);
}

void launch_detector_adjoint(const Geo& g, const Fields& F, const Fields& A, const DetDev& d, int step,
                             const double* dL_ddet, cudaStream_t s) {
  const int64_t n = d.kind == 0 ? 1 : (int64_t)(d.hi[0] - d.lo[0]) * (d.hi[1] - d.lo[1]) * (d.hi[2] - d.lo[2]);
  k_det_adjoint<<<blocks_for(n, 256), 256, 0, s>>>(g, F, A, d, step, dL_ddet);
}

void launch_rev_E(const Geo& g, const Fields& F, const Fields& A, const PsiSet& psiE_old, const PsiSet& psiE_new,
                  const Tables& T, const float* a, const int* dlo, const int* dhi, double* dLda, cudaStream_t s) {
  k_rev_E<<<cell_grid(g), dim3(BX, BY), 0, s>>>(g, F, A, psiE_old, psiE_new, T, a, dlo[0], dlo[1], dlo[2], dhi[0],
                                                dhi[1], dhi[2], dLda);
}

void launch_rev_H(const Geo& g, const Fields& F, const Fields& A, const PsiSet& psiH_old, const PsiSet& psiH_new,
                  const Tables& T, cudaStream_t s) {
  k_rev_H<<<cell_grid(g), dim3(BX, BY), 0, s>>>(g, F, A, psiH_old, psiH_new, T);
}

void launch_grad_finalize(const Geo& g, const float* a, const int* dlo, const int* dhi, const double* dLda,
                          float* dL_deps, double scale, cudaStream_t s) {
  const int64_t n = (int64_t)(dhi[0] - dlo[0]) * (dhi[1] - dlo[1]) * (dhi[2] - dlo[2]);
  if (n <= 0) return;
  k_grad_finalize<<<blocks_for(n, 256), 256, 0, s>>>(g, a, dlo[0], dlo[1], dlo[2], dhi[0], dhi[1], dhi[2], dLda,
                                                     dL_deps, scale);
}

void launch_set_density(const Geo& g, float* a, const int* lo, const int* hi, const float* rho, float eps_lo,
                        float deps, cudaStream_t s) {
  const int64_t n = (int64_t)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  if (n <= 0) return;
  k_set_density<<<blocks_for(n, 256), 256, 0, s>>>(g, a, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2], rho, eps_lo, deps);
}

void launch_pack_fields(const Geo& g, const Fields& F, float* out6, int unpack, cudaStream_t s) {
  k_pack<<<cell_grid(g), dim3(BX, BY), 0, s>>>(g, F, out6, unpack);
}

void launch_set_box(const Geo& g, float* a, const int* lo, const int* hi, const float* box, cudaStream_t s) {
  const int64_t n = (int64_t)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  if (n <= 0) return;
  k_set_box<<<blocks_for(n, 256), 256, 0, s>>>(g, a, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2], box);
}

}  // namespace fdtd
