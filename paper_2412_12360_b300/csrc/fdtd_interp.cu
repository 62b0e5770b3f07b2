// Interpolated detectors (arXiv 2412.12360 Sec. 2.1: composite metrics such as energy and Poynting
// flux need the staggered Yee components brought to one point in space and time; the paper's
// evaluation mode) and their adjoints.
//
// Every component is taken at the cell centre (i+1/2, j+1/2, k+1/2): E_c as the mean of its 4 values
// around the centre (offsets 0/1 along the two axes other than c), H_c as the mean of its 2 values
// (offsets 0/1 along c); values beyond the grid are 0 (the detector box plus one cell lies in the
// grid). Kind 3 sums |E^{n+1}(centre)|^2 per cell over the steps; kind 4 is the per-step flux
// sum over the box of (E^{n+1/2} x H^{n+1/2})[axis] at the centres, E^{n+1/2} = (E^n + E^{n+1}) / 2.
//
// Adjoints, in gather form (one thread per field point of the box extended by one cell, summing the
// cells whose stencil holds the point, so no atomics and a fixed order). With G = dL/dF_n and the
// flux axes a1 = axis+1, a2 = axis+2 (F = e1 h2 - e2 h1 per cell):
//   dF/dE^{n+1}_{a1} and dF/dE^n_{a1}: 1/8 G h2 per stencil point, dF/dE_{a2}: -1/8 G h1;
//   dF/dH_{a2}: 1/2 G e1, dF/dH_{a1}: -1/2 G e2;
//   kind 3: dL/dE^{n+1}_c: 1/4 * 2 g_cell e_c(cell) per stencil point.
// The reverse sweep holds dL/d(E^{n+1}, H^{n+1/2}) before its step-n kernels and dL/d(E^n, H^{n-1/2})
// after them, so the E^{n+1} terms go in before rev_E, the H terms between rev_E and rev_H (E^n is
// rebuilt by then), and the E^n terms after rev_H; the H^{n+1/2} and E^{n+1} values those later terms
// need are copied into small slabs at the start of the step, before the inverse step overwrites them.
#include "../../include/fdtd.h"
#include "fdtd_internal.cuh"

namespace fdtd {

namespace {

__device__ __forceinline__ float val0(const Geo& g, const float* f, int x, int y, int z) {
  return (x < g.n[0] && y < g.n[1] && z < g.n[2]) ? f[cell_index(g, x, y, z)] : 0.f;
}

// slab of the box extended by one cell: [lo, hi + 1) per axis, x fastest, 3 components
struct Slab {
  int lo[3], n[3];
  __host__ __device__ int64_t count() const { return (int64_t)n[0] * n[1] * n[2]; }
};

__host__ __device__ inline Slab slab_of(const DetDev& d) {
  Slab s;
  for (int k = 0; k < 3; ++k) {
    s.lo[k] = d.lo[k];
    s.n[k] = d.hi[k] - d.lo[k] + 1;
  }
  return s;
}

__device__ __forceinline__ float sval(const Slab& s, const float* v, int c, int x, int y, int z) {
  return v[c * s.count() + ((int64_t)(z - s.lo[2]) * s.n[1] + (y - s.lo[1])) * s.n[0] + (x - s.lo[0])];
}

// cell-centre E_c / H_c of cell p from a slab
__device__ __forceinline__ float e_ctr(const Slab& s, const float* v, int c, const int p[3]) {
  float t = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int q[3] = {p[0], p[1], p[2]};
      q[(c + 1) % 3] += a;
      q[(c + 2) % 3] += b;
      t += sval(s, v, c, q[0], q[1], q[2]);
    }
  return 0.25f * t;
}
__device__ __forceinline__ float h_ctr(const Slab& s, const float* v, int c, const int p[3]) {
  int q[3] = {p[0], p[1], p[2]};
  q[c] += 1;
  return 0.5f * (sval(s, v, c, p[0], p[1], p[2]) + sval(s, v, c, q[0], q[1], q[2]));
}
// the same from the fields
__device__ __forceinline__ double e_ctr_f(const Geo& g, const float* E, int c, const int p[3]) {
  double t = 0.0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int q[3] = {p[0], p[1], p[2]};
      q[(c + 1) % 3] += a;
      q[(c + 2) % 3] += b;
      t += val0(g, E, q[0], q[1], q[2]);
    }
  return 0.25 * t;
}
__device__ __forceinline__ double h_ctr_f(const Geo& g, const float* H, int c, const int p[3]) {
  int q[3] = {p[0], p[1], p[2]};
  q[c] += 1;
  return 0.5 * ((double)H[cell_index(g, p[0], p[1], p[2])] + (double)val0(g, H, q[0], q[1], q[2]));
}

// cell m of the box [lo, hi), x fastest
__device__ __forceinline__ void box_point(const DetDev& d, int64_t m, int p[3]) {
  const int bx = d.hi[0] - d.lo[0], by = d.hi[1] - d.lo[1];
  p[0] = d.lo[0] + int(m % bx);
  p[1] = d.lo[1] + int((m / bx) % by);
  p[2] = d.lo[2] + int(m / ((int64_t)bx * by));
}

__device__ __forceinline__ bool in_box(const DetDev& d, const int p[3]) {
  return p[0] >= d.lo[0] && p[0] < d.hi[0] && p[1] >= d.lo[1] && p[1] < d.hi[1] && p[2] >= d.lo[2] && p[2] < d.hi[2];
}

__device__ __forceinline__ void slab_point(const Slab& s, int64_t m, int q[3]) {
  q[0] = s.lo[0] + int(m % s.n[0]);
  q[1] = s.lo[1] + int((m / s.n[0]) % s.n[1]);
  q[2] = s.lo[2] + int(m / ((int64_t)s.n[0] * s.n[1]));
}

// ---- forward sampling -----------------------------------------------------------------------------
__global__ void k_det_e2_interp(Geo g, Fields F, DetDev d, double* out) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= (int64_t)(d.hi[0] - d.lo[0]) * (d.hi[1] - d.lo[1]) * (d.hi[2] - d.lo[2])) return;
  int p[3];
  box_point(d, m, p);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double e = e_ctr_f(g, F.f[c], c, p);
    s += e * e;
  }
  out[d.off + m] += s;
}

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_det_flux_interp(Geo g, Fields P, Fields F, DetDev d, int step,
                                                              double* partial) {
  __shared__ double sh[kThreads];
  const int64_t M = (int64_t)(d.hi[0] - d.lo[0]) * (d.hi[1] - d.lo[1]) * (d.hi[2] - d.lo[2]);
  const int64_t chunk = (M + gridDim.x - 1) / gridDim.x;
  const int64_t m0 = blockIdx.x * chunk, m1 = min(M, m0 + chunk);
  const int a1 = (d.axis + 1) % 3, a2 = (d.axis + 2) % 3;
  double acc = 0.0;
  for (int64_t m = m0 + threadIdx.x; m < m1; m += blockDim.x) {
    int p[3];
    box_point(d, m, p);
    const double e1 = 0.5 * (e_ctr_f(g, P.f[a1], a1, p) + e_ctr_f(g, F.f[a1], a1, p));
    const double e2 = 0.5 * (e_ctr_f(g, P.f[a2], a2, p) + e_ctr_f(g, F.f[a2], a2, p));
    acc += e1 * h_ctr_f(g, F.f[3 + a2], a2, p) - e2 * h_ctr_f(g, F.f[3 + a1], a1, p);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[d.poff + (int64_t)step * gridDim.x + blockIdx.x] = sh[0];
}

// ---- reverse ---------------------------------------------------------------------------------------
// copy E (comp0 = 0) or H (comp0 = 3) on the extended box into a slab
__global__ void k_slab_copy(Geo g, Fields F, DetDev d, int comp0, float* out) {
  const Slab s = slab_of(d);
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= s.count()) return;
  int q[3];
  slab_point(s, m, q);
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c * s.count() + m] = val0(g, F.f[comp0 + c], q[0], q[1], q[2]);
}

// kind 3: E-bar += dL/dE^{n+1} (E^{n+1} read from the fields)
__global__ void k_adj_e2_interp(Geo g, Fields F, Fields A, DetDev d, const double* __restrict__ gy) {
  const Slab s = slab_of(d);
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= s.count()) return;
  int q[3];
  slab_point(s, m, q);
  const int bx = d.hi[0] - d.lo[0], by = d.hi[1] - d.lo[1];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        int p[3] = {q[0], q[1], q[2]};
        p[(c + 1) % 3] -= a;
        p[(c + 2) % 3] -= b;
        if (!in_box(d, p)) continue;
        const int64_t cell = ((int64_t)(p[2] - d.lo[2]) * by + (p[1] - d.lo[1])) * bx + (p[0] - d.lo[0]);
        acc += 0.25 * 2.0 * gy[d.off + cell] * e_ctr_f(g, F.f[c], c, p);
      }
    A.f[c][cell_index(g, q[0], q[1], q[2])] += (float)acc;
  }
}

// kind 4, E terms (of E^{n+1} before rev_E, of E^n after rev_H): E-bar_{a1} += 1/8 G h2, E-bar_{a2} -= 1/8 G h1
__global__ void k_adj_flux_interp_E(Geo g, Fields A, DetDev d, int step, const double* __restrict__ gy,
                                    const float* __restrict__ slabH) {
  const Slab s = slab_of(d);
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= s.count()) return;
  int q[3];
  slab_point(s, m, q);
  const double G = gy[d.off + step];
  const int a1 = (d.axis + 1) % 3, a2 = (d.axis + 2) % 3;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int c = t == 0 ? a1 : a2;  // the E component, paired with H_{a2} (+) or H_{a1} (-)
    const int hc = t == 0 ? a2 : a1;
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        int p[3] = {q[0], q[1], q[2]};
        p[(c + 1) % 3] -= a;
        p[(c + 2) % 3] -= b;
        if (!in_box(d, p)) continue;
        acc += 0.125 * G * h_ctr(s, slabH, hc, p);
      }
    A.f[c][cell_index(g, q[0], q[1], q[2])] += (float)(t == 0 ? acc : -acc);
  }
}

// kind 4, H terms (between rev_E and rev_H): H-bar_{a2} += 1/2 G e1, H-bar_{a1} -= 1/2 G e2, with
// e = (E^n + E^{n+1}) / 2 at the centres
__global__ void k_adj_flux_interp_H(Geo g, Fields A, DetDev d, int step, const double* __restrict__ gy,
                                    const float* __restrict__ slabE0, const float* __restrict__ slabE1) {
  const Slab s = slab_of(d);
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= s.count()) return;
  int q[3];
  slab_point(s, m, q);
  const double G = gy[d.off + step];
  const int a1 = (d.axis + 1) % 3, a2 = (d.axis + 2) % 3;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int hc = t == 0 ? a2 : a1;  // the H component, paired with e_{a1} (+) or e_{a2} (-)
    const int ec = t == 0 ? a1 : a2;
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      int p[3] = {q[0], q[1], q[2]};
      p[hc] -= a;
      if (!in_box(d, p)) continue;
      acc += 0.5 * G * 0.5 * ((double)e_ctr(s, slabE0, ec, p) + (double)e_ctr(s, slabE1, ec, p));
    }
    A.f[3 + hc][cell_index(g, q[0], q[1], q[2])] += (float)(t == 0 ? acc : -acc);
  }
}

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int64_t interp_slab_floats(const DetDev& d) { return 3 * slab_of(d).count(); }

void launch_detector_interp(const Geo& g, const Fields& P, const Fields& F, const DetDev& d, int step, double* out,
                            double* partial, cudaStream_t s) {
  const int64_t n = (int64_t)(d.hi[0] - d.lo[0]) * (d.hi[1] - d.lo[1]) * (d.hi[2] - d.lo[2]);
  if (n <= 0) return;
  if (d.kind == 3) k_det_e2_interp<<<blocks(n, 256), 256, 0, s>>>(g, F, d, out);
  else k_det_flux_interp<<<d.nblk, kThreads, 0, s>>>(g, P, F, d, step, partial);
}

void launch_slab_copy(const Geo& g, const Fields& F, const DetDev& d, int comp0, float* out, cudaStream_t s) {
  k_slab_copy<<<blocks(slab_of(d).count(), 256), 256, 0, s>>>(g, F, d, comp0, out);
}

void launch_interp_adjoint(const Geo& g, const Fields& F, const Fields& A, const DetDev& d, int step,
                           const double* dL_ddet, int part, const float* slabE0, const float* slabE1,
                           const float* slabH, cudaStream_t s) {
  const unsigned nb = blocks(slab_of(d).count(), 256);
  if (d.kind == 3) {
    if (part == 0) k_adj_e2_interp<<<nb, 256, 0, s>>>(g, F, A, d, dL_ddet);
    return;
  }
  if (part == 0 || part == 2) k_adj_flux_interp_E<<<nb, 256, 0, s>>>(g, A, d, step, dL_ddet, slabH);
  else k_adj_flux_interp_H<<<nb, 256, 0, s>>>(g, A, d, step, dL_ddet, slabE0, slabE1);
}

}  // namespace fdtd
