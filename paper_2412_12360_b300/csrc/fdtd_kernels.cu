// Auxiliary per-cell kernels of libfdtd (one thread per cell or per box element): sources and
// detectors beyond the fused kernels' slots, the fixed-order flux sums, the detector adjoints of the
// reverse sweep (the transpose of each sampling, Sec. 2.2 of arXiv 2412.12360), the density map
// eps = eps_lo + (eps_hi - eps_lo) rho, the dL/deps finalisation and field packing.
#include <algorithm>

#include <cmath>

#include "fdtd_internal.cuh"
#include "fdtd_tma.cuh"

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

__device__ __forceinline__ bool box_cell(const int lo[3], const int hi[3], int64_t m64, int p[3]) {
  // 32-bit arithmetic: a box holds fewer than 2^31 cells (it lies inside a grid that does)
  const int m = (int)m64;
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1];
  p[0] = lo[0] + m % bx;
  const int r = m / bx;
  p[1] = lo[1] + r % by;
  p[2] = lo[2] + r / by;
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
  if (only_R && !in_R(g, src.comp % 3, src.comp >= 3, p)) return;  // comp 3..5: an H component
  const float v = src.w[m] * src.g[step];
  float* e = F.f[src.comp] + cell_index(g, p[0], p[1], p[2]);
  *e += sign * v;
}

// Multiply a source's box weights by a = 1/eps of each cell (the E correction of a TFSF plane).
__global__ void k_source_scale_a(Geo g, const float* __restrict__ a, SrcDev src) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= box_count(src.lo, src.hi)) return;
  int p[3];
  box_cell(src.lo, src.hi, m, p);
  const_cast<float*>(src.w)[m] *= a[cell_index(g, p[0], p[1], p[2])];
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

// Boundary-face record of one step (Sec. 2.2): the tangential H on the planes just outside the PML-free
// region, segment by segment. Within a segment the elements run along x where the segment spans x
// (y- and z-faces), else along y, so that the field side of the copy is coalesced wherever it can be.
__global__ void k_face_copy(Geo g, Fields F, FaceSet fs, float* __restrict__ rec, int to_record) {
  pdl_wait();
  const FaceSeg& sg = fs.seg[blockIdx.y];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // a face segment holds fewer than 2^31 cells
  if (t >= sg.n1 * sg.n2) return;
  const int nf = sg.axis == 1 ? sg.n2 : sg.n1;  // extent along the fast axis
  const int f = t % nf, sl = t / nf;
  int x, y, z;
  if (sg.axis == 0) { x = sg.idx; y = sg.lo1 + f; z = sg.lo2 + sl; }
  else if (sg.axis == 1) { y = sg.idx; x = sg.lo2 + f; z = sg.lo1 + sl; }
  else { z = sg.idx; x = sg.lo1 + f; y = sg.lo2 + sl; }
  float* h = F.f[3 + sg.comp] + cell_index(g, x, y, z);
  if (to_record) rec[sg.off + t] = *h;
  else *h = rec[sg.off + t];
}

// the face copies of several requests: blockIdx.z the request, blockIdx.y the segment
__global__ void k_face_copy_group(const __grid_constant__ FaceGroup G) {
  pdl_wait();
  const FaceJob& J = G.e[blockIdx.z];
  if ((int)blockIdx.y >= J.fs.nseg) return;
  const FaceSeg& sg = J.fs.seg[blockIdx.y];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= sg.n1 * sg.n2) return;
  const int nf = sg.axis == 1 ? sg.n2 : sg.n1;
  const int f = t % nf, sl = t / nf;
  int x, y, z;
  if (sg.axis == 0) { x = sg.idx; y = sg.lo1 + f; z = sg.lo2 + sl; }
  else if (sg.axis == 1) { y = sg.idx; x = sg.lo2 + f; z = sg.lo1 + sl; }
  else { z = sg.idx; x = sg.lo1 + f; y = sg.lo2 + sl; }
  float* h = J.F.f[3 + sg.comp] + cell_index(J.g, x, y, z);
  if (G.to_record) J.rec[sg.off + t] = *h;
  else *h = J.rec[sg.off + t];
}

// ---------------------------------------------------------------------------------------------
// reverse: detector adjoint (the transpose of the sampling at step n)
// ---------------------------------------------------------------------------------------------
__global__ void k_det_adjoint(Geo g, Fields F, Fields A, DetDev d, int step, const double* __restrict__ gy) {
  pdl_wait();
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
// non-finite check of the grid cells of nrows rows of nxp floats (the first nx of them cells, the
// rest pitch padding): a value is NaN or infinite exactly when its exponent bits are all ones, a test
// on the bits (integer work, so the kernel runs at memory speed; the FP64 units of this part are far
// too few for a per-value FP64 sum). A warp walks a row in float4 steps (nxp is a multiple of 32 and
// p 16-byte aligned: whole field arrays of pitch-padded planes).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned nonfinite_bit(float v) {
  return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u ? 1u : 0u;
}

__global__ void k_check_finite(const float4* __restrict__ p, int64_t nrows, int nx, int nxp, int* status) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int row4 = nxp / 4, nx4 = (nx + 3) / 4;
  unsigned bad = 0;
  for (int64_t r = w0; r < nrows; r += nw) {
    const float4* row = p + r * row4;
    for (int c = lane; c < nx4; c += 32) {
      const float4 v = row[c];
      const int x = 4 * c;
      bad |= nonfinite_bit(v.x);  // x < nx: c < nx4
      if (x + 1 < nx) bad |= nonfinite_bit(v.y);
      if (x + 2 < nx) bad |= nonfinite_bit(v.z);
      if (x + 3 < nx) bad |= nonfinite_bit(v.w);
    }
  }
  if (bad) atomicOr(status, kStatusNonFinite);
}

// ---------------------------------------------------------------------------------------------
// pitch-padding canaries (a debugging aid): fill the padding columns x0 .. nxp-1 of nrows rows with a
// value, or count the entries there that are no longer NaN (a kernel wrote out of its row)
// ---------------------------------------------------------------------------------------------
__global__ void k_fill_padding(float* base, int64_t nrows, int x0, int nxp, float v) {
  const int w = nxp - x0;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < nrows * w; m += (int64_t)gridDim.x * blockDim.x)
    base[(m / w) * nxp + x0 + m % w] = v;
}

__global__ void k_count_padding(const float* __restrict__ base, int64_t nrows, int x0, int nxp,
                                unsigned long long* count) {
  const int w = nxp - x0;
  unsigned long long c = 0;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < nrows * w; m += (int64_t)gridDim.x * blockDim.x)
    c += isnan(base[(m / w) * nxp + x0 + m % w]) ? 0ull : 1ull;
  if (c) atomicAdd(count, c);
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

// One Adam step of the design loop on the latent variables theta, with the smoothed Heaviside
// projection rho = P(theta) (see fdtd_design_adam_step). P's constants tbe = tanh(beta eta) and
// tden = tanh(beta eta) + tanh(beta (1 - eta)) and the bias corrections bc1 = 1 - beta1^t,
// bc2 = 1 - beta2^t come from the host; beta = 0 selects the identity projection.
__global__ void k_design_adam(const float* __restrict__ g_rho, float* theta, float* m, float* v, float* rho,
                              int64_t n, float lr, float b1, float b2, float eps, float bc1, float bc2,
                              float beta, float eta, float tbe, float tden) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float th = theta[i];
  float dp = 1.f;  // P'(theta)
  if (beta > 0.f) {
    const float t = tanhf(beta * (th - eta));
    dp = beta * (1.f - t * t) / tden;
  }
  const float gr = g_rho[i] * dp;
  const float mm = b1 * m[i] + (1.f - b1) * gr;
  const float vv = b2 * v[i] + (1.f - b2) * gr * gr;
  th -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
  th = fminf(fmaxf(th, 0.f), 1.f);
  m[i] = mm;
  v[i] = vv;
  theta[i] = th;
  rho[i] = beta > 0.f ? (tbe + tanhf(beta * (th - eta))) / tden : th;
}

__global__ void k_design_project(const float* __restrict__ theta, float* rho, int64_t n, float beta, float eta,
                                 float tbe, float tden) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  rho[i] = beta > 0.f ? (tbe + tanhf(beta * (theta[i] - eta))) / tden : theta[i];
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

void launch_source(const Geo& g, const Fields& F, const SrcDev& src, int step, float sign, int only_R,
                   cudaStream_t s) {
  const int64_t n = (int64_t)(src.hi[0] - src.lo[0]) * (src.hi[1] - src.lo[1]) * (src.hi[2] - src.lo[2]);
  if (n <= 0) return;
  k_source<<<blocks_for(n, 256), 256, 0, s>>>(g, F, src, step, sign, only_R);
}

void launch_source_scale_a(const Geo& g, const float* a, const SrcDev& src, cudaStream_t s) {
  const int64_t n = (int64_t)(src.hi[0] - src.lo[0]) * (src.hi[1] - src.lo[1]) * (src.hi[2] - src.lo[2]);
  if (n > 0) k_source_scale_a<<<blocks_for(n, 256), 256, 0, s>>>(g, a, src);
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

void launch_face_copy(const Geo& g, const Fields& F, const FaceSet& fs, float* rec, int to_record, cudaStream_t s) {
  int64_t mx = 0;
  for (int q = 0; q < fs.nseg; ++q) mx = std::max<int64_t>(mx, (int64_t)fs.seg[q].n1 * fs.seg[q].n2);
  if (fs.nseg == 0 || mx == 0) return;
  dim3 grid((unsigned)((mx + 255) / 256), fs.nseg);
  launch_pdl(k_face_copy, grid, dim3(256), 0, s, g, F, fs, rec, to_record);
}

void launch_face_copy_group(const FaceGroup& G, cudaStream_t s) {
  int64_t mx = 0;
  int nseg = 0;
  for (int r = 0; r < G.n; ++r) {
    nseg = std::max(nseg, G.e[r].fs.nseg);
    for (int q = 0; q < G.e[r].fs.nseg; ++q) mx = std::max<int64_t>(mx, (int64_t)G.e[r].fs.seg[q].n1 * G.e[r].fs.seg[q].n2);
  }
  if (G.n == 0 || nseg == 0 || mx == 0) return;
  dim3 grid((unsigned)((mx + 255) / 256), nseg, G.n);
  launch_pdl(k_face_copy_group, grid, dim3(256), 0, s, G);
}

void launch_detector_adjoint(const Geo& g, const Fields& F, const Fields& A, const DetDev& d, int step,
                             const double* dL_ddet, cudaStream_t s) {
  const int64_t n = d.kind == 0 ? 1 : (int64_t)(d.hi[0] - d.lo[0]) * (d.hi[1] - d.lo[1]) * (d.hi[2] - d.lo[2]);
  launch_pdl(k_det_adjoint, dim3(blocks_for(n, 256)), dim3(256), 0, s, g, F, A, d, step, dL_ddet);
}

// One bounded wait, as the stencil kernels make it, on an mbarrier that nothing arrives on: it gives up
// after limit_ns, sets the timeout bit in *status and writes the nanoseconds it waited (diagnostic of
// the timeout path; no copy is ever issued to the barrier, so none is in flight when the block exits).
__global__ void k_wait_probe(int* status, unsigned long long* waited_ns, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_init_fence();
  const uint64_t t0 = global_ns();
  const bool ok = mbar_wait_for(&bar, 0, limit_ns);
  *waited_ns = global_ns() - t0;
  if (!ok) atomicOr(status, kStatusTimeout);
}

void launch_wait_probe(int* status, unsigned long long* waited_ns, unsigned long long limit_ns, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(status, waited_ns, limit_ns);
}

void launch_check_finite(const Geo& g, const float* p, int64_t n, int* status, int nsm, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t nrows = n / g.nxp;  // whole rows of the pitch-padded arrays
  const unsigned blocks = (unsigned)std::min<int64_t>(blocks_for(nrows, 8), 8 * (int64_t)nsm);  // 8 warps a block
  launch_pdl(k_check_finite, dim3(blocks), dim3(256), 0, s, reinterpret_cast<const float4*>(p), nrows, g.n[0],
             g.nxp, status);
}

void launch_fill_padding(const Geo& g, float* base, int64_t nrows, int x0, float v, int nsm, cudaStream_t s) {
  if (x0 >= g.nxp || nrows <= 0) return;
  const unsigned blocks = (unsigned)std::min<int64_t>(blocks_for(nrows * (g.nxp - x0), 256), 4 * (int64_t)nsm);
  k_fill_padding<<<blocks, 256, 0, s>>>(base, nrows, x0, g.nxp, v);
}

void launch_count_padding(const Geo& g, const float* base, int64_t nrows, int x0, unsigned long long* count,
                          int nsm, cudaStream_t s) {
  if (x0 >= g.nxp || nrows <= 0) return;
  const unsigned blocks = (unsigned)std::min<int64_t>(blocks_for(nrows * (g.nxp - x0), 256), 4 * (int64_t)nsm);
  k_count_padding<<<blocks, 256, 0, s>>>(base, nrows, x0, g.nxp, count);
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

void launch_design_adam(const float* g_rho, float* theta, float* m, float* v, float* rho, int64_t n, int t, double lr,
                        double b1, double b2, double eps, double beta, double eta, cudaStream_t s) {
  if (n <= 0) return;
  const double tbe = beta > 0 ? std::tanh(beta * eta) : 0.0;
  const double tden = beta > 0 ? tbe + std::tanh(beta * (1.0 - eta)) : 1.0;
  const double bc1 = 1.0 - std::pow(b1, t), bc2 = 1.0 - std::pow(b2, t);
  k_design_adam<<<blocks_for(n, 256), 256, 0, s>>>(g_rho, theta, m, v, rho, n, (float)lr, (float)b1, (float)b2, (float)eps,
                                                   (float)bc1, (float)bc2, (float)beta, (float)eta, (float)tbe,
                                                   (float)tden);
}

void launch_design_project(const float* theta, float* rho, int64_t n, double beta, double eta, cudaStream_t s) {
  if (n <= 0) return;
  const double tbe = beta > 0 ? std::tanh(beta * eta) : 0.0;
  const double tden = beta > 0 ? tbe + std::tanh(beta * (1.0 - eta)) : 1.0;
  k_design_project<<<blocks_for(n, 256), 256, 0, s>>>(theta, rho, n, (float)beta, (float)eta, (float)tbe, (float)tden);
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
