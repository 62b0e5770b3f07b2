// Poynting flux of caller-provided fields through a cell box, computed without allocating memory.
//
// Some callers cannot call cudaMalloc: hosts that hand the library a fixed memory budget up front,
// or real-time loops where an allocation may stall. This entry point computes the flux with a
// two-pass, fixed-order FP64 reduction (per-block partial sums, then one ordered sum: deterministic
// from call to call, equal to the solver's flux detector to rounding), but keeps the partial sums in
// a fixed array in device memory that the library reserves when it is loaded, instead of scratch it
// allocates.
//
// The array holds kMaxSlots partial sums (8 KiB); every GPU that loads the library keeps it until the
// process exits. Each block reduces kCellsPerBlock cells, so a box may hold at most
// kMaxSlots * kCellsPerBlock cells; larger boxes are rejected.
#include <mutex>

#include "../../include/fdtd.h"
#include "fdtd_internal.cuh"

namespace {

constexpr int kMaxSlots = 1024;
constexpr int kCellsPerBlock = 4096;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; each call overwrites the slots it reads before reading them.
static __device__ __align__(256) double g_flux_slots[kMaxSlots];

std::mutex g_mu;
double* g_slot_ptr[kMaxDevices] = {nullptr};

__global__ void __launch_bounds__(kThreads) k_flux_partial(const float* __restrict__ f6, int nx, int ny, int nz,
                                                           int axis, int lx, int ly, int lz, int bx, int by, int bz,
                                                           double* __restrict__ slots) {
  __shared__ double sh[kThreads];
  const int64_t N = (int64_t)nx * ny * nz;
  const int64_t M = (int64_t)bx * by * bz;
  const int64_t m0 = (int64_t)blockIdx.x * kCellsPerBlock, m1 = min(M, m0 + kCellsPerBlock);
  const int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
  const float* E1 = f6 + a1 * N;
  const float* E2 = f6 + a2 * N;
  const float* H1 = f6 + (3 + a1) * N;
  const float* H2 = f6 + (3 + a2) * N;
  double acc = 0.0;
  for (int64_t m = m0 + threadIdx.x; m < m1; m += kThreads) {
    const int x = lx + (int)(m % bx);
    const int64_t r = m / bx;
    const int y = ly + (int)(r % by);
    const int z = lz + (int)(r / by);
    const int64_t q = ((int64_t)z * ny + y) * nx + x;
    acc += (double)E1[q] * (double)H2[q] - (double)E2[q] * (double)H1[q];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) slots[blockIdx.x] = sh[0];
}

__global__ void k_flux_sum(const double* __restrict__ slots, int nslots, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nslots; ++b) s += slots[b];
  *out = s;
}

// Device address of the slot array on the current device, looked up once per device and kept for the
// life of the process (a cudaDeviceReset after the first call is not supported: the address would
// be stale).
int slot_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fdtd::set_error(FDTD_ERR_CUDA, "fdtd_plane_flux_noalloc: no usable current CUDA device");
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_slot_ptr[dev]) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_flux_slots);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fdtd::set_error(FDTD_ERR_CUDA, "fdtd_plane_flux_noalloc: cudaGetSymbolAddress failed");
    }
    g_slot_ptr[dev] = p;
  }
  *out = g_slot_ptr[dev];
  return FDTD_OK;
}

}  // namespace

extern "C" int fdtd_plane_flux_noalloc(const float* fields6, const fdtd_grid* grid, int32_t axis,
                                       const int32_t lo[3], const int32_t hi[3], double* out,
                                       void* cuda_stream) {
  if (!fields6 || !grid || !lo || !hi || !out)
    return fdtd::set_error(FDTD_ERR_INVALID_ARG, "fdtd_plane_flux_noalloc: NULL argument");
  const int n[3] = {grid->nx, grid->ny, grid->nz};
  if (axis < 0 || axis > 2) return fdtd::set_error(FDTD_ERR_INVALID_ARG, "fdtd_plane_flux_noalloc: axis must be 0..2");
  for (int d = 0; d < 3; ++d)
    if (n[d] < 1 || lo[d] < 0 || hi[d] > n[d] || lo[d] >= hi[d])
      return fdtd::set_error(FDTD_ERR_INVALID_ARG, "fdtd_plane_flux_noalloc: empty box or box outside the grid");
  const int64_t cells = (int64_t)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  const int64_t nslots = (cells + kCellsPerBlock - 1) / kCellsPerBlock;
  if (nslots > kMaxSlots)
    return fdtd::set_error(FDTD_ERR_INVALID_ARG,
                           "fdtd_plane_flux_noalloc: box exceeds the 4194304-cell maximum of the fixed scratch");
  // both buffers must be device (or managed) memory of the current device: a host pointer or another
  // GPU's buffer is refused before anything is launched
  if (!fdtd::on_current_device(fields6) || !fdtd::on_current_device(out))
    return fdtd::set_error(FDTD_ERR_INVALID_ARG,
                           "fdtd_plane_flux_noalloc: fields6 and out must be device memory of the current device");
  double* slots = nullptr;
  const int rc = slot_address(&slots);
  if (rc != FDTD_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_flux_partial<<<(unsigned)nslots, kThreads, 0, st>>>(fields6, n[0], n[1], n[2], axis, lo[0], lo[1], lo[2],
                                                       hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], slots);
  k_flux_sum<<<1, 32, 0, st>>>(slots, (int)nslots, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fdtd::set_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
  return FDTD_OK;
}
