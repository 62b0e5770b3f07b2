// Internal device-side types and kernel launchers of libfdtd (not part of the C ABI).
//
// Data layout in HBM (one solver):
//   - six field arrays Ex, Ey, Ez, Hx, Hy, Hz, float32, [nz][ny][nxp] with x fastest and the row pitch
//     nxp rounded up to 32 floats (128-byte rows);
//   - a = 1/eps, float32, same layout;
//   - CPML memories psi only inside the layers: for the derivative along axis d, component c != d,
//     a compact array whose axis-d extent is the total layer width (x: [nz][ny][Lx], y: [nz][Ly][nxp],
//     z: [Lz][ny][nxp]);
//   - per-axis CPML tables b, c, 1/kappa at integer and half positions (float32);
//   - boundary-face history: per step, the tangential H on the planes just outside the PML-free
//     region, packed segment by segment;
//   - adjoint fields with the same layout as the fields; dL/da accumulated in float64 over the design box.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {

constexpr int kMaxFaceSeg = 12;
constexpr int kPitchAlign = 32;
constexpr int kMaxSrc = 4;    // sources handled inside the fused kernels (the rest by extra launches)
constexpr int kMaxDet = 4;    // detectors handled inside the fused kernels
// bits of the device status word
constexpr int kStatusTimeout = 1;    // a bounded wait for a TMA copy gave up
constexpr int kStatusNonFinite = 2;  // a field check found a NaN or an infinity

struct Geo {
  int n[3];           // cells nx, ny, nz
  int nxp;            // row pitch in floats
  int64_t plane;      // nxp * ny
  int64_t vol;        // plane * nz
  int pml[6];         // layer widths x-lo, x-hi, y-lo, y-hi, z-lo, z-hi
  int slab[3];        // pml[2d] + pml[2d+1]
  float S;            // Courant number
  // PML-free region R, inclusive index ranges along each axis for integer and half positions
  int rint_lo[3], rint_hi[3], rhalf_lo[3], rhalf_hi[3];
};

struct Tables {
  // [axis][0 = integer positions, 1 = half positions], n[axis] entries each
  const float* b[3][2];
  const float* c[3][2];
  const float* ik[3][2];   // 1 / kappa
  const int* sidx[3];      // slab index of each position along the axis, -1 off the layers
};

struct Fields {
  float* f[6];
};

struct PsiSet {
  float* p[3][3];          // [component][axis]; nullptr on the diagonal or when the axis has no layer
};

struct FaceSeg {
  int axis, idx, comp;     // plane normal, index along it, H component
  int lo1, n1, lo2, n2;    // box along e1 = axis+1 and e2 = axis+2 (mod 3)
  int64_t off;             // offset of the segment inside one step's record
};

struct FaceSet {
  int nseg;
  int64_t per_step;        // floats per step
  FaceSeg seg[kMaxFaceSeg];
};

struct SrcDev {
  int comp;
  int lo[3], hi[3];
  const float* w;          // box-shaped amplitude * profile (0 where E is held by a PEC wall)
  const float* g;          // waveform samples g(n + 1/2), one per step
};

struct DetDev {
  int kind, comp, axis;
  int lo[3], hi[3];
  int64_t off;             // offset into the concatenated detector output
  int nblk;                // flux: partial-sum slots per step
  int64_t poff;            // flux: offset of this detector's slots in the partial-sum buffer
};

// Arguments of one fused forward step (read `cur`, write `nxt`).
struct FwdArgs {
  Geo g;
  Tables T;
  Fields cur, nxt;
  PsiSet psiE_cur, psiE_nxt, psiH_cur, psiH_nxt;
  const float* a;
  int step;
  int tz;                  // z-planes per block
  int nstage;              // stages of the plane ring (3 or 4)
  int nsrc;
  SrcDev src[kMaxSrc];
  int ndet;
  DetDev det[kMaxDet];
  double* det_out;
  double* partial;
  int* status;             // device status word: bit 0 set when a bounded wait gave up
};

__host__ __device__ inline int64_t cell_index(const Geo& g, int i, int j, int k) {
  return (int64_t)k * g.plane + (int64_t)j * g.nxp + i;
}

__host__ __device__ inline int slab_index(const Geo& g, int d, int x) {
  const int p0 = g.pml[2 * d], p1 = g.pml[2 * d + 1];
  if (x < p0) return x;
  if (x >= g.n[d] - p1) return p0 + x - (g.n[d] - p1);
  return -1;
}

// slab index of position x along an axis with n cells and layers p0, p1 (-1 off the layers): the
// same index for the integer and the half position x (+ 1/2)
__host__ __device__ inline int slab_of_pos(int x, int n, int p0, int p1) {
  return x < p0 ? x : (x >= n - p1 ? p0 + x - (n - p1) : -1);
}

__host__ __device__ inline int64_t psi_index(const Geo& g, int d, int i, int j, int k, int s) {
  if (d == 0) return ((int64_t)k * g.n[1] + j) * g.slab[0] + s;
  if (d == 1) return ((int64_t)k * g.slab[1] + s) * g.nxp + i;
  return ((int64_t)s * g.n[1] + j) * g.nxp + i;
}

__host__ __device__ inline int64_t psi_elems(const Geo& g, int d) {
  if (d == 0) return (int64_t)g.n[2] * g.n[1] * g.slab[0];
  if (d == 1) return (int64_t)g.n[2] * g.slab[1] * g.nxp;
  return (int64_t)g.slab[2] * g.n[1] * g.nxp;
}

// ---- launchers (fdtd_kernels.cu) --------------------------------------------------------------
void launch_source(const Geo& g, const Fields& F, const SrcDev& src, int step, float sign, int only_R,
                   cudaStream_t s);
// interpolated detectors (fdtd_interp.cu)
int64_t interp_slab_floats(const DetDev& d);
void launch_detector_interp(const Geo& g, const Fields& P, const Fields& F, const DetDev& d, int step, double* out,
                            double* partial, cudaStream_t s);
void launch_slab_copy(const Geo& g, const Fields& F, const DetDev& d, int comp0, float* out, cudaStream_t s);
void launch_interp_adjoint(const Geo& g, const Fields& F, const Fields& A, const DetDev& d, int step,
                           const double* dL_ddet, int part, const float* slabE0, const float* slabE1,
                           const float* slabH, cudaStream_t s);
void launch_source_scale_a(const Geo& g, const float* a, const SrcDev& src, cudaStream_t s);
void launch_detector_sample(const Geo& g, const Fields& F, const DetDev& d, int step, double* out,
                            double* partial, cudaStream_t s);
void launch_flux_finalize(const DetDev& d, int nsteps, const double* partial, double* out, cudaStream_t s);
void launch_face_copy(const Geo& g, const Fields& F, const FaceSet& fs, float* rec, int to_record, cudaStream_t s);
// The face record (to_record = 1) or replay of several requests in one launch (at most 8).
struct FaceJob {
  Geo g;
  Fields F;
  FaceSet fs;
  float* rec;
};
struct FaceGroup {
  int n;
  int to_record;
  FaceJob e[8];
};
void launch_face_copy_group(const FaceGroup& G, cudaStream_t s);
void launch_detector_adjoint(const Geo& g, const Fields& F, const Fields& A, const DetDev& d, int step,
                             const double* dL_ddet, cudaStream_t s);
// Flag kStatusNonFinite in *status if one of the grid cells of the n floats at p (whole pitch-padded
// arrays: n a multiple of 4, p 16-byte aligned) is NaN or infinite; the pitch padding is not read.
void launch_check_finite(const Geo& g, const float* p, int64_t n, int* status, int nsm, cudaStream_t s);
void launch_wait_probe(int* status, unsigned long long* waited_ns, unsigned long long limit_ns, cudaStream_t s);
// Pitch-padding canaries of nrows rows at base, in columns x0 .. nxp-1: fill them with v, or add the
// number of them that are not NaN to *count (a debugging aid against writes out of a row).
void launch_fill_padding(const Geo& g, float* base, int64_t nrows, int x0, float v, int nsm, cudaStream_t s);
void launch_count_padding(const Geo& g, const float* base, int64_t nrows, int x0, unsigned long long* count,
                          int nsm, cudaStream_t s);
void launch_grad_finalize(const Geo& g, const float* a, const int* dlo, const int* dhi, const double* dLda,
                          float* dL_deps, double scale, cudaStream_t s);
void launch_design_adam(const float* g_rho, float* theta, float* m, float* v, float* rho, int64_t n, int t, double lr,
                        double b1, double b2, double eps, double beta, double eta, cudaStream_t s);
void launch_design_project(const float* theta, float* rho, int64_t n, double beta, double eta, cudaStream_t s);
void launch_set_density(const Geo& g, float* a, const int* lo, const int* hi, const float* rho, float eps_lo,
                        float deps, cudaStream_t s);
// Arguments of the reverse-step kernels (in place on the fields F and the adjoint fields B).
struct RevArgs {
  Geo g;
  Tables T;
  Fields F, B;
  PsiSet pin, pout;        // psi-bar of E (rev_E) or of H (rev_H): read pin, write pout
  const float* a;
  int step;
  int tz;
  int dlo[3], dhi[3];      // design box
  double* dLda;
  int nsrc;
  SrcDev src[kMaxSrc];
  int* status;             // device status word: bit 0 set when a bounded wait gave up
  int nstage;              // stages of the plane ring (3 or 4)
  int inverse;             // 1: rebuild the previous fields in place (time reversal); 0: adjoint only
                           // (the forward state comes from elsewhere, e.g. recomputation)
  // Detector adjoints folded into rev_H's E-bar write: the terms of detector step det_step (-1: none)
  // of the ndet detectors in det (points on an E component, boxes of time-integrated |E|^2), which
  // use only E after that step, the E that rev_H of the following step holds. gy: dL/d(outputs).
  int ndet = 0;
  int det_step = -1;
  const double* gy = nullptr;
  DetDev det[kMaxDet];
};

// Arguments of the fused inverse step (fdtd_inverse.cu): read `cur` (E^{n+1}, H^{n+1/2} with the
// boundary faces replayed), write `nxt` (E^n, H^{n-1/2} on the PML-free region R), and accumulate
// dL/da += S Ebar . curl_b(H^{n+1/2}) on the design box from the adjoint of E^{n+1} in `eb`.
struct InvArgs {
  Geo g;
  Fields cur, nxt;
  const float* a;
  int step;
  int tz;
  int nstage;
  int nsrc;
  SrcDev src[kMaxSrc];
  int dlo[3], dhi[3];      // design box
  double* dLda;            // null: no gradient
  const float* eb[3];      // adjoint of E^{n+1}
  int* status;
};

// Arguments of the fused adjoint step (fdtd_adjoint.cu): read the adjoint fields `cur`, write `nxt`;
// psi-bar memories of E and H read from pinE/pinH and written to poutE/poutH; the folded detector
// adjoints of step det_step (-1: none) read E of that step from `prim`.
struct AdjArgs {
  Geo g;
  Tables T;
  Fields cur, nxt;
  Fields prim;
  PsiSet pinE, poutE, pinH, poutH;
  const float* a;
  int tz;
  int nstage;
  int* status;
  int ndet = 0;
  int det_step = -1;
  const double* gy = nullptr;
  DetDev det[kMaxDet];
  // A split step (split = 1) runs as two launches: the tiles that need the x/y CPML path (a frame:
  // the first xl and last xh tile columns, the first yl and last yh tile rows) with z-chunks of tz_xy,
  // then the plain tiles inside it with z-chunks of tz. Each launch's kernel holds only its own plane
  // loop, which runs faster than a loop that also holds the other. split = 0: one launch of all tiles.
  int split = 0;
  int xl = 0, xh = 0, yl = 0, yh = 0;
  int tz_xy = 8;
};

int fused_tile_x();
int fused_max_tz();   // z-planes one block of the forward kernel may march at most
int fused_tile_y();
int rev_tile_x();     // column tile of the reverse kernels
int rev_tile_y();
void launch_pack_fields(const Geo& g, const Fields& F, float* out6, int unpack, cudaStream_t s);
void launch_set_box(const Geo& g, float* a, const int* lo, const int* hi, const float* box, cudaStream_t s);

// Launch with programmatic dependent launch allowed: the kernel may be scheduled while the previous
// kernel in the stream finishes, and must call pdl_wait() before it touches memory that kernel
// reads or writes. Inside a captured graph this becomes a programmatic dependency edge.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

#if defined(__CUDACC__)
// Wait until the previous kernel of the stream has completed and its memory operations are visible.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// Record `msg` as the calling thread's last error (fdtd_last_error) and return `code`.
int set_error(int code, const char* msg);

// Whether p points to device or managed memory of the current CUDA device (false for host memory,
// another GPU's memory, or when no device can be queried).
bool on_current_device(const void* p);

}  // namespace fdtd
