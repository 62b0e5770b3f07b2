// Host side of the libfdtd C ABI (include/fdtd.h): validation, device memory, CPML and source tables,
// and the forward and reverse time loops of arXiv 2412.12360 Sec. 2.1-2.2.
//
// The time loops are captured once into CUDA graphs (one per phase, keyed by step count and flags)
// and replayed for every later solve of the same shape, so a solve costs one graph launch per phase
// instead of thousands of kernel launches.
#include <algorithm>
#include <memory>
#include <limits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/fdtd.h"
#include "fdtd_internal.cuh"
#include "fdtd_tma.cuh"

#include <cudaTypedefs.h>
#include <mutex>

using namespace fdtd;

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
}

namespace fdtd {

int encode_field_map(CUtensorMap* m, const float* base, const Geo& g, int ncomp, MapBox box) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return set_error(FDTD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[4] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2], (cuuint64_t)ncomp};
  const cuuint64_t strides[3] = {(cuuint64_t)g.nxp * 4, (cuuint64_t)g.plane * 4, (cuuint64_t)g.vol * 4};
  const cuuint32_t boxd[4] = {(cuuint32_t)box.w, (cuuint32_t)box.h, 1, (cuuint32_t)ncomp};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims, strides, boxd, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(FDTD_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return FDTD_OK;
}

}  // namespace fdtd

namespace {

thread_local std::string g_last_error;
int64_t g_byte_budget = -1;  // process-wide cap on bytes one handle may allocate (-1 = none)

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CK(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return fail(FDTD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

#define TRY(x)                      \
  do {                              \
    int rc_ = (x);                  \
    if (rc_ != FDTD_OK) return rc_; \
  } while (0)

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// z-planes per block of a z-marching kernel over nxy column tiles and nz planes with `slots` blocks
// resident on the device at once. A march of tz planes takes about tz + 2 plane-times (the pipeline
// start and the extra plane beside the chunk), so the sweep takes waves x (tz + 2): pick tz in
// [1, 32] minimising that (the larger tz on ties). On one B300 this gives 6 (forward, 4 blocks/SM)
// and 8 (reverse, 3/SM) planes on 96^3 and 32 on 600^3, where a sweep over 16..32 measured within a
// few percent and 300 planes per block measured 20 % slower.
int choose_tz(int64_t nxy, int nz, int64_t slots) {
  int best = 1;
  double bestc = 1e300;
  for (int tz = 1; tz <= std::min(32, nz); ++tz) {
    const int64_t chunks = (nz + tz - 1) / tz;
    const int64_t waves = (nxy * chunks + slots - 1) / slots;
    const double c = double(waves) * (tz + 2);
    if (c <= bestc) {
      bestc = c;
      best = tz;
    }
  }
  return best;
}

// The z-chunk of the requests of a grouped launch whose results do not depend on it (free[r]; the
// others keep own[r]), chosen as choose_tz chooses one grid's: the group's blocks in waves of `slots`
// resident blocks, a wave costing its longest march plus two planes of start-up. Each request alone
// fills the GPU with short chunks; side by side they fill it with longer ones, which recompute fewer
// halo planes per plane marched.
int group_tz(int n, const int64_t* nxy, const int* nz, const int* own, const bool* free_, int64_t slots, int tz_max) {
  int best = 1;
  double bestc = 1e300;
  for (int tz = 1; tz <= tz_max; ++tz) {
    int64_t blocks = 0;
    int longest = 0;
    for (int r = 0; r < n; ++r) {
      const int t = free_[r] ? std::min(tz, nz[r]) : own[r];
      blocks += nxy[r] * ((nz[r] + t - 1) / t);
      longest = std::max(longest, std::min(t, nz[r]));
    }
    const double c = double((blocks + slots - 1) / slots) * (longest + 2);
    if (c <= bestc) {
      bestc = c;
      best = tz;
    }
  }
  return best;
}

// The frame of the split adjoint step: the leading and trailing tile columns (f[0], f[1]) and rows
// (f[2], f[3]) whose march needs the x/y CPML loop; false when no rectangle of plain tiles is left
// inside them (the step is then one launch).
bool adjoint_frame(const Geo& g, int f[4]) {
  const int ntx = adj_tiles_x(g), nty = adj_tiles_y(g);
  int xl = 0, xh = 0, yl = 0, yh = 0;
  while (xl < ntx && adj_tile_xy(g, 0, xl)) ++xl;
  while (xh < ntx - xl && adj_tile_xy(g, 0, ntx - 1 - xh)) ++xh;
  while (yl < nty && adj_tile_xy(g, 1, yl)) ++yl;
  while (yh < nty - yl && adj_tile_xy(g, 1, nty - 1 - yh)) ++yh;
  bool ok = xl + xh < ntx && yl + yh < nty;
  for (int b = xl; ok && b < ntx - xh; ++b) ok = !adj_tile_xy(g, 0, b);
  for (int b = yl; ok && b < nty - yh; ++b) ok = !adj_tile_xy(g, 1, b);
  f[0] = xl;
  f[1] = xh;
  f[2] = yl;
  f[3] = yh;
  return ok;
}

// The reverse-step kind of a grid. The fused pair moves 104 B per cell against 148 but does its CPML
// work (the adjoint's coefficients gathered from both neighbours) in every tile that touches an x or y
// layer, and its 32 x 16 tiles give small grids fewer blocks. On one B300, fwd+grad ms per step with
// the fused / in-place pair (fraction of tiles touching an x or y layer): 600^3 7.1 / 7.6 (18 %), 400^3
// 2.42 / 2.63 (22 %), 240x240x960 2.29 / 2.40 (35 %), 256^3 0.765 / 0.796 (34 %), 200^3 0.501 / 0.473
// (56 %), 128x128x256 0.306 / 0.266 (63 %), 96^3 (78 %) slower still. So: the fused pair for grids of
// at least 12 M cells whose tiles touch a layer in at most 40 % of the cases.
bool fused_reverse(const Geo& g) {
  const int tx = fused_tile_x(), ty = fused_tile_y();
  const int nx = g.n[0], ny = g.n[1];
  const int ntx = (nx + tx - 1) / tx, nty = (ny + ty - 1) / ty;
  int plain_x = 0, plain_y = 0;
  for (int b = 0; b < ntx; ++b) plain_x += !(b * tx - 1 < g.pml[0] || b * tx + tx >= nx - g.pml[1] - 1);
  for (int b = 0; b < nty; ++b) plain_y += !(b * ty - 1 < g.pml[2] || b * ty + ty >= ny - g.pml[3] - 1);
  const double xy_frac = 1.0 - (double)plain_x * plain_y / ((double)ntx * nty);
  return (int64_t)nx * ny * g.n[2] >= (int64_t)12 << 20 && xy_frac <= 0.4;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no link to libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// CPML grading at one position (d = depth of the component's own position into the layer).
void cpml_coef(double x, int N, int p0, int p1, const fdtd_pml& pm, double& b, double& c, double& ik) {
  double d = 0.0;
  if (p0 > 0 && x < p0) d = (p0 - x) / p0;
  else if (p1 > 0 && x > N - p1) d = (x - (N - p1)) / p1;
  if (d <= 0.0) {
    b = 1.0;
    c = 0.0;
    ik = 1.0;
    return;
  }
  const double dm = std::pow(d, pm.grading_m);
  const double sigma = pm.sigma_max * dm;
  const double kappa = 1.0 + (pm.kappa_max - 1.0) * dm;
  const double alpha = pm.alpha_max * (1.0 - d);
  b = std::exp(-(sigma / kappa + alpha));
  c = sigma == 0.0 ? 0.0 : sigma / (sigma * kappa + kappa * kappa * alpha) * (b - 1.0);
  ik = 1.0 / kappa;
}

double pulse(const fdtd_source& s, double S, double t) {
  const double P = s.wavelength_cells / S;
  const double u = t - s.t0_steps;
  return std::sin(2.0 * M_PI * u / P) * std::exp(-(u / s.tau_steps) * (u / s.tau_steps));
}

// A one-sided TFSF plane source (see fdtd_source): travel axis and direction, its E and H components
// c and h, and sE, sH = +-1, the signs of the axis derivatives in (curl H)_c and (curl E)_h.
struct Tfsf {
  fdtd_source s;
  int axis, dir, c, h;
  double sE, sH;
};

Tfsf make_tfsf(const fdtd_source& s) {
  Tfsf t;
  t.s = s;
  t.s.profile = nullptr;
  t.axis = std::abs(s.tfsf) - 1;
  t.dir = s.tfsf > 0 ? 1 : -1;
  t.c = s.component;
  t.h = 3 - t.axis - t.c;
  t.sE = t.axis == (t.c + 1) % 3 ? 1.0 : -1.0;  // (curl H)_c = dH_{c+2}/dx_{c+1} - dH_{c+1}/dx_{c+2}
  t.sH = t.axis == (t.h + 1) % 3 ? 1.0 : -1.0;  // (curl E)_h = dE_{h+2}/dx_{h+1} - dE_{h+1}/dx_{h+2}
  return t;
}

// Incident field of a TFSF source for steps 0..nsteps-1, in FP64 on the host (it does not depend on
// the 3-D fields): a one-dimensional Yee line along the travel axis, the 3-D update restricted to the
// axis with a = 1/eps_background, driven by the source's soft pulse four cells upstream of the
// sampling point K. einc[n] = E^n at K (the plane), hinc[n] = H^{n+1/2} at K - 1/2 (travel +) or
// K + 1/2 (travel -). The line is long enough that nothing reflected from its ends returns to K
// within nsteps (waves move at most S cells per step).
void tfsf_incident(const Tfsf& t, double S, int nsteps, std::vector<double>& einc, std::vector<double>& hinc) {
  const int L = 2 * nsteps + 16, K = nsteps + 8, ks = K - 4 * t.dir;
  const double ab = 1.0 / t.s.eps_background;
  std::vector<double> E(L, 0.0), H(L, 0.0);  // H[k] at k + 1/2; E[0] stays 0
  einc.assign(nsteps, 0.0);
  hinc.assign(nsteps, 0.0);
  for (int n = 0; n < nsteps; ++n) {
    einc[n] = E[K];
    for (int k = 0; k < L - 1; ++k) H[k] -= S * t.sH * (E[k + 1] - E[k]);
    hinc[n] = H[t.dir > 0 ? K - 1 : K];
    for (int k = 1; k < L; ++k) E[k] += S * ab * t.sE * (H[k] - H[k - 1]);
    E[ks] += t.s.amplitude * pulse(t.s, S, n + 0.5);
  }
}

bool box_ok(const int32_t lo[3], const int32_t hi[3], const int n[3], bool allow_empty) {
  for (int d = 0; d < 3; ++d) {
    if (lo[d] < 0 || hi[d] > n[d] || lo[d] > hi[d]) return false;
    if (!allow_empty && lo[d] == hi[d]) return false;
  }
  return true;
}

int64_t box_cells(const int32_t lo[3], const int32_t hi[3]) {
  return int64_t(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
}

Geo make_geo(const fdtd_grid& gr, const fdtd_pml& pm, double S) {
  Geo g;
  g.n[0] = gr.nx;
  g.n[1] = gr.ny;
  g.n[2] = gr.nz;
  g.nxp = (int)round_up(gr.nx, kPitchAlign);
  g.plane = (int64_t)g.nxp * gr.ny;
  g.vol = g.plane * gr.nz;
  for (int f = 0; f < 6; ++f) g.pml[f] = pm.thickness[f];
  for (int d = 0; d < 3; ++d) {
    g.slab[d] = pm.thickness[2 * d] + pm.thickness[2 * d + 1];
    g.rint_lo[d] = pm.thickness[2 * d];
    g.rint_hi[d] = std::min(g.n[d] - pm.thickness[2 * d + 1], g.n[d] - 1);
    g.rhalf_lo[d] = pm.thickness[2 * d];
    g.rhalf_hi[d] = g.n[d] - pm.thickness[2 * d + 1] - 1;
  }
  g.S = (float)S;
  return g;
}

// Tangential H on the planes just outside the PML-free region R (Sec. 2.2, "six two-dimensional
// slices"): along axis d, components d+1 and d+2 at index p_lo - 1 and at n - p_hi, over the
// integer-position range of R on the two other axes.
FaceSet make_faces(const Geo& g) {
  FaceSet fs;
  fs.nseg = 0;
  fs.per_step = 0;
  for (int d = 0; d < 3; ++d) {
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    for (int side = 0; side < 2; ++side) {
      const int p = g.pml[2 * d + side];
      if (p == 0) continue;
      for (int comp : {e1, e2}) {
        FaceSeg& s = fs.seg[fs.nseg++];
        s.axis = d;
        s.idx = side == 0 ? p - 1 : g.n[d] - p;
        s.comp = comp;
        s.lo1 = g.rint_lo[e1];
        s.n1 = g.rint_hi[e1] - g.rint_lo[e1] + 1;
        s.lo2 = g.rint_lo[e2];
        s.n2 = g.rint_hi[e2] - g.rint_lo[e2] + 1;
        s.off = fs.per_step;
        fs.per_step += (int64_t)s.n1 * s.n2;
      }
    }
  }
  return fs;
}

int64_t psi_bytes(const Geo& g) {
  int64_t t = 0;
  for (int d = 0; d < 3; ++d) t += 2 * psi_elems(g, d);  // two components per axis
  return t * (int64_t)sizeof(float);
}

int validate(const fdtd_grid* grid, double courant, const fdtd_pml* pml) {
  if (!grid || !pml) return fail(FDTD_ERR_INVALID_ARG, "grid and pml are required");
  const int n[3] = {grid->nx, grid->ny, grid->nz};
  for (int d = 0; d < 3; ++d)
    if (n[d] < 2 || n[d] > (1 << 16)) return fail(FDTD_ERR_INVALID_ARG, "grid size %d out of range [2, 65536]", n[d]);
  // the kernels index each field array with 32-bit offsets
  if ((int64_t)round_up(n[0], kPitchAlign) * n[1] * n[2] >= (int64_t(1) << 31))
    return fail(FDTD_ERR_INVALID_ARG, "grid of %d x %d x %d cells exceeds 2^31 cells per field array", n[0], n[1], n[2]);
  if (!(courant > 0.0)) return fail(FDTD_ERR_INVALID_ARG, "courant must be positive");
  if (courant > (1.0 / std::sqrt(3.0)) * (1.0 + 1e-12))
    return fail(FDTD_ERR_UNSTABLE, "courant %.9g exceeds the 3D stability limit 1/sqrt(3)", courant);
  for (int d = 0; d < 3; ++d) {
    const int p0 = pml->thickness[2 * d], p1 = pml->thickness[2 * d + 1];
    if (p0 < 0 || p1 < 0) return fail(FDTD_ERR_INVALID_ARG, "negative PML thickness");
    if (p0 + p1 > n[d] - 2) return fail(FDTD_ERR_INVALID_ARG, "PML thicker than the grid along axis %d", d);
  }
  if (pml->grading_m < 1 || pml->grading_m > 16) return fail(FDTD_ERR_INVALID_ARG, "grading_m out of range");
  if (!(pml->kappa_max >= 1.0) || !(pml->sigma_max >= 0.0) || !(pml->alpha_max >= 0.0))
    return fail(FDTD_ERR_INVALID_ARG, "PML parameters need kappa_max >= 1, sigma_max >= 0, alpha_max >= 0");
  return FDTD_OK;
}

struct Ev {
  cudaEvent_t a, b;
  int kind;
};

// A captured time loop, replayed while its shape and buffers stay the same.
struct LoopGraph {
  cudaGraphExec_t exec = nullptr;
  int nsteps = -1;
  int64_t key = -1;
  uint64_t gen = 0;
  std::vector<Ev> ev;      // timing events recorded by the graph (profiling only)
  int64_t launches = 0;    // kernels per replay
  int cur_after = 0;       // field buffer holding the state after the loop
  bool pending = false;    // a profiled replay whose events have not been read yet
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    for (auto& e : ev) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    ev.clear();
    nsteps = -1;
    key = -1;
    pending = false;
  }
};

}  // namespace

int fdtd::set_error(int code, const char* msg) {
  g_last_error = msg;
  return code;
}

bool fdtd::on_current_device(const void* p) {
  int dev = -1;
  cudaPointerAttributes at;
  if (!p || cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

struct fdtd_handle {
  Geo g{};
  fdtd_pml pml{};
  double spacing = 0, courant = 0;
  cudaStream_t stream = nullptr;  // caller's stream
  cudaStream_t cap = nullptr;     // private stream used only to capture the time loops
  cudaStream_t side = nullptr;    // captured beside `cap`: the face copies, off the critical path
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};  // fork / join points of `side`
  cudaStream_t side2 = nullptr;   // the frame launch of a split adjoint step, beside its plain launch
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
  bool adj_overlap = true;        // use side2 (FDTD_ADJ_OVERLAP=0: one stream)
  bool face_overlap = true;  // face copies on `side`, beside the stencil kernels (else in line on the stream)
  bool use_graphs = true;    // time loops captured into CUDA graphs (else launched directly)
  bool capturing = false;    // a time loop is being captured
  int32_t design_lo[3] = {0, 0, 0}, design_hi[3] = {0, 0, 0};
  FaceSet faces{};
  int tz = 8;                     // z-planes per block of the forward kernel
  int tz_rev = 8;                 // z-planes per block of the reverse kernels
  int rev_nstage = 4;             // stages of the reverse kernels' plane rings (checkpointing gradient)
  int fwd_nstage = 3;             // stages of the forward kernel's plane ring
  int tz_inv = 8, inv_nstage = 4; // fused inverse step: z-planes per block, ring stages
  int tz_adj = 8, adj_nstage = 4; // fused adjoint step
  // the fused adjoint step as two launches (x/y CPML frame, plain rectangle): see AdjArgs::split
  int adj_split = 0, adj_xl = 0, adj_xh = 0, adj_yl = 0, adj_yh = 0, tz_adj_xy = 8;
  // for grouped launches, whose z-chunks follow the group: column tiles of the 32 x 16 kernels
  // (forward, inverse, adjoint) and of the in-place pair, and resident-block slots of each kernel
  int64_t nxy_f = 1, nxy_r = 1;
  int64_t slots_fwd = 1, slots_rev = 1, slots_inv = 1, slots_adj = 1;
  bool tz_free = true;      // not pinned by FDTD_TZ
  bool fwd_tz_free = true;  // no flux detector summed by the fused forward (its slots follow tz)
  // reverse step kind: the fused inverse + adjoint kernels (52 + 52 B per cell, double-buffered
  // fields; faster on large grids with thin layers), or the in-place pair rev_E + rev_H (76 + 72 B per
  // cell, one cell per thread and more blocks per SM; faster on small grids and thick layers)
  bool rev_fused = false;

  std::vector<fdtd_source> src_host;
  std::vector<SrcDev> srcs;       // E sources: soft sources and the E corrections of TFSF planes
  std::vector<SrcDev> hsrcs;      // H corrections of TFSF planes (added to H^{n-1/2} before step n)
  std::vector<int> src_tfsf, hsrc_tfsf;  // per entry of srcs / hsrcs: its index in tfsf, or -1
  std::vector<Tfsf> tfsf;
  std::vector<DetDev> dets;
  std::vector<char> det_inline;   // per detector: sampled inside the fused forward kernel
  std::vector<char> det_fold;     // per detector: its adjoint added by rev_H of the following step
  std::vector<float*> det_slab;   // per detector: 3 slabs (E^{n+1}, H^{n+1/2}, E^n) for kind 4, else null
  int64_t det_total_per_step = 0, det_total_fixed = 0;

  // device memory
  float* fields = nullptr;     // 2 x 6 x vol: double-buffered (the fused kernels read cur, write 1 - cur)
  int cur = 0;
  float* a = nullptr;          // vol
  float* psiE = nullptr;       // CPML memories of E (compact slabs), double-buffered like the fields
  float* psiH = nullptr;
  float* tables = nullptr;     // 3 axes x 2 positions x (b, c, 1/kappa) x n
  float* init = nullptr;       // optional initial state, 6 x vol
  std::vector<float*> src_w;   // per source box weights
  float* gtab = nullptr;       // (srcs + hsrcs) x gtab_cap waveform samples
  int gtab_cap = 0;
  double* det_out = nullptr;   // concatenated detector outputs
  int64_t det_out_cap = 0;
  double* partial = nullptr;   // flux partial sums (scratch)
  int64_t partial_cap = 0;
  float* face_hist = nullptr;  // steps x faces.per_step (the steps from seg_first on)
  // face-history segments: with seg_steps = L > 0 a recorded forward of T steps keeps the faces of its
  // last segment only (steps from seg_first = (S - 1) L, S = ceil(T / L)) and full states (fields and
  // CPML memories) at the starts L, 2L, .., (S - 2) L of the others; the reverse sweep regenerates a
  // segment's faces by running its forward again from its start state
  int seg_steps = 0;
  int seg_first = 0;
  float* seg_states = nullptr;
  int64_t seg_cap = 0;
  int64_t face_cap_steps = 0;
  float* adj = nullptr;        // 2 x 6 x vol adjoint fields, double-buffered (the fused adjoint step reads
                               // one and writes the other; the checkpointing gradient uses buffer 0)
  float* psibar = nullptr;     // 2 buffers x (psi-bar E + psi-bar H)
  double* dLda = nullptr;      // design box
  double* dLddet = nullptr;    // device copy of dL/d(detectors)
  int64_t dLddet_cap = 0;
  float* staging = nullptr;    // 6 x N, unpitched
  int* status = nullptr;       // device status word written by the kernels (bounded waits)
  FwdMaps fmaps[2];            // TMA maps of the forward kernel reading field buffer 0 or 1
  RevMaps rmaps[2];            // TMA maps of the reverse kernels on field buffer 0 or 1 (and adj 0)
  InvMaps imaps[2];            // TMA maps of the fused inverse step reading field buffer 0 or 1
  AdjMaps amaps[2];            // TMA maps of the fused adjoint step reading adjoint buffer 0 or 1
  int64_t bytes = 0;
  uint64_t gen = 1;            // bumped whenever a buffer used by a captured loop is reallocated

  int last_nsteps = -1;
  // incremental solve advanced by fdtd_group_step (fdtd_begin ... fdtd_finish_backward)
  int phase = FDTD_PHASE_IDLE;
  int step_next = 0;           // forward: the next step to run; reverse: the next step to reverse
  bool solve_record = false;
  int rev_pc = 0, rev_ac = 0, rev_pb = 0;  // reverse: primal buffer, adjoint buffer, psi-bar set
  bool recorded = false;
  bool consumed = false;
  bool density = false;        // the design box was last set from a density rho
  double eps_lo = 0, eps_hi = 0;

  LoopGraph gfwd, gbwd;

  // launch accounting and sampled event timing
  int64_t launches = 0;
  int prof_every = 0;  // 0 = off
  int check_every = 0;  // non-finite field check every this many forward steps (0: at the end of a sweep only)
  bool canary = false;  // NaN canaries in the pitch padding of the field, adjoint and a arrays
  int nsm = 148;        // SMs of the device
  double prof_ms[FDTD_KERNEL_KINDS] = {0};
  int64_t prof_n[FDTD_KERNEL_KINDS] = {0};

  Tables tab() const {
    Tables T;
    int64_t off = 0;
    for (int d = 0; d < 3; ++d) {
      const int n = g.n[d];
      for (int h = 0; h < 2; ++h) {
        T.b[d][h] = tables + off;
        off += n;
        T.c[d][h] = tables + off;
        off += n;
        T.ik[d][h] = tables + off;
        off += n;
      }
    }
    for (int d = 0; d < 3; ++d) {
      T.sidx[d] = reinterpret_cast<const int*>(tables + off);
      off += g.n[d];
    }
    return T;
  }
  Fields F(int b) const {
    Fields f;
    for (int c = 0; c < 6; ++c) f.f[c] = fields + (int64_t)b * 6 * g.vol + c * g.vol;
    return f;
  }
  Fields F() const { return F(cur); }
  Fields A(int b = 0) const {
    Fields f;
    for (int c = 0; c < 6; ++c) f.f[c] = adj + (int64_t)b * 6 * g.vol + c * g.vol;
    return f;
  }
  // psi pointers over a buffer laid out axis by axis, two components per axis
  PsiSet psi_set(float* base) const {
    PsiSet P;
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) P.p[c][d] = nullptr;
    int64_t off = 0;
    for (int d = 0; d < 3; ++d) {
      const int64_t n = psi_elems(g, d);
      for (int c = 0; c < 3; ++c) {
        if (c == d) continue;
        P.p[c][d] = (n > 0) ? base + off : nullptr;
        off += n;
      }
    }
    return P;
  }
  int64_t psi_floats() const { return psi_bytes(g) / (int64_t)sizeof(float); }
  int64_t state_floats() const { return 6 * g.vol + 2 * psi_floats(); }
  float* face_at(int n) const { return face_hist + (int64_t)(n - seg_first) * faces.per_step; }
  int segments(int nsteps) const { return seg_steps > 0 ? (nsteps + seg_steps - 1) / seg_steps : 1; }
};

namespace {

// Brackets every `every`-th launch of kernel `kind` with events recorded into `evs` (profiling only).
struct ProfScope {
  std::vector<Ev>* evs;
  cudaStream_t st;
  int idx = -1;
  ProfScope(fdtd_handle* h, std::vector<Ev>* evs_, cudaStream_t st_, int kind, int step) : evs(evs_), st(st_) {
    if (!evs || h->prof_every <= 0 || step % h->prof_every != 0) return;
    Ev e;
    if (cudaEventCreate(&e.a) != cudaSuccess) return;
    if (cudaEventCreate(&e.b) != cudaSuccess) {
      cudaEventDestroy(e.a);
      return;
    }
    e.kind = kind;
    evs->push_back(e);
    idx = (int)evs->size() - 1;
    ext = h->capturing;
    record((*evs)[idx].a);
  }
  ~ProfScope() {
    if (idx >= 0) record((*evs)[idx].b);
  }
  bool ext = false;  // inside a capture: the event becomes an event-record node of the graph
  void record(cudaEvent_t e) const {
    if (ext) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
  }
};

int dev_alloc(fdtd_handle* h, void** p, int64_t bytes) {
  *p = nullptr;
  if (bytes <= 0) return FDTD_OK;
  if (g_byte_budget >= 0 && h->bytes + bytes > g_byte_budget)
    return fail(FDTD_ERR_OOM, "byte budget %lld exceeded (%lld held, %lld requested)", (long long)g_byte_budget,
                (long long)h->bytes, (long long)bytes);
  // stream-ordered: no device-wide synchronisation, so handles can come and go while others run
  cudaError_t e = cudaMallocAsync(p, (size_t)bytes, h->stream);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(FDTD_ERR_OOM, "cudaMallocAsync of %lld bytes failed", (long long)bytes);
  }
  if (e != cudaSuccess) return fail(FDTD_ERR_CUDA, "cudaMallocAsync: %s", cudaGetErrorString(e));
  h->bytes += bytes;
  h->gen += 1;
  return FDTD_OK;
}

void dev_free(fdtd_handle* h, void* p, int64_t bytes) {
  if (p) {
    cudaFreeAsync(p, h->stream);
    h->bytes -= bytes;
    h->gen += 1;
  }
}

// (Re)allocate *p to hold at least `need` elements of `esize` bytes, tracking the capacity.
template <class T>
int ensure_buf(fdtd_handle* h, T** p, int64_t* cap, int64_t need, int64_t esize) {
  if (need <= *cap) return FDTD_OK;
  if (*p) CK(cudaStreamSynchronize(h->stream));  // (a first allocation waits for nothing)
  dev_free(h, *p, *cap * esize);
  *p = nullptr;
  *cap = 0;
  TRY(dev_alloc(h, (void**)p, need * esize));
  *cap = need;
  return FDTD_OK;
}

int upload_tables(fdtd_handle* h) {
  const Geo& g = h->g;
  std::vector<float> host;
  for (int d = 0; d < 3; ++d) {
    const int n = g.n[d];
    for (int half = 0; half < 2; ++half) {
      std::vector<float> b(n), c(n), ik(n);
      for (int i = 0; i < n; ++i) {
        double bb, cc, kk;
        cpml_coef(half ? i + 0.5 : (double)i, n, g.pml[2 * d], g.pml[2 * d + 1], h->pml, bb, cc, kk);
        b[i] = (float)bb;
        c[i] = (float)cc;
        ik[i] = (float)kk;
      }
      host.insert(host.end(), b.begin(), b.end());
      host.insert(host.end(), c.begin(), c.end());
      host.insert(host.end(), ik.begin(), ik.end());
    }
  }
  for (int d = 0; d < 3; ++d)  // slab index tables, stored as int bit patterns after the float tables
    for (int i = 0; i < g.n[d]; ++i) {
      const int si = slab_index(g, d, i);
      float f;
      std::memcpy(&f, &si, 4);
      host.push_back(f);
    }
  TRY(dev_alloc(h, (void**)&h->tables, (int64_t)host.size() * 4));
  CK(cudaMemcpyAsync(h->tables, host.data(), host.size() * 4, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));  // `host` dies on return
  return FDTD_OK;
}

// Waveform tables of every source entry for steps 0..nsteps-1 (rows: srcs, then hsrcs): g(n + 1/2)
// for a soft source; for a TFSF plane the incident H^{n+1/2} (its E correction) and E^n (its H
// correction). A table built for more steps serves fewer (the incident line is causal).
int ensure_gtab(fdtd_handle* h, int nsteps) {
  const int ns = (int)h->srcs.size(), nh = (int)h->hsrcs.size(), nr = ns + nh;
  if (nr == 0) return FDTD_OK;
  if (h->gtab_cap < nsteps) {
    CK(cudaStreamSynchronize(h->stream));
    dev_free(h, h->gtab, (int64_t)nr * h->gtab_cap * 4);
    h->gtab = nullptr;
    h->gtab_cap = 0;
    TRY(dev_alloc(h, (void**)&h->gtab, (int64_t)nr * nsteps * 4));
    std::vector<std::vector<double>> einc(h->tfsf.size()), hinc(h->tfsf.size());
    for (size_t t = 0; t < h->tfsf.size(); ++t) tfsf_incident(h->tfsf[t], h->courant, nsteps, einc[t], hinc[t]);
    std::vector<float> t((size_t)nr * nsteps);
    for (int q = 0; q < ns; ++q)
      for (int n = 0; n < nsteps; ++n)
        t[(size_t)q * nsteps + n] = h->src_tfsf[q] < 0 ? (float)pulse(h->src_host[q], h->courant, n + 0.5)
                                                       : (float)hinc[h->src_tfsf[q]][n];
    for (int q = 0; q < nh; ++q)
      for (int n = 0; n < nsteps; ++n) t[(size_t)(ns + q) * nsteps + n] = (float)einc[h->hsrc_tfsf[q]][n];
    CK(cudaMemcpyAsync(h->gtab, t.data(), t.size() * 4, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));  // `t` dies on return
    h->gtab_cap = nsteps;
  }
  for (int q = 0; q < ns; ++q) h->srcs[q].g = h->gtab + (size_t)q * h->gtab_cap;
  for (int q = 0; q < nh; ++q) h->hsrcs[q].g = h->gtab + (size_t)(ns + q) * h->gtab_cap;
  return FDTD_OK;
}

int64_t det_total_for(const fdtd_handle* h, int nsteps) {
  return h->det_total_fixed + h->det_total_per_step * (int64_t)nsteps;
}

int ensure_det(fdtd_handle* h, int nsteps) {
  const int64_t need = det_total_for(h, nsteps);
  TRY(ensure_buf(h, &h->det_out, &h->det_out_cap, need, 8));
  int64_t off = 0, pneed = 0;
  for (auto& d : h->dets) {
    d.off = off;
    const bool per_cell = d.kind == FDTD_DET_PLANE_E2_SUM || d.kind == FDTD_DET_PLANE_E2_SUM_INTERP;
    off += per_cell ? box_cells(d.lo, d.hi) : nsteps;
    if (d.kind == FDTD_DET_PLANE_FLUX || d.kind == FDTD_DET_PLANE_FLUX_INTERP) {
      d.poff = pneed;
      pneed += (int64_t)d.nblk * nsteps;
    }
  }
  TRY(ensure_buf(h, &h->partial, &h->partial_cap, pneed, 8));
  if (need > 0) CK(cudaMemsetAsync(h->det_out, 0, need * 8, h->stream));
  return FDTD_OK;
}

// NaN canaries in the pitch padding of both field buffers, the adjoint fields and a (canary mode).
// For odd nx the forward kernel, which stores x-adjacent cell pairs, writes zeros into column nx of
// the field arrays (never read: the tensor maps end at nx), so their canaries start one column later.
int field_canary_x0(const fdtd_handle* h) { return h->g.n[0] + (h->g.n[0] & 1); }

void fill_canaries(fdtd_handle* h, bool fields, bool adj, bool a) {
  if (!h->canary) return;
  const int64_t rows = (int64_t)h->g.n[1] * h->g.n[2];
  const float nan = std::numeric_limits<float>::quiet_NaN();
  if (fields) launch_fill_padding(h->g, h->fields, 12 * rows, field_canary_x0(h), nan, h->nsm, h->stream);
  if (adj && h->adj) launch_fill_padding(h->g, h->adj, 12 * rows, h->g.n[0], nan, h->nsm, h->stream);
  if (a) launch_fill_padding(h->g, h->a, rows, h->g.n[0], nan, h->nsm, h->stream);
}

int reset_state(fdtd_handle* h) {
  h->cur = 0;
  if (h->init) CK(cudaMemcpyAsync(h->fields, h->init, 6 * h->g.vol * 4, cudaMemcpyDeviceToDevice, h->stream));
  else CK(cudaMemsetAsync(h->fields, 0, 6 * h->g.vol * 4, h->stream));
  fill_canaries(h, true, false, false);
  const int64_t pf = h->psi_floats();
  if (pf > 0) {
    CK(cudaMemsetAsync(h->psiE, 0, 2 * pf * 4, h->stream));
    CK(cudaMemsetAsync(h->psiH, 0, 2 * pf * 4, h->stream));
  }
  return FDTD_OK;
}

bool in_r_cells(const fdtd_handle* h, const int32_t lo[3], const int32_t hi[3]) {
  for (int d = 0; d < 3; ++d) {
    if (lo[d] == hi[d]) continue;
    if (lo[d] < h->g.pml[2 * d] || hi[d] > h->g.n[d] - h->g.pml[2 * d + 1]) return false;
  }
  return true;
}

int ensure_staging(fdtd_handle* h) {
  if (!h->staging) {
    const int64_t N = (int64_t)h->g.n[0] * h->g.n[1] * h->g.n[2];
    TRY(dev_alloc(h, (void**)&h->staging, 6 * N * 4));
  }
  return FDTD_OK;
}

bool is_host_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged;
}

// Both adjoint buffers, with the TMA maps of the kernels that read them: the fused adjoint step (either
// buffer) and the reverse kernels of the checkpointing gradient (buffer 0).
int encode_rev_maps(fdtd_handle* h);
int ensure_adjoint(fdtd_handle* h) {
  if (h->adj) return FDTD_OK;
  const Geo& g = h->g;
  TRY(dev_alloc(h, (void**)&h->adj, 12 * g.vol * 4));
  TRY(encode_rev_maps(h));
  for (int b = 0; b < 2; ++b) {
    const Fields Ab = h->A(b);
    TRY(encode_field_map(&h->amaps[b].eb, Ab.f[0], g, 3, adj_box_e()));
    TRY(encode_field_map(&h->amaps[b].hb, Ab.f[3], g, 3, adj_box_h()));
    TRY(encode_field_map(&h->amaps[b].a, h->a, g, 1, adj_box_e()));
  }
  return FDTD_OK;
}

// TMA maps of the reverse kernels (fdtd_reverse.cu): over each field buffer and the adjoint fields.
int encode_rev_maps(fdtd_handle* h) {
  const Geo& g = h->g;
  const MapBox own = rev_box_own(), wide = rev_box_wide();
  const Fields B = h->A();
  for (int b = 0; b < 2; ++b) {
    const Fields Fb = h->F(b);
    RevMaps& m = h->rmaps[b];
    TRY(encode_field_map(&m.e_own, Fb.f[0], g, 3, own));
    TRY(encode_field_map(&m.e_high, Fb.f[0], g, 3, wide));
    TRY(encode_field_map(&m.h_own, Fb.f[3], g, 3, own));
    TRY(encode_field_map(&m.h_low, Fb.f[3], g, 3, wide));
    TRY(encode_field_map(&m.eb_own, B.f[0], g, 3, own));
    TRY(encode_field_map(&m.eb_high, B.f[0], g, 3, wide));
    TRY(encode_field_map(&m.hb_own, B.f[3], g, 3, own));
    TRY(encode_field_map(&m.hb_low, B.f[3], g, 3, wide));
    TRY(encode_field_map(&m.a_high, h->a, g, 1, wide));
  }
  return FDTD_OK;
}

// ---- the time loops -------------------------------------------------------------------------------

// Detector adjoints of reverse step n, part 0 (start of the step: every detector's terms through the
// state after step n; the interpolated flux first copies E^{n+1} and H^{n+1/2} into its slabs),
// part 1 (after rev_E: the interpolated flux's H terms, with E^n copied from the rebuilt fields, or
// already in its slab when `e0_ready`) and part 2 (after rev_H: the interpolated flux's E^n terms).
// With `folded`, part 0 skips the detectors whose adjoint rev_H of step n+1 has already added.
int64_t enqueue_det_adjoint(fdtd_handle* h, const Fields& F, const Fields& A, int n, int part, cudaStream_t st,
                            bool e0_ready = false, bool folded = false) {
  const Geo& g = h->g;
  int64_t launches = 0;
  for (size_t q = 0; q < h->dets.size(); ++q) {
    const DetDev& d = h->dets[q];
    if (folded && h->det_fold[q]) continue;
    float* sl = h->det_slab[q];
    const int64_t sf = sl ? interp_slab_floats(d) : 0;
    float *sE1 = sl, *sH = sl + sf, *sE0 = sl + 2 * sf;
    if (d.kind <= FDTD_DET_PLANE_FLUX) {
      if (part == 0) {
        launch_detector_adjoint(g, F, A, d, n, h->dLddet, st);
        ++launches;
      }
    } else if (d.kind == FDTD_DET_PLANE_E2_SUM_INTERP) {
      if (part == 0) {
        launch_interp_adjoint(g, F, A, d, n, h->dLddet, 0, nullptr, nullptr, nullptr, st);
        ++launches;
      }
    } else {
      if (part == 0) {
        launch_slab_copy(g, F, d, 0, sE1, st);
        launch_slab_copy(g, F, d, 3, sH, st);
        launches += 2;
      } else if (part == 1 && !e0_ready) {
        launch_slab_copy(g, F, d, 0, sE0, st);
        ++launches;
      }
      launch_interp_adjoint(g, F, A, d, n, h->dLddet, part, sE0, sE1, sH, st);
      ++launches;
    }
  }
  return launches;
}


// ---- one forward step, in pieces shared by the solo time loop and the grouped launches --------------

// The arguments of the fused forward kernel that do not change from step to step.
FwdArgs fwd_base(fdtd_handle* h) {
  FwdArgs fa;
  fa.g = h->g;
  fa.T = h->tab();
  fa.a = h->a;
  fa.tz = h->tz;
  fa.nstage = h->fwd_nstage;
  fa.nsrc = (int)std::min<size_t>(h->srcs.size(), kMaxSrc);
  for (int q = 0; q < fa.nsrc; ++q) fa.src[q] = h->srcs[q];
  fa.ndet = 0;
  for (size_t q = 0; q < h->dets.size(); ++q)
    if (h->det_inline[q]) fa.det[fa.ndet++] = h->dets[q];
  fa.det_out = h->det_out;
  fa.partial = h->partial;
  fa.status = h->status;
  return fa;
}

// The buffers and step index of step n (reading field buffer h->cur).
void fwd_step_args(fdtd_handle* h, FwdArgs& fa, int n) {
  const int64_t pf = h->psi_floats();
  const int c = h->cur, x = 1 - c;
  fa.cur = h->F(c);
  fa.nxt = h->F(x);
  fa.psiE_cur = h->psi_set(h->psiE + c * pf);
  fa.psiE_nxt = h->psi_set(h->psiE + x * pf);
  fa.psiH_cur = h->psi_set(h->psiH + c * pf);
  fa.psiH_nxt = h->psi_set(h->psiH + x * pf);
  fa.step = n;
}

// Before the fused kernel of step n: the TFSF H corrections of the step, added to H^{n-1/2} so that
// the fused kernel's H update yields H^{n-1/2} - S curl E^n + correction in every cell, halos included.
int64_t fwd_step_pre(fdtd_handle* h, int n, cudaStream_t st) {
  for (const SrcDev& hs : h->hsrcs) launch_source(h->g, h->F(h->cur), hs, n, +1.f, 0, st);
  return (int64_t)h->hsrcs.size();
}

// After the fused kernel of step n (its output in buffer 1 - h->cur) and the face record: the sources
// and detectors beyond the fused kernel's slots, and the non-finite check (periodic and at the end).
int64_t fwd_step_post(fdtd_handle* h, int n, int nsteps, cudaStream_t st) {
  const Geo& g = h->g;
  const Fields Fn = h->F(1 - h->cur);
  int64_t launches = 0;
  for (size_t q = kMaxSrc; q < h->srcs.size(); ++q, ++launches) launch_source(g, Fn, h->srcs[q], n, +1.f, 0, st);
  for (size_t q = 0; q < h->dets.size(); ++q) {
    if (h->det_inline[q]) continue;
    const DetDev& d = h->dets[q];
    if (d.kind <= FDTD_DET_PLANE_FLUX) launch_detector_sample(g, Fn, d, n, h->det_out, h->partial, st);
    else launch_detector_interp(g, h->F(h->cur), Fn, d, n, h->det_out, h->partial, st);  // E^n is in cur
    ++launches;
  }
  if (n == nsteps - 1 || (h->check_every > 0 && (n + 1) % h->check_every == 0)) {
    launch_check_finite(g, Fn.f[0], 6 * g.vol, h->status, h->nsm, st);
    ++launches;
  }
  return launches;
}

// After the last forward step: the fixed-order sums of the flux detectors.
int64_t fwd_finish(fdtd_handle* h, int nsteps, cudaStream_t st) {
  int64_t launches = 0;
  for (const auto& d : h->dets)
    if ((d.kind == FDTD_DET_PLANE_FLUX || d.kind == FDTD_DET_PLANE_FLUX_INTERP) && nsteps > 0) {
      launch_flux_finalize(d, nsteps, h->partial, h->det_out, st);
      launches += 1;
    }
  return launches;
}

// The state at the start of segment s (time s L: fields of the current buffer and its CPML memories)
// into its slot.
void save_segment_state(fdtd_handle* h, int s, cudaStream_t st) {
  const int64_t pf = h->psi_floats(), V = 6 * h->g.vol;
  float* slot = h->seg_states + (int64_t)(s - 1) * h->state_floats();
  const int c = h->cur;
  cudaMemcpyAsync(slot, h->fields + (int64_t)c * V, V * 4, cudaMemcpyDeviceToDevice, st);
  if (pf > 0) {
    cudaMemcpyAsync(slot + V, h->psiE + c * pf, pf * 4, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(slot + V + pf, h->psiH + c * pf, pf * 4, cudaMemcpyDeviceToDevice, st);
  }
}

// Regenerate the faces of segment s for the reverse sweep: its start state (the initial state for
// s = 0, else the saved one) into field buffer b = pn ^ (L & 1), then its L forward steps with the face
// record and without detectors, which ends with the exact forward state at time (s + 1) L in buffer
// pn. Returns the launches.
int64_t regen_segment(fdtd_handle* h, int s, int pn, cudaStream_t st) {
  const Geo& g = h->g;
  const int L = h->seg_steps;
  const int64_t pf = h->psi_floats(), V = 6 * g.vol;
  const int b = pn ^ (L & 1);
  if (s == 0) {
    if (h->init) cudaMemcpyAsync(h->fields + (int64_t)b * V, h->init, V * 4, cudaMemcpyDeviceToDevice, st);
    else cudaMemsetAsync(h->fields + (int64_t)b * V, 0, V * 4, st);
    if (pf > 0) {
      cudaMemsetAsync(h->psiE + b * pf, 0, pf * 4, st);
      cudaMemsetAsync(h->psiH + b * pf, 0, pf * 4, st);
    }
  } else {
    const float* slot = h->seg_states + (int64_t)(s - 1) * h->state_floats();
    cudaMemcpyAsync(h->fields + (int64_t)b * V, slot, V * 4, cudaMemcpyDeviceToDevice, st);
    if (pf > 0) {
      cudaMemcpyAsync(h->psiE + b * pf, slot + V, pf * 4, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(h->psiH + b * pf, slot + V + pf, pf * 4, cudaMemcpyDeviceToDevice, st);
    }
  }
  h->seg_first = s * L;
  const int keep = h->cur;
  h->cur = b;
  FwdArgs fa = fwd_base(h);
  fa.ndet = 0;  // the detectors were sampled by the original forward
  int64_t launches = 0;
  for (int n = s * L; n < (s + 1) * L; ++n) {
    const int c = h->cur;
    fwd_step_args(h, fa, n);
    launches += fwd_step_pre(h, n, st);
    launch_fwd_fused(fa, h->fmaps[c], st);
    launch_face_copy(g, h->F(1 - c), h->faces, h->face_at(n), 1, st);
    for (size_t q = kMaxSrc; q < h->srcs.size(); ++q, ++launches)
      launch_source(g, h->F(1 - c), h->srcs[q], n, +1.f, 0, st);
    launches += 2;
    h->cur = 1 - c;
  }
  h->cur = keep;
  return launches;
}

// Forward: one fused launch per step (plus extra launches for sources and detectors beyond the
// fused kernel's slots), then the fixed-order flux sums. Mutates h->cur as it goes.
int64_t enqueue_forward(fdtd_handle* h, int nsteps, bool record, cudaStream_t st, std::vector<Ev>* evs) {
  const Geo& g = h->g;
  const bool faces = record && h->faces.per_step > 0;
  int64_t launches = 0;
  FwdArgs fa = fwd_base(h);
  // The face record of step n runs on the side stream, beside step n+1 (which only reads that
  // buffer); step n+2 overwrites it, so its fused kernel waits for the copy, and so does a TFSF H
  // correction of step n+1, which writes that buffer's H. Without face_overlap (or with segments, whose
  // first steps record no faces) it runs in line.
  const bool ovl = faces && h->face_overlap && h->seg_steps == 0;
  for (int n = 0; n < nsteps; ++n) {
    const int c = h->cur, x = 1 - c;
    if (ovl && n >= 2) cudaStreamWaitEvent(st, h->ev_join[n % 2], 0);
    if (ovl && n >= 1 && !h->hsrcs.empty()) cudaStreamWaitEvent(st, h->ev_join[(n - 1) % 2], 0);
    fwd_step_args(h, fa, n);
    launches += fwd_step_pre(h, n, st);
    {
      ProfScope ps(h, evs, st, FDTD_KERNEL_FUSED_FWD, n);
      launch_fwd_fused(fa, h->fmaps[c], st);
    }
    launches += 1;
    if (faces && n >= h->seg_first) {  // H^{n+1/2} on the boundary faces
      cudaStream_t fs = ovl ? h->side : st;
      if (ovl) {
        cudaEventRecord(h->ev_fork, st);
        cudaStreamWaitEvent(h->side, h->ev_fork, 0);
      }
      {
        ProfScope ps(h, evs, fs, FDTD_KERNEL_FACE_COPY, n);
        launch_face_copy(g, h->F(x), h->faces, h->face_at(n), 1, fs);
      }
      if (ovl) cudaEventRecord(h->ev_join[n % 2], h->side);
      launches += 1;
    }
    launches += fwd_step_post(h, n, nsteps, st);
    h->cur = x;
    if (faces && h->seg_steps > 0 && (n + 1) % h->seg_steps == 0 && (n + 1) / h->seg_steps <= h->segments(nsteps) - 2)
      save_segment_state(h, (n + 1) / h->seg_steps, st);
  }
  if (ovl) {  // join the side stream
    if (nsteps >= 2) cudaStreamWaitEvent(st, h->ev_join[(nsteps - 2) % 2], 0);
    if (nsteps >= 1) cudaStreamWaitEvent(st, h->ev_join[(nsteps - 1) % 2], 0);
  }
  launches += fwd_finish(h, nsteps, st);
  return launches;
}

// ---- one reverse step, in pieces shared by the solo time loop and the grouped launches --------------
// Reverse step n starts from the state after step n: E^{n+1}, H^{n+1/2} in field buffer pc and the
// adjoint of that state in adjoint buffer ac; psi-bar memories read from set pb.

PsiSet psibar_set(const fdtd_handle* h, int which, int pb) {  // which 0: of E, 1: of H
  return h->psi_set(h->psibar + (2 * pb + which) * h->psi_floats());
}

InvArgs inv_base(fdtd_handle* h) {
  InvArgs ia;
  ia.g = h->g;
  ia.a = h->a;
  ia.tz = h->tz_inv;
  ia.nstage = h->inv_nstage;
  ia.nsrc = (int)std::min<size_t>(h->srcs.size(), kMaxSrc);
  for (int q = 0; q < ia.nsrc; ++q) ia.src[q] = h->srcs[q];
  for (int d = 0; d < 3; ++d) {
    ia.dlo[d] = h->design_lo[d];
    ia.dhi[d] = h->design_hi[d];
  }
  ia.dLda = box_cells(h->design_lo, h->design_hi) > 0 ? h->dLda : nullptr;
  ia.status = h->status;
  return ia;
}

void inv_step_args(fdtd_handle* h, InvArgs& ia, int n, int pc, int ac) {
  ia.cur = h->F(pc);
  ia.nxt = h->F(1 - pc);
  ia.step = n;
  const Fields Ac = h->A(ac);
  for (int c = 0; c < 3; ++c) ia.eb[c] = Ac.f[c];
}

AdjArgs adj_base(fdtd_handle* h) {
  AdjArgs aa;
  aa.g = h->g;
  aa.T = h->tab();
  aa.a = h->a;
  aa.tz = h->tz_adj;
  aa.nstage = h->adj_nstage;
  aa.split = h->adj_split;
  aa.xl = h->adj_xl;
  aa.xh = h->adj_xh;
  aa.yl = h->adj_yl;
  aa.yh = h->adj_yh;
  aa.tz_xy = h->tz_adj_xy;
  aa.status = h->status;
  aa.gy = h->dLddet;
  aa.ndet = 0;
  for (size_t q = 0; q < h->dets.size(); ++q)
    if (h->det_fold[q]) {
      DetDev d = h->dets[q];
      if (d.kind == FDTD_DET_POINT_SERIES)  // the point is the one-cell box at lo
        for (int k = 0; k < 3; ++k) d.hi[k] = d.lo[k] + 1;
      aa.det[aa.ndet++] = d;
    }
  return aa;
}

void adj_step_args(fdtd_handle* h, AdjArgs& aa, int n, int pc, int ac, int pb) {
  aa.cur = h->A(ac);
  aa.nxt = h->A(1 - ac);
  aa.prim = h->F(1 - pc);
  aa.pinE = psibar_set(h, 0, pb);
  aa.poutE = psibar_set(h, 0, 1 - pb);
  aa.pinH = psibar_set(h, 1, pb);
  aa.poutH = psibar_set(h, 1, 1 - pb);
  aa.det_step = n - 1;  // -1 at n = 0: nothing left to fold
}

// Before the inverse step of n: the detector adjoints of step n that need a launch of their own (all of
// them at the last step, whose folded adjoints no later adjoint step has added), and the sources beyond
// the inverse kernel's slots taken off E^{n+1} on R.
int64_t rev_step_pre(fdtd_handle* h, int n, int nsteps, int pc, int ac, cudaStream_t st, std::vector<Ev>* evs) {
  const Fields Fc = h->F(pc), Ac = h->A(ac);
  bool unfolded = false;
  int nfold = 0;
  for (size_t q = 0; q < h->dets.size(); ++q) {
    unfolded |= !h->det_fold[q];
    nfold += h->det_fold[q];
  }
  const bool folded = n < nsteps - 1;
  int64_t launches = 0;
  if (unfolded || (!folded && nfold > 0)) {
    ProfScope ps(h, evs, st, FDTD_KERNEL_DET_ADJ, n);
    launches += enqueue_det_adjoint(h, Fc, Ac, n, 0, st, false, folded);
  }
  for (size_t q = kMaxSrc; q < h->srcs.size(); ++q, ++launches) launch_source(h->g, Fc, h->srcs[q], n, -1.f, 1, st);
  return launches;
}

// Between the inverse and the adjoint half of the step: the interpolated fluxes' H terms (E^n now in
// field buffer pn) into adjoint buffer ac.
int64_t rev_step_mid(fdtd_handle* h, int n, int pn, int ac, cudaStream_t st) {
  return enqueue_det_adjoint(h, h->F(pn), h->A(ac), n, 1, st);
}

// After the step (rebuilt fields in buffer pn, adjoint in an): the TFSF H corrections of step n
// removed from the rebuilt H^{n-1/2} on R, and the interpolated fluxes' E^n terms.
int64_t rev_step_post(fdtd_handle* h, int n, int pn, int an, cudaStream_t st) {
  const Fields Fn = h->F(pn);
  for (const SrcDev& hs : h->hsrcs) launch_source(h->g, Fn, hs, n, -1.f, 1, st);
  return (int64_t)h->hsrcs.size() + enqueue_det_adjoint(h, Fn, h->A(an), n, 2, st);
}

// The in-place pair: arguments of rev_E (which = 0) or rev_H (which = 1) of step n on field buffer pc
// and adjoint buffer 0.
RevArgs split_base(fdtd_handle* h) {
  RevArgs ra;
  ra.g = h->g;
  ra.T = h->tab();
  ra.B = h->A(0);
  ra.a = h->a;
  ra.tz = h->tz_rev;
  ra.nstage = h->rev_nstage;
  for (int d = 0; d < 3; ++d) {
    ra.dlo[d] = h->design_lo[d];
    ra.dhi[d] = h->design_hi[d];
  }
  ra.dLda = h->dLda;
  ra.inverse = 1;
  ra.nsrc = (int)std::min<size_t>(h->srcs.size(), kMaxSrc);
  for (int q = 0; q < ra.nsrc; ++q) ra.src[q] = h->srcs[q];
  ra.status = h->status;
  ra.gy = h->dLddet;
  ra.ndet = 0;
  for (size_t q = 0; q < h->dets.size(); ++q)
    if (h->det_fold[q]) {
      DetDev d = h->dets[q];
      if (d.kind == FDTD_DET_POINT_SERIES)  // the point is the one-cell box at lo
        for (int k = 0; k < 3; ++k) d.hi[k] = d.lo[k] + 1;
      ra.det[ra.ndet++] = d;
    }
  return ra;
}

void split_step_args(fdtd_handle* h, RevArgs& ra, int n, int pc, int pb, int which) {
  ra.F = h->F(pc);
  ra.step = n;
  ra.pin = psibar_set(h, which, pb);
  ra.pout = psibar_set(h, which, 1 - pb);
  ra.det_step = which == 1 ? n - 1 : -1;  // rev_H folds the E-only detectors of step n - 1
}

// After the last reverse step: the non-finite check of the rebuilt and the adjoint fields.
int64_t rev_finish(fdtd_handle* h, int pc, int ac, cudaStream_t st) {
  launch_check_finite(h->g, h->F(pc).f[0], 6 * h->g.vol, h->status, h->nsm, st);
  launch_check_finite(h->g, h->A(ac).f[0], 6 * h->g.vol, h->status, h->nsm, st);
  return 2;
}

// Reverse (Sec. 2.2), per step n:
//   the detector adjoints of step n that need a launch of their own;
//   the recorded H^{n+1/2} written back on the boundary faces (just outside R) of buffer pc;
//   the fused inverse step: E^n, H^{n-1/2} on R into buffer 1 - pc, and dL/da on the design box;
//   the fused adjoint step: the adjoint of (E^n, H^{n-1/2}) into adjoint buffer 1 - ac, plus the
//   adjoints of the E-only detectors of step n - 1 (from E^n in buffer 1 - pc);
//   the TFSF H corrections of step n removed from H^{n-1/2} on R.
int64_t enqueue_backward(fdtd_handle* h, int nsteps, cudaStream_t st, std::vector<Ev>* evs) {
  const Geo& g = h->g;
  InvArgs ia = inv_base(h);
  AdjArgs aa = adj_base(h);
  int64_t launches = 0;
  int pc = h->cur, ac = 0, pb = 0;
  // The face replay of step n (the recorded H^{n+1/2} written back outside R into buffer pc) runs on
  // the side stream beside the adjoint step of n + 1, which does not touch the primal fields; the
  // inverse step of n waits for it. Without face_overlap (or with segments) it runs in line.
  const bool faces = h->faces.per_step > 0;
  const bool ovl = faces && h->face_overlap && h->seg_steps == 0;
  auto replay = [&](int n, int buf) {
    cudaStream_t fs = ovl ? h->side : st;
    if (ovl) cudaStreamWaitEvent(h->side, h->ev_fork, 0);
    {
      ProfScope ps(h, evs, fs, FDTD_KERNEL_FACE_COPY, n);
      launch_face_copy(g, h->F(buf), h->faces, h->face_at(n), 0, fs);
    }
    if (ovl) cudaEventRecord(h->ev_join[n % 2], h->side);
    launches += 1;
  };
  if (ovl && nsteps > 0) {
    cudaEventRecord(h->ev_fork, st);
    replay(nsteps - 1, pc);
  }
  for (int n = nsteps - 1; n >= 0; --n) {
    if (faces && n < h->seg_first) launches += regen_segment(h, n / h->seg_steps, pc, st);
    launches += rev_step_pre(h, n, nsteps, pc, ac, st, evs);
    if (ovl) cudaStreamWaitEvent(st, h->ev_join[n % 2], 0);  // H^{n+1/2} on the faces is in place
    else if (faces) replay(n, pc);
    {
      ProfScope ps(h, evs, st, FDTD_KERNEL_INV_FUSED, n);
      inv_step_args(h, ia, n, pc, ac);
      launch_inv(ia, h->imaps[pc], st);
    }
    if (ovl && n > 0) {  // the faces of step n - 1 go into buffer 1 - pc, which the inverse step has written
      cudaEventRecord(h->ev_fork, st);
      replay(n - 1, 1 - pc);
    }
    launches += rev_step_mid(h, n, 1 - pc, ac, st);
    {
      ProfScope ps(h, evs, st, FDTD_KERNEL_ADJ_FUSED, n);
      adj_step_args(h, aa, n, pc, ac, pb);
      launches += h->adj_overlap ? launch_adj(aa, h->amaps[ac], st, h->side2, h->ev_fork2, h->ev_join2)
                                 : launch_adj(aa, h->amaps[ac], st);
    }
    launches += 1;
    launches += rev_step_post(h, n, 1 - pc, 1 - ac, st);
    pc = 1 - pc;
    ac = 1 - ac;
    pb = 1 - pb;
  }
  h->cur = pc;
  if (nsteps > 0) launches += rev_finish(h, pc, ac, st);
  return launches;
}

// The same reverse sweep with the in-place pair rev_E + rev_H: per step n the detector adjoints, the
// face replay into H, rev_E (inverse E, adjoint H-bar, dL/da) and rev_H (inverse H, adjoint E-bar, the
// folded detector adjoints of step n - 1), on field buffer h->cur and adjoint buffer 0.
int64_t enqueue_backward_split(fdtd_handle* h, int nsteps, cudaStream_t st, std::vector<Ev>* evs) {
  const Geo& g = h->g;
  RevArgs ra = split_base(h);
  const int pc = h->cur;
  const RevMaps& rm = h->rmaps[pc];
  int64_t launches = 0;
  int pb = 0;
  // The face replay of step n runs on the side stream beside rev_H(n+1), which neither reads nor
  // writes H outside R; rev_E(n) waits for it. Without face_overlap it runs in line.
  const bool faces = h->faces.per_step > 0;
  const bool ovl = faces && h->face_overlap && h->seg_steps == 0;
  auto replay = [&](int n) {
    cudaStream_t fs = ovl ? h->side : st;
    if (ovl) cudaStreamWaitEvent(h->side, h->ev_fork, 0);
    {
      ProfScope ps(h, evs, fs, FDTD_KERNEL_FACE_COPY, n);
      launch_face_copy(g, h->F(pc), h->faces, h->face_at(n), 0, fs);
    }
    if (ovl) cudaEventRecord(h->ev_join[n % 2], h->side);
    launches += 1;
  };
  if (ovl && nsteps > 0) {
    cudaEventRecord(h->ev_fork, st);
    replay(nsteps - 1);
  }
  for (int n = nsteps - 1; n >= 0; --n) {
    if (faces && n < h->seg_first) launches += regen_segment(h, n / h->seg_steps, pc, st);
    launches += rev_step_pre(h, n, nsteps, pc, 0, st, evs);
    if (ovl) cudaStreamWaitEvent(st, h->ev_join[n % 2], 0);  // H^{n+1/2} on the faces is in place
    else if (faces) replay(n);
    {
      ProfScope ps(h, evs, st, FDTD_KERNEL_REV_E, n);
      split_step_args(h, ra, n, pc, pb, 0);
      launch_rev_E(ra, rm, st);
    }
    if (ovl && n > 0) {  // rev_E(n) has read the faces of step n: replay those of step n-1
      cudaEventRecord(h->ev_fork, st);
      replay(n - 1);
    }
    launches += rev_step_mid(h, n, pc, 0, st);
    {
      ProfScope ps(h, evs, st, FDTD_KERNEL_REV_H, n);
      split_step_args(h, ra, n, pc, pb, 1);
      launch_rev_H(ra, rm, st);
    }
    launches += 2;
    launches += rev_step_post(h, n, pc, 0, st);
    pb = 1 - pb;
  }
  if (nsteps > 0) launches += rev_finish(h, pc, 0, st);
  return launches;
}

// Wait for the handle's stream and report what the kernels flagged in the status word, clearing it.
int sync_status(fdtd_handle* h) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, h->status, 4, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (st == 0) return FDTD_OK;
  CK(cudaMemsetAsync(h->status, 0, 4, h->stream));
  if (st & kStatusTimeout)
    return fail(FDTD_ERR_TIMEOUT, "a device-side wait for a TMA copy gave up (status %d); results are invalid", st);
  return fail(FDTD_ERR_NONFINITE, "a field check found a NaN or an infinity; results are invalid");
}

// NVTX range over a host call (the enqueue; the GPU work of a captured loop is one graph launch), so
// that profilers can attribute and filter by phase
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// Read the timing events of every profiled replay still pending (waits for the stream). Called
// before a pending graph is replayed again, after a backward, and by fdtd_profile_read, so a
// forward followed by a backward costs one wait at the end instead of one between the two.
int prof_collect(fdtd_handle* h) {
  LoopGraph* gs[2] = {&h->gfwd, &h->gbwd};
  bool any = false;
  for (LoopGraph* lg : gs) any |= lg->pending;
  if (!any) return FDTD_OK;
  CK(cudaStreamSynchronize(h->stream));
  for (LoopGraph* lg : gs) {
    if (!lg->pending) continue;
    for (auto& e : lg->ev) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e.a, e.b));
      h->prof_ms[e.kind] += ms;
      h->prof_n[e.kind] += 1;
    }
    lg->pending = false;
  }
  return FDTD_OK;
}

// Replay the cached graph of a time loop, capturing it first if its shape or buffers changed; with
// use_graphs off, launch the loop's kernels directly on the stream instead (no graph to build: the
// cheaper choice for a handle that solves once).
template <class Enqueue>
int run_loop(fdtd_handle* h, LoopGraph& lg, int nsteps, int64_t key, Enqueue enqueue) {
  if (nsteps == 0) return FDTD_OK;
  if (lg.pending) TRY(prof_collect(h));  // its events are about to be recorded again
  if (!h->use_graphs) {
    lg.reset();
    const int64_t n = enqueue(h->stream, h->prof_every > 0 ? &lg.ev : nullptr);
    CK(cudaGetLastError());
    h->launches += n;
    lg.pending = h->prof_every > 0 && !lg.ev.empty();
    return FDTD_OK;
  }
  const int cur0 = h->cur;
  if (!(lg.exec && lg.nsteps == nsteps && lg.key == key && lg.gen == h->gen)) {
    lg.reset();
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    lg.launches = enqueue(h->cap, h->prof_every > 0 ? &lg.ev : nullptr);
    h->capturing = false;
    cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (e != cudaSuccess) {
      h->cur = cur0;
      lg.reset();
      return fail(FDTD_ERR_CUDA, "capture of the time loop failed: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&lg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->cur = cur0;
      lg.reset();
      return fail(FDTD_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    lg.cur_after = h->cur;
    lg.nsteps = nsteps;
    lg.key = key;
    lg.gen = h->gen;
  }
  CK(cudaGraphLaunch(lg.exec, h->stream));
  h->cur = lg.cur_after;
  h->launches += lg.launches;
  lg.pending = h->prof_every > 0 && !lg.ev.empty();
  return FDTD_OK;
}

}  // namespace

extern "C" {

const char* fdtd_last_error(void) { return g_last_error.c_str(); }

const char* fdtd_version(void) { return "libfdtd 0.2 (sm_103a)"; }

int fdtd_set_byte_budget(int64_t bytes) {
  g_byte_budget = bytes;
  return FDTD_OK;
}

int64_t fdtd_footprint_bytes(const fdtd_grid* grid, const fdtd_pml* pml, int32_t nsteps, int32_t record_faces,
                             const int32_t design_lo[3], const int32_t design_hi[3]) {
  if (validate(grid, 0.5, pml) != FDTD_OK || nsteps < 0) return -1;
  const Geo g = make_geo(*grid, *pml, 0.5);
  int64_t b = 0;
  b += 13 * g.vol * 4;                                // fields (double-buffered) + a
  b += 4 * psi_bytes(g);                              // forward psi of E and H, double-buffered
  b += (int64_t)7 * (g.n[0] + g.n[1] + g.n[2]) * 4;   // CPML and slab-index tables
  b += 12 * g.vol * 4;                                // adjoint fields (double-buffered)
  b += 4 * psi_bytes(g);                              // adjoint psi, double-buffered
  int64_t design = 0;
  if (design_lo && design_hi) design = box_cells(design_lo, design_hi);
  b += design * 8;
  if (record_faces) b += make_faces(g).per_step * (int64_t)nsteps * 4;
  return b;
}

int fdtd_create(fdtd_handle** out, const fdtd_grid* grid, double spacing, double courant, const float* eps_inv,
                const fdtd_source* src, int32_t nsrc, const fdtd_detector* det, int32_t ndet, const fdtd_pml* pml,
                const int32_t design_lo[3], const int32_t design_hi[3], void* cuda_stream) {
  if (!out) return fail(FDTD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  TRY(validate(grid, courant, pml));
  if (!eps_inv) return fail(FDTD_ERR_INVALID_ARG, "eps_inv is NULL");
  if (nsrc < 0 || ndet < 0 || (nsrc > 0 && !src) || (ndet > 0 && !det))
    return fail(FDTD_ERR_INVALID_ARG, "bad source or detector list");
  const int n[3] = {grid->nx, grid->ny, grid->nz};
  for (int q = 0; q < nsrc; ++q) {
    const fdtd_source& s = src[q];
    if (s.component < 0 || s.component > 2) return fail(FDTD_ERR_INVALID_ARG, "source %d: component must be 0..2", q);
    if (!box_ok(s.lo, s.hi, n, false)) return fail(FDTD_ERR_INVALID_ARG, "source %d: box outside the grid", q);
    if (!(s.tau_steps > 0) || !(s.wavelength_cells > 0))
      return fail(FDTD_ERR_INVALID_ARG, "source %d: tau and wavelength must be positive", q);
    if (s.tfsf != 0) {
      const int ax = std::abs(s.tfsf) - 1;
      if (ax > 2) return fail(FDTD_ERR_INVALID_ARG, "source %d: tfsf must be 0 or +-1..3", q);
      if (s.component == ax) return fail(FDTD_ERR_INVALID_ARG, "source %d: a TFSF component must be transverse", q);
      if (s.hi[ax] - s.lo[ax] != 1)
        return fail(FDTD_ERR_INVALID_ARG, "source %d: a TFSF plane is one cell thick along its axis", q);
      if (s.tfsf > 0 ? s.lo[ax] < 1 : s.lo[ax] > n[ax] - 2)
        return fail(FDTD_ERR_INVALID_ARG, "source %d: the TFSF plane needs its scattered-field side in the grid", q);
      if (!(s.eps_background > 0)) return fail(FDTD_ERR_INVALID_ARG, "source %d: eps_background must be positive", q);
    }
  }
  for (int q = 0; q < ndet; ++q) {
    const fdtd_detector& d = det[q];
    if (d.kind < 0 || d.kind > 4) return fail(FDTD_ERR_INVALID_ARG, "detector %d: unknown kind", q);
    if (!box_ok(d.lo, d.hi, n, false)) return fail(FDTD_ERR_INVALID_ARG, "detector %d: box outside the grid", q);
    if (d.kind >= FDTD_DET_PLANE_E2_SUM_INTERP && (d.hi[0] >= n[0] || d.hi[1] >= n[1] || d.hi[2] >= n[2]))
      return fail(FDTD_ERR_INVALID_ARG, "detector %d: an interpolated box needs one more cell inside the grid", q);
    if (d.kind == FDTD_DET_POINT_SERIES && (d.component < 0 || d.component > 5))
      return fail(FDTD_ERR_INVALID_ARG, "detector %d: component must be 0..5", q);
    if ((d.kind == FDTD_DET_PLANE_FLUX || d.kind == FDTD_DET_PLANE_FLUX_INTERP) && (d.axis < 0 || d.axis > 2))
      return fail(FDTD_ERR_INVALID_ARG, "detector %d: axis must be 0..2", q);
  }
  int32_t zlo[3] = {0, 0, 0};
  const int32_t* dlo = design_lo ? design_lo : zlo;
  const int32_t* dhi = design_hi ? design_hi : zlo;
  if (!box_ok(dlo, dhi, n, true)) return fail(FDTD_ERR_INVALID_ARG, "design box outside the grid");
  for (int q = 0; q < nsrc; ++q) {  // a TFSF plane (E) and its H half plane stay off the design box
    const fdtd_source& s = src[q];
    if (s.tfsf == 0) continue;
    const int ax = std::abs(s.tfsf) - 1;
    for (int side = 0; side < 2; ++side) {
      int lo[3] = {s.lo[0], s.lo[1], s.lo[2]}, hi[3] = {s.hi[0], s.hi[1], s.hi[2]};
      if (side == 1) {
        lo[ax] -= s.tfsf > 0 ? 1 : 0;
        hi[ax] = lo[ax] + 1;
      }
      bool meet = true;
      for (int d = 0; d < 3; ++d) meet = meet && lo[d] < dhi[d] && hi[d] > dlo[d];
      if (meet) return fail(FDTD_ERR_INVALID_ARG, "source %d: a TFSF plane must not meet the design box", q);
    }
  }

  fdtd_handle* h = new fdtd_handle();
  h->pml = *pml;
  h->spacing = spacing;
  h->courant = courant;
  h->stream = (cudaStream_t)cuda_stream;
  h->g = make_geo(*grid, *pml, courant);
  h->faces = make_faces(h->g);
  for (int d = 0; d < 3; ++d) {
    h->design_lo[d] = dlo[d];
    h->design_hi[d] = dhi[d];
  }
  auto cleanup = [&](int rc) {
    fdtd_destroy(h);
    return rc;
  };
  const Geo& g = h->g;
  int rc;
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaError_t e = cudaGetLastError();
    return cleanup(fail(FDTD_ERR_CUDA, "stream or event creation: %s", cudaGetErrorString(e)));
  }
  {
    // z-chunks of the marching kernels, each for its own number of resident blocks per SM
    int per_sm3 = 0, per_sm4 = 0, nsm = 0;
    if ((rc = prepare_fwd_fused(3, &per_sm3)) != FDTD_OK) return cleanup(rc);
    if ((rc = prepare_fwd_fused(4, &per_sm4)) != FDTD_OK) return cleanup(rc);
    int per_sm_rev3 = 0, per_sm_rev4 = 0;
    if ((rc = prepare_rev(3, &per_sm_rev3)) != FDTD_OK) return cleanup(rc);
    if ((rc = prepare_rev(4, &per_sm_rev4)) != FDTD_OK) return cleanup(rc);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cleanup(fail(FDTD_ERR_CUDA, "device attributes: %s", cudaGetErrorString(cudaGetLastError())));
    h->nsm = nsm;
    // column tiles of the forward and of the reverse kernels
    const int64_t nxy = (int64_t)((n[0] + fused_tile_x() - 1) / fused_tile_x()) *
                        ((n[1] + fused_tile_y() - 1) / fused_tile_y());
    const int64_t nxy_rev = (int64_t)((n[0] + rev_tile_x() - 1) / rev_tile_x()) *
                            ((n[1] + rev_tile_y() - 1) / rev_tile_y());
    // forward: a 4-stage ring (more planes in flight per block) when it keeps as many blocks
    // resident per SM as 3 stages do (two, on one B300), else 3 stages
    const int64_t slots4 = (int64_t)nsm * std::max(1, per_sm4), slots3 = (int64_t)nsm * std::max(1, per_sm3);
    const bool ring4 = per_sm4 >= per_sm3;
    h->fwd_nstage = ring4 ? 4 : 3;
    const int64_t slots_f = ring4 ? slots4 : slots3;
    // reverse: a 4-stage ring (three blocks per SM) when the sweep fills at least four waves of
    // them, else 3 stages (four per SM: on one B300 the 96^3 solve ran 8 % faster, 600^3 3 % slower)
    const int64_t slots_r4 = (int64_t)nsm * std::max(1, per_sm_rev4), slots_r3 = (int64_t)nsm * std::max(1, per_sm_rev3);
    const int tz_r4 = choose_tz(nxy_rev, n[2], slots_r4);
    const bool rev_ring4 = nxy_rev * ((n[2] + tz_r4 - 1) / tz_r4) >= 4 * slots_r4;
    h->rev_nstage = rev_ring4 ? 4 : 3;
    const int64_t slots_r = rev_ring4 ? slots_r4 : slots_r3;
    h->tz = choose_tz(nxy, n[2], slots_f);
    h->tz_rev = choose_tz(nxy_rev, n[2], slots_r);
    h->nxy_f = nxy;
    h->nxy_r = nxy_rev;
    h->slots_fwd = slots_f;
    h->slots_rev = slots_r;
    // fused inverse and adjoint steps: like the forward, a 4-stage ring when it keeps as many blocks
    // resident per SM as 3 stages do, else 3 stages; z-chunks for their own resident blocks
    for (int which = 0; which < 2; ++which) {
      int b3 = 0, b4 = 0;
      if ((rc = (which == 0 ? prepare_inv(3, &b3) : prepare_adj(3, &b3))) != FDTD_OK) return cleanup(rc);
      if ((rc = (which == 0 ? prepare_inv(4, &b4) : prepare_adj(4, &b4))) != FDTD_OK) return cleanup(rc);
      const bool r4 = b4 >= b3;
      const int64_t slots = (int64_t)nsm * std::max(1, r4 ? b4 : b3);
      const int tzv = std::min(choose_tz(nxy, n[2], slots), which == 0 ? inv_max_tz() : adj_max_tz());
      (which == 0 ? h->inv_nstage : h->adj_nstage) = r4 ? 4 : 3;
      (which == 0 ? h->tz_inv : h->tz_adj) = tzv;
      (which == 0 ? h->slots_inv : h->slots_adj) = slots;
      if (which == 1) {
        // the tiles of the split adjoint step: leading and trailing tile columns and rows that need
        // the x/y CPML loop, each launch's z-chunks for its own tiles
        const int ntx = adj_tiles_x(g), nty = adj_tiles_y(g);
        int f[4];
        bool ok = adjoint_frame(g, f);
        const int xl = f[0], xh = f[1], yl = f[2], yh = f[3];
        if (const char* e = std::getenv("FDTD_ADJ_SPLIT")) ok &= std::atoi(e) != 0;  // override
        if (const char* e = std::getenv("FDTD_ADJ_OVERLAP")) h->adj_overlap = std::atoi(e) != 0;  // override
        h->adj_split = ok ? 1 : 0;
        h->adj_xl = xl;
        h->adj_xh = xh;
        h->adj_yl = yl;
        h->adj_yh = yh;
        if (ok) {
          const int64_t rect = (int64_t)(ntx - xl - xh) * (nty - yl - yh), frame = (int64_t)ntx * nty - rect;
          h->tz_adj = std::min(choose_tz(rect, n[2], slots), adj_max_tz());
          // the frame launch runs beside the plain one and does best in long chunks: on 600^3 the
          // adjoint step took 2.76 / 2.73 / 2.72 / 2.71 ms with frame chunks of 24 (choose_tz) / 48 /
          // 96 / 256 planes, 2.81 and 2.86 ms with 12 and 8
          h->tz_adj_xy = std::min(std::min(std::max(choose_tz(frame, n[2], slots), 96), n[2]), adj_max_tz());
        }
      }
    }
    if (const char* e = std::getenv("FDTD_TZ")) {  // tuning override: z-planes per block
      const int v = std::atoi(e);
      if (v >= 1) h->tz = h->tz_rev = h->tz_inv = h->tz_adj = h->tz_adj_xy = std::min(v, n[2]);
      h->tz_free = v < 1;
    }
    h->tz_inv = std::min(h->tz_inv, inv_max_tz());
    if (const char* e = std::getenv("FDTD_TZ_FRAME")) {  // tuning override: z-planes per block of the frame launch
      const int v = std::atoi(e);
      if (v >= 1) h->tz_adj_xy = std::min(v, n[2]);
    }
    h->tz_adj = std::min(h->tz_adj, adj_max_tz());
    h->tz_adj_xy = std::min(h->tz_adj_xy, adj_max_tz());
    if (const char* e = std::getenv("FDTD_REV_NSTAGE")) {  // override: ring stages of the reverse kernels
      const int v = std::atoi(e);
      if (v == 3 || v == 4) h->rev_nstage = h->inv_nstage = h->adj_nstage = v;
    }
    {
      h->rev_fused = fused_reverse(g);
      if (const char* e = std::getenv("FDTD_REV_FUSED")) h->rev_fused = std::atoi(e) != 0;  // override
    }
    h->tz = std::min(h->tz, fused_max_tz());
    h->tz_rev = std::min(h->tz_rev, fused_max_tz());
  }
  if ((rc = dev_alloc(h, (void**)&h->fields, 2 * 6 * g.vol * 4)) != FDTD_OK) return cleanup(rc);
  if ((rc = dev_alloc(h, (void**)&h->a, g.vol * 4)) != FDTD_OK) return cleanup(rc);
  if ((rc = dev_alloc(h, (void**)&h->status, 4)) != FDTD_OK) return cleanup(rc);
  if (cudaMemsetAsync(h->status, 0, 4, h->stream) != cudaSuccess)
    return cleanup(fail(FDTD_ERR_CUDA, "status reset: %s", cudaGetErrorString(cudaGetLastError())));
  for (int b = 0; b < 2; ++b) {
    const Fields Fb = h->F(b);
    if ((rc = encode_field_map(&h->fmaps[b].e, Fb.f[0], g, 3, fwd_box_e())) != FDTD_OK) return cleanup(rc);
    if ((rc = encode_field_map(&h->fmaps[b].h, Fb.f[3], g, 3, fwd_box_h())) != FDTD_OK) return cleanup(rc);
    if ((rc = encode_field_map(&h->fmaps[b].a, h->a, g, 1, fwd_box_a())) != FDTD_OK) return cleanup(rc);
    if ((rc = encode_field_map(&h->imaps[b].e, Fb.f[0], g, 3, inv_box_e())) != FDTD_OK) return cleanup(rc);
    if ((rc = encode_field_map(&h->imaps[b].h, Fb.f[3], g, 3, inv_box_h())) != FDTD_OK) return cleanup(rc);
    if ((rc = encode_field_map(&h->imaps[b].a, h->a, g, 1, inv_box_e())) != FDTD_OK) return cleanup(rc);
  }
  const int64_t pf = h->psi_floats();
  if ((rc = dev_alloc(h, (void**)&h->psiE, 2 * pf * 4)) != FDTD_OK) return cleanup(rc);
  if ((rc = dev_alloc(h, (void**)&h->psiH, 2 * pf * 4)) != FDTD_OK) return cleanup(rc);
  if ((rc = upload_tables(h)) != FDTD_OK) return cleanup(rc);
  {
    // a = eps_inv with the row pitch (padding cells hold 0 and are never read)
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    float* tmp = nullptr;
    if ((rc = dev_alloc(h, (void**)&tmp, N * 4)) != FDTD_OK) return cleanup(rc);
    cudaError_t e = cudaMemcpyAsync(tmp, eps_inv, N * 4, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->a, 0, g.vol * 4, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(h->a, (size_t)g.nxp * 4, tmp, (size_t)n[0] * 4, (size_t)n[0] * 4, (size_t)n[1] * n[2],
                            cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // eps_inv may be a host buffer
    dev_free(h, tmp, N * 4);
    if (e != cudaSuccess) return cleanup(fail(FDTD_ERR_CUDA, "copy of eps_inv: %s", cudaGetErrorString(e)));
  }
  // sources: weights = amplitude * profile for a soft source; for a TFSF plane the correction
  // coefficients times the profile (E: -dir S sE a, H: dir S sH); zero where E is held by a PEC wall
  auto add_entry = [&](const fdtd_source& s, int comp, const int* lo, const int* hi, double coef, bool times_a,
                       std::vector<SrcDev>& list) -> int {
    const int64_t m = box_cells(lo, hi);
    const int bx = hi[0] - lo[0], by = hi[1] - lo[1];
    const int c1 = (comp + 1) % 3, c2 = (comp + 2) % 3;
    std::vector<float> w((size_t)m);
    for (int64_t t = 0; t < m; ++t) {
      const int p[3] = {lo[0] + int(t % bx), lo[1] + int((t / bx) % by), lo[2] + int(t / ((int64_t)bx * by))};
      const double prof = s.profile ? (double)s.profile[t] : 1.0;
      const bool held = comp < 3 && (p[c1] == 0 || p[c2] == 0);
      w[(size_t)t] = held ? 0.f : (float)(coef * prof);
    }
    float* dw = nullptr;
    int r = dev_alloc(h, (void**)&dw, m * 4);
    if (r != FDTD_OK) return r;
    h->src_w.push_back(dw);
    if (cudaMemcpyAsync(dw, w.data(), m * 4, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)  // `w` dies on return
      return fail(FDTD_ERR_CUDA, "source upload failed");
    SrcDev sd;
    sd.comp = comp;
    for (int d = 0; d < 3; ++d) {
      sd.lo[d] = lo[d];
      sd.hi[d] = hi[d];
    }
    sd.w = dw;
    sd.g = nullptr;
    if (times_a) launch_source_scale_a(g, h->a, sd, h->stream);
    list.push_back(sd);
    return FDTD_OK;
  };
  for (int q = 0; q < nsrc; ++q) {
    const fdtd_source& s = src[q];
    h->src_host.push_back(s);
    h->src_host.back().profile = nullptr;
    if (s.tfsf == 0) {
      if ((rc = add_entry(s, s.component, s.lo, s.hi, s.amplitude, false, h->srcs)) != FDTD_OK) return cleanup(rc);
      h->src_tfsf.push_back(-1);
      continue;
    }
    const Tfsf t = make_tfsf(s);
    const int it = (int)h->tfsf.size();
    h->tfsf.push_back(t);
    if ((rc = add_entry(s, t.c, s.lo, s.hi, -t.dir * courant * t.sE, true, h->srcs)) != FDTD_OK) return cleanup(rc);
    h->src_tfsf.push_back(it);
    int lo[3] = {s.lo[0], s.lo[1], s.lo[2]}, hi[3] = {s.hi[0], s.hi[1], s.hi[2]};
    lo[t.axis] = s.lo[t.axis] - (t.dir > 0 ? 1 : 0);  // the scattered-side H half plane
    hi[t.axis] = lo[t.axis] + 1;
    if ((rc = add_entry(s, 3 + t.h, lo, hi, t.dir * courant * t.sH, false, h->hsrcs)) != FDTD_OK) return cleanup(rc);
    h->hsrc_tfsf.push_back(it);
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cleanup(fail(FDTD_ERR_CUDA, "source set-up failed"));
  for (int q = 0; q < ndet; ++q) {
    const fdtd_detector& d = det[q];
    DetDev dd;
    dd.kind = d.kind;
    dd.comp = d.component;
    dd.axis = d.axis;
    for (int k = 0; k < 3; ++k) {
      dd.lo[k] = d.lo[k];
      dd.hi[k] = d.hi[k];
    }
    dd.off = 0;
    dd.nblk = 0;
    dd.poff = 0;
    const int64_t m = box_cells(d.lo, d.hi);
    // the first kMaxDet same-index detectors are sampled inside the fused forward kernel
    int ninline = 0;
    for (char c : h->det_inline) ninline += c;
    const bool inl = d.kind <= FDTD_DET_PLANE_FLUX && ninline < kMaxDet;
    if (d.kind == FDTD_DET_PLANE_FLUX || d.kind == FDTD_DET_PLANE_FLUX_INTERP) {
      if (inl) {  // summed inside the fused kernel: one slot per block that meets the box
        h->fwd_tz_free = false;
        const int tx = fused_tile_x(), ty = fused_tile_y();
        dd.nblk = ((d.hi[0] - 1) / tx - d.lo[0] / tx + 1) * ((d.hi[1] - 1) / ty - d.lo[1] / ty + 1) *
                  ((d.hi[2] - 1) / h->tz - d.lo[2] / h->tz + 1);
      } else {
        dd.nblk = (int)std::min<int64_t>(148, std::max<int64_t>(1, (m + 4095) / 4096));
      }
    }
    if (d.kind == FDTD_DET_PLANE_E2_SUM || d.kind == FDTD_DET_PLANE_E2_SUM_INTERP) h->det_total_fixed += m;
    else h->det_total_per_step += 1;
    float* slab = nullptr;
    if (d.kind == FDTD_DET_PLANE_FLUX_INTERP &&
        (rc = dev_alloc(h, (void**)&slab, 3 * interp_slab_floats(dd) * 4)) != FDTD_OK)
      return cleanup(rc);
    // the first kMaxDet detectors whose adjoint reads only E are folded into rev_H's E-bar write
    int nfold = 0;
    for (char c : h->det_fold) nfold += c;
    const bool fold = (d.kind == FDTD_DET_PLANE_E2_SUM || (d.kind == FDTD_DET_POINT_SERIES && d.component < 3)) &&
                      nfold < kMaxDet;
    h->dets.push_back(dd);
    h->det_inline.push_back(inl ? 1 : 0);
    h->det_fold.push_back(fold ? 1 : 0);
    h->det_slab.push_back(slab);
  }
  *out = h;
  return FDTD_OK;
}

int fdtd_destroy(fdtd_handle* h) {
  if (!h) return FDTD_OK;
  // a captured time loop may still be running: finish the stream before its graph goes; without one,
  // the frees below are ordered after the enqueued work and nothing needs to wait
  const bool graphs = h->gfwd.exec || h->gbwd.exec;
  if (graphs) cudaStreamSynchronize(h->stream);
  h->gfwd.reset();
  h->gbwd.reset();
  void* bufs[] = {h->fields, h->a, h->psiE, h->psiH, h->tables, h->init, h->gtab, h->det_out, h->partial,
                  h->face_hist, h->adj, h->psibar, h->dLda, h->dLddet, h->staging, h->status, h->seg_states};
  for (void* p : bufs)
    if (p) cudaFreeAsync(p, h->stream);
  for (float* p : h->src_w) cudaFreeAsync(p, h->stream);
  for (float* p : h->det_slab)
    if (p) cudaFreeAsync(p, h->stream);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->side2) cudaStreamDestroy(h->side2);
  if (h->ev_fork2) cudaEventDestroy(h->ev_fork2);
  if (h->ev_join2) cudaEventDestroy(h->ev_join2);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  for (cudaEvent_t e : h->ev_join)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  delete h;
  return FDTD_OK;
}

int fdtd_set_design_eps_inv(fdtd_handle* h, const float* eps_inv_box) {
  if (!h || !eps_inv_box) return fail(FDTD_ERR_INVALID_ARG, "NULL argument");
  h->density = false;
  const int64_t m = box_cells(h->design_lo, h->design_hi);
  if (m == 0) return FDTD_OK;
  TRY(ensure_staging(h));
  CK(cudaMemcpyAsync(h->staging, eps_inv_box, m * 4, cudaMemcpyDefault, h->stream));
  launch_set_box(h->g, h->a, h->design_lo, h->design_hi, h->staging, h->stream);
  h->launches += 1;
  CK(cudaGetLastError());
  return FDTD_OK;
}

int fdtd_set_initial_fields(fdtd_handle* h, const float* fields6) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (!fields6) {
    if (h->init) {
      CK(cudaStreamSynchronize(h->stream));
      dev_free(h, h->init, 6 * h->g.vol * 4);
      h->init = nullptr;
    }
    return FDTD_OK;
  }
  if (!h->init) {
    TRY(dev_alloc(h, (void**)&h->init, 6 * h->g.vol * 4));
    CK(cudaMemsetAsync(h->init, 0, 6 * h->g.vol * 4, h->stream));
  }
  TRY(ensure_staging(h));
  const int64_t N = (int64_t)h->g.n[0] * h->g.n[1] * h->g.n[2];
  CK(cudaMemcpyAsync(h->staging, fields6, 6 * N * 4, cudaMemcpyDefault, h->stream));
  Fields I;
  for (int c = 0; c < 6; ++c) I.f[c] = h->init + c * h->g.vol;
  launch_pack_fields(h->g, I, h->staging, 1, h->stream);
  h->launches += 1;
  CK(cudaGetLastError());
  return FDTD_OK;
}

// Checks and buffers of a forward solve of nsteps steps, and the initial state (no step runs).
static int forward_prepare(fdtd_handle* h, int32_t nsteps, uint32_t flags) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (nsteps < 0) return fail(FDTD_ERR_INVALID_ARG, "nsteps must be >= 0");
  const bool record = (flags & FDTD_RECORD_FACES) != 0;
  if (record) {
    for (const auto& d : h->dets) {
      int hi[3] = {d.hi[0], d.hi[1], d.hi[2]};
      if (d.kind >= FDTD_DET_PLANE_E2_SUM_INTERP)  // the interpolation stencil reaches one cell further
        for (int k = 0; k < 3; ++k) hi[k] += 1;
      if (!in_r_cells(h, d.lo, hi))
        return fail(FDTD_ERR_INVALID_ARG, "a detector lies in the PML; backward needs detectors in the PML-free region");
    }
    if (!in_r_cells(h, h->design_lo, h->design_hi))
      return fail(FDTD_ERR_INVALID_ARG, "the design box must lie in the PML-free region");
  }
  h->recorded = false;
  h->consumed = false;
  h->last_nsteps = nsteps;
  TRY(ensure_gtab(h, nsteps));
  TRY(ensure_det(h, nsteps));
  h->seg_first = 0;
  if (record && h->faces.per_step > 0) {
    const int S = h->segments(nsteps);
    const int held = S > 1 ? h->seg_steps : nsteps;  // steps whose faces the history holds
    h->seg_first = (S - 1) * h->seg_steps;
    TRY(ensure_buf(h, &h->face_hist, &h->face_cap_steps, (int64_t)held, h->faces.per_step * 4));
    if (S > 2) TRY(ensure_buf(h, &h->seg_states, &h->seg_cap, (int64_t)(S - 2), h->state_floats() * 4));
  }
  TRY(reset_state(h));
  h->phase = FDTD_PHASE_IDLE;
  return FDTD_OK;
}

int fdtd_forward(fdtd_handle* h, int32_t nsteps, uint32_t flags) {
  NvtxRange range("fdtd_forward");
  TRY(forward_prepare(h, nsteps, flags));
  const bool record = (flags & FDTD_RECORD_FACES) != 0;
  const int64_t key = (record ? 1 : 0) | ((int64_t)h->face_overlap << 1) | ((int64_t)h->prof_every << 2) |
                      ((int64_t)h->check_every << 32) | ((int64_t)h->seg_steps << 44);
  TRY(run_loop(h, h->gfwd, nsteps, key, [&](cudaStream_t st, std::vector<Ev>* evs) {
    return enqueue_forward(h, nsteps, record, st, evs);
  }));
  CK(cudaGetLastError());
  h->recorded = record;
  return FDTD_OK;
}

// Checks and buffers of the reverse sweep of the last recorded forward: dL/d(det) uploaded, the
// adjoint fields, their CPML memories and dL/da zeroed.
static int backward_prepare(fdtd_handle* h, const double* dL_ddet) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (!h->recorded || h->consumed)
    return fail(FDTD_ERR_STATE, "backward needs a forward with FDTD_RECORD_FACES that no backward has consumed");
  const int nsteps = h->last_nsteps;
  const int64_t ndet = det_total_for(h, nsteps);
  if (ndet > 0 && !dL_ddet) return fail(FDTD_ERR_INVALID_ARG, "dL_ddet is NULL");
  const int64_t M = box_cells(h->design_lo, h->design_hi);
  const Geo& g = h->g;
  const int64_t pf = h->psi_floats();
  TRY(ensure_adjoint(h));
  if (!h->psibar && pf > 0) TRY(dev_alloc(h, (void**)&h->psibar, 4 * pf * 4));
  if (!h->dLda && M > 0) TRY(dev_alloc(h, (void**)&h->dLda, M * 8));
  TRY(ensure_buf(h, &h->dLddet, &h->dLddet_cap, ndet, 8));
  if (M > 0) TRY(ensure_staging(h));
  if (ndet > 0) CK(cudaMemcpyAsync(h->dLddet, dL_ddet, ndet * 8, cudaMemcpyDefault, h->stream));
  CK(cudaMemsetAsync(h->adj, 0, 12 * g.vol * 4, h->stream));
  fill_canaries(h, false, true, false);
  if (pf > 0) CK(cudaMemsetAsync(h->psibar, 0, 4 * pf * 4, h->stream));
  if (M > 0) CK(cudaMemsetAsync(h->dLda, 0, M * 8, h->stream));
  return FDTD_OK;
}

// dL/deps (times scale) from dL/da into the caller's buffer, after the reverse sweep.
static int backward_finish(fdtd_handle* h, float* dL_deps, double scale) {
  const int64_t M = box_cells(h->design_lo, h->design_hi);
  if (M > 0) {
    launch_grad_finalize(h->g, h->a, h->design_lo, h->design_hi, h->dLda, h->staging, scale, h->stream);
    h->launches += 1;
    CK(cudaMemcpyAsync(dL_deps, h->staging, M * 4, cudaMemcpyDefault, h->stream));
  }
  CK(cudaGetLastError());
  h->consumed = true;
  TRY(prof_collect(h));
  if (M > 0 && is_host_pointer(dL_deps)) return sync_status(h);
  return FDTD_OK;
}

static int backward_scaled(fdtd_handle* h, const double* dL_ddet, float* dL_deps, double scale) {
  if (h && box_cells(h->design_lo, h->design_hi) > 0 && !dL_deps) return fail(FDTD_ERR_INVALID_ARG, "dL_deps is NULL");
  TRY(backward_prepare(h, dL_ddet));
  const int nsteps = h->last_nsteps;
  h->phase = FDTD_PHASE_IDLE;
  const int64_t key = h->cur | ((int64_t)h->face_overlap << 1) | ((int64_t)h->prof_every << 2);
  TRY(run_loop(h, h->gbwd, nsteps, key | ((int64_t)h->rev_fused << 40) | ((int64_t)h->seg_steps << 44),
               [&](cudaStream_t st, std::vector<Ev>* evs) {
    return h->rev_fused ? enqueue_backward(h, nsteps, st, evs) : enqueue_backward_split(h, nsteps, st, evs);
  }));
  return backward_finish(h, dL_deps, scale);
}

int fdtd_backward(fdtd_handle* h, const double* dL_ddet, float* dL_deps) {
  NvtxRange range("fdtd_backward");
  return backward_scaled(h, dL_ddet, dL_deps, 1.0);
}

// ---- grouped and incremental solves -------------------------------------------------------------

int fdtd_poll_status(fdtd_handle* h) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  int st = 0;
  // on the handle's private stream, so that the stream it shares with others keeps running
  CK(cudaMemcpyAsync(&st, h->status, 4, cudaMemcpyDeviceToHost, h->cap));
  CK(cudaStreamSynchronize(h->cap));
  if (st == 0) return FDTD_OK;
  CK(cudaMemsetAsync(h->status, 0, 4, h->cap));
  CK(cudaStreamSynchronize(h->cap));
  if (st & kStatusTimeout)
    return fail(FDTD_ERR_TIMEOUT, "a device-side wait for a TMA copy gave up (status %d); results are invalid", st);
  return fail(FDTD_ERR_NONFINITE, "a field check found a NaN or an infinity; results are invalid");
}

int fdtd_set_stream(fdtd_handle* h, void* cuda_stream) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  h->stream = (cudaStream_t)cuda_stream;
  return FDTD_OK;
}

int fdtd_begin(fdtd_handle* h, int32_t nsteps, uint32_t flags) {
  if (h && h->seg_steps > 0 && (flags & FDTD_RECORD_FACES) && h->segments(nsteps) > 1)
    return fail(FDTD_ERR_INVALID_ARG, "segmented face histories are solved with fdtd_forward / fdtd_backward");
  TRY(forward_prepare(h, nsteps, flags));
  h->solve_record = (flags & FDTD_RECORD_FACES) != 0;
  h->step_next = 0;
  h->phase = FDTD_PHASE_FORWARD;
  if (nsteps == 0) {
    h->phase = FDTD_PHASE_FORWARD_DONE;
    h->recorded = h->solve_record;
  }
  return FDTD_OK;
}

int fdtd_begin_backward(fdtd_handle* h, const double* dL_ddet) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (h->phase != FDTD_PHASE_FORWARD_DONE) return fail(FDTD_ERR_STATE, "fdtd_begin_backward needs a finished forward");
  TRY(backward_prepare(h, dL_ddet));
  h->rev_pc = h->cur;
  h->rev_ac = 0;
  h->rev_pb = 0;
  h->step_next = h->last_nsteps - 1;
  h->phase = FDTD_PHASE_BACKWARD;
  if (h->last_nsteps == 0) h->phase = FDTD_PHASE_DONE;
  return FDTD_OK;
}

int fdtd_phase(fdtd_handle* h, int32_t* phase, int32_t* steps_left) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (phase) *phase = h->phase;
  if (steps_left)
    *steps_left = h->phase == FDTD_PHASE_FORWARD ? h->last_nsteps - h->step_next
                                                 : (h->phase == FDTD_PHASE_BACKWARD ? h->step_next + 1 : 0);
  return FDTD_OK;
}

static int finish_backward_scaled(fdtd_handle* h, float* out, double scale) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (h->phase != FDTD_PHASE_DONE) return fail(FDTD_ERR_STATE, "the reverse sweep has not finished");
  if (box_cells(h->design_lo, h->design_hi) > 0 && !out) return fail(FDTD_ERR_INVALID_ARG, "dL_deps is NULL");
  h->phase = FDTD_PHASE_IDLE;
  return backward_finish(h, out, scale);
}

int fdtd_finish_backward(fdtd_handle* h, float* dL_deps) { return finish_backward_scaled(h, dL_deps, 1.0); }

int fdtd_finish_backward_density(fdtd_handle* h, float* dL_drho) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (!h->density) return fail(FDTD_ERR_STATE, "no design density was set");
  return finish_backward_scaled(h, dL_drho, h->eps_hi - h->eps_lo);
}

}  // extern "C"

namespace {
// The z-chunks of the n requests of a grouped launch of one kernel (0 the forward, 1 the inverse step,
// 2 the adjoint step, 3 either kernel of the in-place pair), chosen together by group_tz; a[r] holds
// request r's arguments with its own z-chunk, hs[r] its handle. The results do not depend on them.
template <class Args>
void group_chunks(Args* a, fdtd_handle* const* hs, int n, int kind) {
  if (n < 2) return;
  int64_t nxy[FDTD_MAX_GROUP];
  int nz[FDTD_MAX_GROUP], own[FDTD_MAX_GROUP];
  bool fr[FDTD_MAX_GROUP];
  for (int r = 0; r < n; ++r) {
    const fdtd_handle* h = hs[r];
    nxy[r] = kind == 3 ? h->nxy_r : h->nxy_f;
    nz[r] = h->g.n[2];
    own[r] = a[r].tz;
    fr[r] = h->tz_free && (kind != 0 || h->fwd_tz_free);
  }
  const fdtd_handle* h0 = hs[0];  // the launch runs request 0's ring stages, so its slots per SM
  const int64_t slots = kind == 0 ? h0->slots_fwd : kind == 1 ? h0->slots_inv : kind == 2 ? h0->slots_adj : h0->slots_rev;
  const int cap = kind == 1 ? inv_max_tz() : kind == 2 ? adj_max_tz() : fused_max_tz();
  const int tz = group_tz(n, nxy, nz, own, fr, slots, std::min(64, cap));
  for (int r = 0; r < n; ++r)
    if (fr[r]) a[r].tz = std::min(tz, nz[r]);
}
}  // namespace

extern "C" {

int fdtd_group_step(fdtd_handle* const* hs, int32_t n, int32_t nsteps) {
  NvtxRange range("fdtd_group_step");
  if (!hs || n < 1 || n > FDTD_MAX_GROUP || nsteps < 0)
    return fail(FDTD_ERR_INVALID_ARG, "a group holds 1..%d handles and nsteps >= 0", FDTD_MAX_GROUP);
  for (int r = 0; r < n; ++r) {
    if (!hs[r]) return fail(FDTD_ERR_INVALID_ARG, "NULL handle in the group");
    if (hs[r]->stream != hs[0]->stream) return fail(FDTD_ERR_INVALID_ARG, "the handles of a group share one stream");
    for (int q = 0; q < r; ++q)
      if (hs[q] == hs[r]) return fail(FDTD_ERR_INVALID_ARG, "a handle appears twice in the group");
  }
  cudaStream_t st = hs[0]->stream;
  static_assert(FDTD_MAX_GROUP <= kMaxGroup, "group structures hold FDTD_MAX_GROUP requests");
  for (int t = 0; t < nsteps; ++t) {
    fdtd_handle* F[FDTD_MAX_GROUP];
    fdtd_handle* Rv[FDTD_MAX_GROUP];
    int nf = 0, nr = 0;
    for (int r = 0; r < n; ++r) {
      fdtd_handle* h = hs[r];
      if (h->phase == FDTD_PHASE_FORWARD && h->step_next < h->last_nsteps) F[nf++] = h;
      else if (h->phase == FDTD_PHASE_BACKWARD && h->step_next >= 0) Rv[nr++] = h;
    }
    if (nf + nr == 0) break;
    if (nf > 0) {  // one forward step of every handle in its forward phase
      // the group's kernel parameters (large, so kept per host thread rather than on the stack)
      static thread_local std::unique_ptr<FwdGroup> Gp;
      if (!Gp) Gp.reset(new FwdGroup());
      FwdGroup& FG = *Gp;
      FaceGroup faces{};
      faces.to_record = 1;
      for (int r = 0; r < nf; ++r) {
        fdtd_handle* h = F[r];
        h->launches += fwd_step_pre(h, h->step_next, st);
        FG.a[r] = fwd_base(h);
        fwd_step_args(h, FG.a[r], h->step_next);
        FG.m[r] = h->fmaps[h->cur];
      }
      FG.n = nf;
      group_chunks(FG.a, F, nf, 0);
      // a launch of one request goes through the single-request kernels (same arithmetic, small
      // parameter blocks; a lone served request then steps as fast as a solo solve)
      if (nf == 1) launch_fwd_fused(FG.a[0], FG.m[0], st);
      else launch_fwd_group(FG, st);
      for (int r = 0; r < nf; ++r) {
        fdtd_handle* h = F[r];
        h->launches += 1;
        if (h->solve_record && h->faces.per_step > 0) {
          FaceJob& J = faces.e[faces.n++];
          J.g = h->g;
          J.F = h->F(1 - h->cur);
          J.fs = h->faces;
          J.rec = h->face_hist + (int64_t)h->step_next * h->faces.per_step;
          h->launches += 1;
        }
      }
      if (faces.n == 1) launch_face_copy(faces.e[0].g, faces.e[0].F, faces.e[0].fs, faces.e[0].rec, faces.to_record, st);
      else if (faces.n > 0) launch_face_copy_group(faces, st);
      for (int r = 0; r < nf; ++r) {
        fdtd_handle* h = F[r];
        h->launches += fwd_step_post(h, h->step_next, h->last_nsteps, st);
        h->cur = 1 - h->cur;
        if (++h->step_next == h->last_nsteps) {
          h->launches += fwd_finish(h, h->last_nsteps, st);
          h->recorded = h->solve_record;
          h->phase = FDTD_PHASE_FORWARD_DONE;
        }
      }
    }
    if (nr > 0) {  // one reverse step of every handle in its reverse phase
      static thread_local std::unique_ptr<InvGroup> IGp;
      static thread_local std::unique_ptr<AdjGroup> AGp;
      static thread_local std::unique_ptr<RevGroup> RGp;
      if (!IGp) IGp.reset(new InvGroup());
      if (!AGp) AGp.reset(new AdjGroup());
      if (!RGp) RGp.reset(new RevGroup());
      InvGroup& IG = *IGp;
      AdjGroup& AG = *AGp;
      RevGroup& RG = *RGp;
      FaceGroup faces{};
      faces.to_record = 0;
      for (int r = 0; r < nr; ++r) {
        fdtd_handle* h = Rv[r];
        h->launches += rev_step_pre(h, h->step_next, h->last_nsteps, h->rev_pc, h->rev_ac, st, nullptr);
        if (h->faces.per_step > 0) {  // H^{n+1/2} on the boundary faces
          FaceJob& J = faces.e[faces.n++];
          J.g = h->g;
          J.F = h->F(h->rev_pc);
          J.fs = h->faces;
          J.rec = h->face_hist + (int64_t)h->step_next * h->faces.per_step;
          h->launches += 1;
        }
      }
      if (faces.n == 1) launch_face_copy(faces.e[0].g, faces.e[0].F, faces.e[0].fs, faces.e[0].rec, faces.to_record, st);
      else if (faces.n > 0) launch_face_copy_group(faces, st);
      // first halves: the fused inverse steps, and rev_E of the in-place pairs
      fdtd_handle* fh[FDTD_MAX_GROUP];  // the handles of the fused kind, and of the in-place pair
      fdtd_handle* sh[FDTD_MAX_GROUP];
      IG.n = RG.n = 0;
      for (int r = 0; r < nr; ++r) {
        fdtd_handle* h = Rv[r];
        if (h->rev_fused) {
          InvArgs& ia = IG.a[IG.n];
          ia = inv_base(h);
          inv_step_args(h, ia, h->step_next, h->rev_pc, h->rev_ac);
          fh[IG.n] = h;
          IG.m[IG.n++] = h->imaps[h->rev_pc];
        } else {
          RevArgs& ra = RG.a[RG.n];
          ra = split_base(h);
          split_step_args(h, ra, h->step_next, h->rev_pc, h->rev_pb, 0);
          sh[RG.n] = h;
          RG.m[RG.n++] = h->rmaps[h->rev_pc];
        }
        h->launches += 1;
      }
      group_chunks(IG.a, fh, IG.n, 1);
      group_chunks(RG.a, sh, RG.n, 3);
      if (IG.n == 1) launch_inv(IG.a[0], IG.m[0], st);
      else if (IG.n > 0) launch_inv_group(IG, st);
      if (RG.n == 1) launch_rev_E(RG.a[0], RG.m[0], st);
      else if (RG.n > 0) launch_rev_group(RG, 0, st);
      // second halves: the fused adjoint steps, and rev_H of the in-place pairs
      AG.n = RG.n = 0;
      for (int r = 0; r < nr; ++r) {
        fdtd_handle* h = Rv[r];
        const int pn = h->rev_fused ? 1 - h->rev_pc : h->rev_pc;
        h->launches += rev_step_mid(h, h->step_next, pn, h->rev_ac, st);
        if (h->rev_fused) {
          AdjArgs& aa = AG.a[AG.n];
          aa = adj_base(h);
          adj_step_args(h, aa, h->step_next, h->rev_pc, h->rev_ac, h->rev_pb);
          AG.m[AG.n++] = h->amaps[h->rev_ac];
        } else {
          RevArgs& ra = RG.a[RG.n];
          ra = split_base(h);
          split_step_args(h, ra, h->step_next, h->rev_pc, h->rev_pb, 1);
          RG.m[RG.n++] = h->rmaps[h->rev_pc];
        }
        h->launches += 1;
      }
      group_chunks(AG.a, fh, AG.n, 2);
      group_chunks(RG.a, sh, RG.n, 3);
      if (AG.n == 1) fh[0]->launches += launch_adj(AG.a[0], AG.m[0], st) - 1;  // one or two launches
      else if (AG.n > 0) launch_adj_group(AG, st);
      if (RG.n == 1) launch_rev_H(RG.a[0], RG.m[0], st);
      else if (RG.n > 0) launch_rev_group(RG, 1, st);
      for (int r = 0; r < nr; ++r) {
        fdtd_handle* h = Rv[r];
        if (h->rev_fused) {
          h->launches += rev_step_post(h, h->step_next, 1 - h->rev_pc, 1 - h->rev_ac, st);
          h->rev_pc = 1 - h->rev_pc;
          h->rev_ac = 1 - h->rev_ac;
        } else {
          h->launches += rev_step_post(h, h->step_next, h->rev_pc, 0, st);
        }
        h->rev_pb = 1 - h->rev_pb;
        if (--h->step_next < 0) {
          h->cur = h->rev_pc;
          h->launches += rev_finish(h, h->rev_pc, h->rev_ac, st);
          h->phase = FDTD_PHASE_DONE;
        }
      }
    }
  }
  CK(cudaGetLastError());
  return FDTD_OK;
}

int fdtd_group_forward(fdtd_handle* const* hs, int32_t n, const int32_t* nsteps, uint32_t flags) {
  if (!hs || !nsteps || n < 1 || n > FDTD_MAX_GROUP) return fail(FDTD_ERR_INVALID_ARG, "bad group");
  int32_t most = 0;
  for (int r = 0; r < n; ++r) {
    TRY(fdtd_begin(hs[r], nsteps[r], flags));
    most = std::max(most, nsteps[r]);
  }
  return fdtd_group_step(hs, n, most);
}

int fdtd_group_backward(fdtd_handle* const* hs, int32_t n, const double* const* dL_ddet, float* const* dL_deps) {
  if (!hs || !dL_ddet || !dL_deps || n < 1 || n > FDTD_MAX_GROUP) return fail(FDTD_ERR_INVALID_ARG, "bad group");
  int32_t most = 0;
  for (int r = 0; r < n; ++r) {
    TRY(fdtd_begin_backward(hs[r], dL_ddet[r]));
    most = std::max(most, hs[r]->last_nsteps);
  }
  TRY(fdtd_group_step(hs, n, most));
  for (int r = 0; r < n; ++r) TRY(fdtd_finish_backward(hs[r], dL_deps[r]));
  return FDTD_OK;
}

// ---- Checkpointing gradient (Sec. 2.2: the recomputation alternative to time reversal) -------------
// The adjoint of step n needs the forward state after step n. Instead of rebuilding it with the
// inverse step, a checkpointing schedule keeps full states (fields and CPML memories) in `slots`
// buffers and recomputes the others forward from the nearest one. Each adjoint step re-evaluates its
// own forward step from its input state (as in Griewank's revolve), so reversing l steps evaluates
// at least l forward steps.
//   recursive halving: split the range in the middle, keep the middle state while the upper half is
//     reversed, recurse; ceil(log2 l) + 1 states, (l/2) log2 l extra forward steps for l = 2^j;
//   treeverse (binomial checkpointing) with c states: the split minimising the forward steps, by
//     dynamic programming over T(l, k) = min_m [m + T(l - m, k - 1) + T(m, k)], T(1, k) = 1,
//     T(l, 0) = l (l + 1) / 2 (k free states besides the one holding the range's start).
namespace {

struct CkptTable {
  int L = 0, K = 0;
  std::vector<int64_t> T;  // (L + 1) x (K + 1)
  std::vector<int> M;      // argmin split length
  int64_t& t(int l, int k) { return T[(size_t)l * (K + 1) + k]; }
  int& m(int l, int k) { return M[(size_t)l * (K + 1) + k]; }
  void build(int L_, int K_) {
    L = L_;
    K = K_;
    T.assign((size_t)(L + 1) * (K + 1), 0);
    M.assign((size_t)(L + 1) * (K + 1), 0);
    for (int l = 1; l <= L; ++l) t(l, 0) = (int64_t)l * (l + 1) / 2;
    for (int k = 1; k <= K; ++k) {
      t(1, k) = 1;
      for (int l = 2; l <= L; ++l) {
        int64_t best = INT64_MAX;
        int bm = 1;
        for (int s = 1; s < l; ++s) {
          const int64_t c = s + t(l - s, k - 1) + t(s, k);
          if (c < best) {
            best = c;
            bm = s;
          }
        }
        t(l, k) = best;
        m(l, k) = bm;
      }
    }
  }
};

// The same T in closed form (binomial checkpointing; it equals the dynamic programme, which the tests
// check): with c = k + 1 states and r the least integer with l <= C(c + r - 1, c),
// T(l, k) = r l - C(c + r - 1, c + 1). Used where the table would be too large (l above kTableMax).
constexpr int kTableMax = 4096;

int64_t binom_sat(int64_t n, int64_t k) {  // C(n, k), saturating at 2^62
  if (k < 0 || k > n) return 0;
  k = std::min(k, n - k);
  long double v = 1;
  for (int64_t i = 1; i <= k; ++i) {
    v = v * (long double)(n - k + i) / (long double)i;
    if (v > 4.6e18L) return int64_t(1) << 62;
  }
  return (int64_t)(v + 0.5L);
}

int64_t ckpt_closed(int64_t l, int k) {
  if (l <= 1) return l;
  const int64_t c = k + 1;
  int64_t r = 1;
  while (binom_sat(c + r - 1, c) < l) ++r;
  return r * l - binom_sat(c + r - 1, c + 1);
}

// The optimal first split for (l, k): f(m) = m + T(l - m, k - 1) + T(m, k) is a sum of convex
// functions of m (T is piecewise linear with growing slopes), so its first minimum is the smallest m
// with f(m + 1) - f(m) >= 0, found by bisection.
int ckpt_split(int l, int k) {
  auto f = [&](int m) { return m + ckpt_closed(l - m, k - 1) + ckpt_closed(m, k); };
  int lo = 1, hi = l - 1;  // answer in [lo, hi]
  while (lo < hi) {
    const int mid = lo + (hi - lo) / 2;
    if (f(mid + 1) - f(mid) >= 0) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

int64_t halving_cost(int l) { return l <= 1 ? l : l / 2 + halving_cost(l - l / 2) + halving_cost(l / 2); }

int halving_depth(int l) { return l <= 1 ? 1 : 1 + std::max(halving_depth(l - l / 2), halving_depth(l / 2)); }

struct Checkpointer {
  fdtd_handle* h = nullptr;
  cudaStream_t st = nullptr;
  bool dry = false;         // count the schedule's forward steps without running anything
  int method;
  int nslots;
  CkptTable tab;
  std::vector<float*> slot;
  int64_t slot_floats = 0;
  int pos = -1;             // step index of the state held in the solver's current buffers
  int64_t fsteps = 0;       // forward steps evaluated
  int pb = 0;               // psi-bar ping-pong
  FwdArgs fa;
  RevArgs ra;
  PsiSet PEb[2], PHb[2];

  float* state_field() const { return h->fields + (int64_t)h->cur * 6 * h->g.vol; }
  void copy_state(float* dst_f, float* dst_e, float* dst_h, const float* src_f, const float* src_e, const float* src_h) {
    const int64_t pf = h->psi_floats();
    cudaMemcpyAsync(dst_f, src_f, 6 * h->g.vol * 4, cudaMemcpyDeviceToDevice, st);
    if (pf > 0) {
      cudaMemcpyAsync(dst_e, src_e, pf * 4, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(dst_h, src_h, pf * 4, cudaMemcpyDeviceToDevice, st);
    }
  }
  void save(int s) {
    if (dry) return;
    const int64_t pf = h->psi_floats(), V = 6 * h->g.vol;
    float* b = slot[s];
    copy_state(b, b + V, b + V + pf, state_field(), h->psiE + h->cur * pf, h->psiH + h->cur * pf);
  }
  void restore(int s, int step) {
    if (pos == step) return;
    if (dry) {
      pos = step;
      return;
    }
    const int64_t pf = h->psi_floats(), V = 6 * h->g.vol;
    const float* b = slot[s];
    copy_state(state_field(), h->psiE + h->cur * pf, h->psiH + h->cur * pf, b, b + V, b + V + pf);
    pos = step;
  }
  void advance_to(int target) {
    if (dry) {
      fsteps += std::max(0, target - pos);
      pos = std::max(pos, target);
      return;
    }
    const Geo& g = h->g;
    const int64_t pf = h->psi_floats();
    for (; pos < target; ++pos) {
      const int c = h->cur, x = 1 - c;
      fa.cur = h->F(c);
      fa.nxt = h->F(x);
      fa.psiE_cur = h->psi_set(h->psiE + c * pf);
      fa.psiE_nxt = h->psi_set(h->psiE + x * pf);
      fa.psiH_cur = h->psi_set(h->psiH + c * pf);
      fa.psiH_nxt = h->psi_set(h->psiH + x * pf);
      fa.step = pos;
      if (pos == target - 1)  // E^n of the step the next adjoint reverses, for the interpolated flux
        for (size_t q = 0; q < h->dets.size(); ++q)
          if (h->dets[q].kind == FDTD_DET_PLANE_FLUX_INTERP)
            launch_slab_copy(g, fa.cur, h->dets[q], 0, h->det_slab[q] + 2 * interp_slab_floats(h->dets[q]), st);
      for (const SrcDev& hs : h->hsrcs) launch_source(g, fa.cur, hs, pos, +1.f, 0, st);
      launch_fwd_fused(fa, h->fmaps[c], st);
      const Fields Fn = h->F(x);
      for (size_t q = kMaxSrc; q < h->srcs.size(); ++q) launch_source(g, Fn, h->srcs[q], pos, +1.f, 0, st);
      h->launches += 1 + (int64_t)h->hsrcs.size() + (int64_t)(h->srcs.size() > kMaxSrc ? h->srcs.size() - kMaxSrc : 0);
      h->cur = x;
      ++fsteps;
    }
  }
  void adjoint(int n) {  // the forward state after step n is current (E^n of it in the slabs)
    if (dry) return;
    const Fields F = h->F(), A = h->A();
    h->launches += enqueue_det_adjoint(h, F, A, n, 0, st);
    ra.F = F;
    ra.step = n;
    ra.pin = PEb[pb];
    ra.pout = PEb[1 - pb];
    launch_rev_E(ra, h->rmaps[h->cur], st);
    h->launches += enqueue_det_adjoint(h, F, A, n, 1, st, true);
    ra.pin = PHb[pb];
    ra.pout = PHb[1 - pb];
    launch_rev_H(ra, h->rmaps[h->cur], st);
    h->launches += enqueue_det_adjoint(h, F, A, n, 2, st);
    pb = 1 - pb;
    h->launches += 2;
  }
  // reverse steps [a, b); the state at a is in slot sa; slots from `top` up are free
  void reverse(int a, int b, int sa, int top) {
    const int l = b - a;
    if (l == 1) {
      restore(sa, a);
      advance_to(a + 1);
      adjoint(a);
      return;
    }
    const int kfree = nslots - top;
    if (kfree <= 0) {  // no free state: recompute each output from the range's start
      for (int i = b - 1; i >= a; --i) {
        restore(sa, a);
        advance_to(i + 1);
        adjoint(i);
      }
      return;
    }
    const int m = a + (method == 0 ? l / 2 : (tab.L > 0 ? tab.m(l, kfree) : ckpt_split(l, kfree)));
    restore(sa, a);
    advance_to(m);
    save(top);
    reverse(m, b, top, top + 1);
    reverse(a, m, sa, top);
  }
};

}  // namespace

int64_t fdtd_checkpoint_cost(int32_t nsteps, int32_t method, int32_t slots) {
  if (nsteps < 0 || (method != 0 && method != 1) || (method == 1 && slots < 1)) return -1;
  if (nsteps == 0) return 0;
  // run the schedule fdtd_backward_checkpointed runs, counting its forward steps
  Checkpointer C;
  C.dry = true;
  C.method = method;
  C.nslots = method == 0 ? halving_depth(nsteps) : slots;
  if (method == 1 && nsteps <= kTableMax) C.tab.build(nsteps, slots - 1);
  C.pos = 0;
  C.reverse(0, nsteps, 0, 1);
  return C.fsteps;
}

int fdtd_backward_checkpointed(fdtd_handle* h, const double* dL_ddet, float* dL_deps, int32_t method, int32_t slots,
                               int64_t* forward_steps) {
  NvtxRange range("fdtd_backward_checkpointed");
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (method != 0 && method != 1) return fail(FDTD_ERR_INVALID_ARG, "method must be 0 (halving) or 1 (treeverse)");
  if (method == 1 && slots < 1) return fail(FDTD_ERR_INVALID_ARG, "treeverse needs at least one state slot");
  if (h->last_nsteps < 0) return fail(FDTD_ERR_STATE, "no forward has run");
  const int nsteps = h->last_nsteps;
  const int64_t ndet = det_total_for(h, nsteps);
  if (ndet > 0 && !dL_ddet) return fail(FDTD_ERR_INVALID_ARG, "dL_ddet is NULL");
  const int64_t M = box_cells(h->design_lo, h->design_hi);
  if (M > 0 && !dL_deps) return fail(FDTD_ERR_INVALID_ARG, "dL_deps is NULL");
  if (!in_r_cells(h, h->design_lo, h->design_hi))
    return fail(FDTD_ERR_INVALID_ARG, "the design box must lie in the PML-free region");
  const Geo& g = h->g;
  const int64_t pf = h->psi_floats();
  TRY(ensure_adjoint(h));
  if (!h->psibar && pf > 0) TRY(dev_alloc(h, (void**)&h->psibar, 4 * pf * 4));
  if (!h->dLda && M > 0) TRY(dev_alloc(h, (void**)&h->dLda, M * 8));
  TRY(ensure_buf(h, &h->dLddet, &h->dLddet_cap, ndet, 8));
  if (M > 0) TRY(ensure_staging(h));
  TRY(ensure_gtab(h, nsteps));
  Checkpointer C;
  C.h = h;
  C.st = h->stream;
  C.method = method;
  C.nslots = method == 0 ? halving_depth(nsteps) : slots;
  if (method == 1 && nsteps <= kTableMax) C.tab.build(nsteps, slots - 1);
  C.slot_floats = 6 * g.vol + 2 * pf;
  C.slot.assign(C.nslots, nullptr);
  struct SlotGuard {  // frees the stored states on every way out (stream-ordered, after the work)
    Checkpointer& c;
    ~SlotGuard() {
      for (float*& b : c.slot) {
        dev_free(c.h, b, c.slot_floats * 4);
        b = nullptr;
      }
    }
  } guard{C};
  for (int s = 0; s < C.nslots; ++s) TRY(dev_alloc(h, (void**)&C.slot[s], C.slot_floats * 4));
  FwdArgs& fa = C.fa;
  fa.g = g;
  fa.T = h->tab();
  fa.a = h->a;
  fa.tz = h->tz;
  fa.nstage = h->fwd_nstage;
  fa.nsrc = (int)std::min<size_t>(h->srcs.size(), kMaxSrc);
  for (int q = 0; q < fa.nsrc; ++q) fa.src[q] = h->srcs[q];
  fa.ndet = 0;  // recomputed steps sample no detectors
  fa.det_out = h->det_out;
  fa.partial = h->partial;
  fa.status = h->status;
  RevArgs& ra = C.ra;
  ra.g = g;
  ra.T = h->tab();
  ra.B = h->A();
  ra.a = h->a;
  ra.tz = h->tz_rev;
  ra.nstage = h->rev_nstage;
  for (int d = 0; d < 3; ++d) {
    ra.dlo[d] = h->design_lo[d];
    ra.dhi[d] = h->design_hi[d];
  }
  ra.dLda = h->dLda;
  ra.inverse = 0;
  ra.nsrc = 0;  // sources only matter to the inverse step
  ra.ndet = 0;  // every detector adjoint by its own launch: rev_H of the next step runs on another state
  ra.status = h->status;
  for (int k = 0; k < 2; ++k) {
    C.PEb[k] = h->psi_set(h->psibar + (2 * k) * pf);
    C.PHb[k] = h->psi_set(h->psibar + (2 * k + 1) * pf);
  }
  if (ndet > 0) CK(cudaMemcpyAsync(h->dLddet, dL_ddet, ndet * 8, cudaMemcpyDefault, h->stream));
  CK(cudaMemsetAsync(h->adj, 0, 6 * g.vol * 4, h->stream));
  fill_canaries(h, false, true, false);
  if (pf > 0) CK(cudaMemsetAsync(h->psibar, 0, 4 * pf * 4, h->stream));
  if (M > 0) CK(cudaMemsetAsync(h->dLda, 0, M * 8, h->stream));
  TRY(reset_state(h));
  C.pos = 0;
  if (nsteps > 0) {
    C.save(0);
    C.reverse(0, nsteps, 0, 1);
  }
  if (nsteps > 0) {  // the non-finite check of the adjoint fields
    launch_check_finite(g, h->adj, 6 * g.vol, h->status, h->nsm, h->stream);
    h->launches += 1;
  }
  if (M > 0) {
    launch_grad_finalize(g, h->a, h->design_lo, h->design_hi, h->dLda, h->staging, 1.0, h->stream);
    h->launches += 1;
    CK(cudaMemcpyAsync(dL_deps, h->staging, M * 4, cudaMemcpyDefault, h->stream));
  }
  CK(cudaGetLastError());
  h->recorded = false;
  if (forward_steps) *forward_steps = C.fsteps;
  return sync_status(h);
}

int fdtd_backward_density(fdtd_handle* h, const double* dL_ddet, float* dL_drho) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (!h->density) return fail(FDTD_ERR_STATE, "no design density was set");
  return backward_scaled(h, dL_ddet, dL_drho, h->eps_hi - h->eps_lo);
}

int fdtd_set_design_density(fdtd_handle* h, const float* rho_box, double eps_lo, double eps_hi) {
  if (!h || !rho_box) return fail(FDTD_ERR_INVALID_ARG, "NULL argument");
  if (!(eps_lo > 0.0) || !(eps_hi > 0.0)) return fail(FDTD_ERR_INVALID_ARG, "eps_lo and eps_hi must be positive");
  const int64_t m = box_cells(h->design_lo, h->design_hi);
  h->density = true;
  h->eps_lo = eps_lo;
  h->eps_hi = eps_hi;
  if (m == 0) return FDTD_OK;
  TRY(ensure_staging(h));
  CK(cudaMemcpyAsync(h->staging, rho_box, m * 4, cudaMemcpyDefault, h->stream));
  launch_set_density(h->g, h->a, h->design_lo, h->design_hi, h->staging, (float)eps_lo, (float)(eps_hi - eps_lo),
                     h->stream);
  h->launches += 1;
  CK(cudaGetLastError());
  return FDTD_OK;
}

int fdtd_design_adam_step(fdtd_handle* h, const float* dL_drho, float* theta, float* m, float* v, float* rho_out,
                          int32_t t, double lr, double beta1, double beta2, double eps, double proj_beta,
                          double proj_eta) {
  if (!h || !dL_drho || !theta || !m || !v || !rho_out) return fail(FDTD_ERR_INVALID_ARG, "NULL argument");
  if (is_host_pointer(dL_drho) || is_host_pointer(theta) || is_host_pointer(m) || is_host_pointer(v) ||
      is_host_pointer(rho_out))
    return fail(FDTD_ERR_INVALID_ARG, "the design-loop arrays must be device memory");
  if (t < 1 || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) ||
      !(proj_beta >= 0.0) || !(proj_eta > 0.0 && proj_eta < 1.0))
    return fail(FDTD_ERR_INVALID_ARG, "design step: need t >= 1, lr > 0, beta1/beta2 in [0, 1), eps > 0, "
                                      "proj_beta >= 0, proj_eta in (0, 1)");
  const int64_t n = box_cells(h->design_lo, h->design_hi);
  launch_design_adam(dL_drho, theta, m, v, rho_out, n, t, lr, beta1, beta2, eps, proj_beta, proj_eta, h->stream);
  if (n > 0) h->launches += 1;
  CK(cudaGetLastError());
  return FDTD_OK;
}

int fdtd_design_project(fdtd_handle* h, const float* theta, float* rho_out, double proj_beta, double proj_eta) {
  if (!h || !theta || !rho_out) return fail(FDTD_ERR_INVALID_ARG, "NULL argument");
  if (is_host_pointer(theta) || is_host_pointer(rho_out))
    return fail(FDTD_ERR_INVALID_ARG, "the design-loop arrays must be device memory");
  if (!(proj_beta >= 0.0) || !(proj_eta > 0.0 && proj_eta < 1.0))
    return fail(FDTD_ERR_INVALID_ARG, "projection: need proj_beta >= 0 and proj_eta in (0, 1)");
  const int64_t n = box_cells(h->design_lo, h->design_hi);
  launch_design_project(theta, rho_out, n, proj_beta, proj_eta, h->stream);
  if (n > 0) h->launches += 1;
  CK(cudaGetLastError());
  return FDTD_OK;
}

int fdtd_read_detectors(fdtd_handle* h, double* out) {
  if (!h || !out) return fail(FDTD_ERR_INVALID_ARG, "NULL argument");
  if (h->last_nsteps < 0) return fail(FDTD_ERR_STATE, "no forward has run");
  const int64_t n = det_total_for(h, h->last_nsteps);
  if (n == 0) return FDTD_OK;
  CK(cudaMemcpyAsync(out, h->det_out, n * 8, cudaMemcpyDefault, h->stream));
  if (is_host_pointer(out)) return sync_status(h);
  return FDTD_OK;
}

int64_t fdtd_detector_size(fdtd_handle* h, int32_t idx) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (idx < 0 || idx >= (int32_t)h->dets.size()) return fail(FDTD_ERR_INVALID_ARG, "detector %d does not exist", idx);
  const DetDev& d = h->dets[idx];
  const bool per_cell = d.kind == FDTD_DET_PLANE_E2_SUM || d.kind == FDTD_DET_PLANE_E2_SUM_INTERP;
  return per_cell ? box_cells(d.lo, d.hi) : (h->last_nsteps < 0 ? 0 : h->last_nsteps);
}

int fdtd_read_detector(fdtd_handle* h, int32_t idx, double* out) {
  if (!h || !out) return fail(FDTD_ERR_INVALID_ARG, "NULL argument");
  if (idx < 0 || idx >= (int32_t)h->dets.size()) return fail(FDTD_ERR_INVALID_ARG, "detector %d does not exist", idx);
  if (h->last_nsteps < 0) return fail(FDTD_ERR_STATE, "no forward has run");
  const int64_t n = fdtd_detector_size(h, idx);
  if (n == 0) return FDTD_OK;
  CK(cudaMemcpyAsync(out, h->det_out + h->dets[idx].off, n * 8, cudaMemcpyDefault, h->stream));
  if (is_host_pointer(out)) return sync_status(h);
  return FDTD_OK;
}

int64_t fdtd_detector_total(fdtd_handle* h) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  return det_total_for(h, h->last_nsteps < 0 ? 0 : h->last_nsteps);
}

int fdtd_get_fields(fdtd_handle* h, float* out6) {
  if (!h || !out6) return fail(FDTD_ERR_INVALID_ARG, "NULL argument");
  TRY(ensure_staging(h));
  launch_pack_fields(h->g, h->F(), h->staging, 0, h->stream);
  h->launches += 1;
  const int64_t N = (int64_t)h->g.n[0] * h->g.n[1] * h->g.n[2];
  CK(cudaMemcpyAsync(out6, h->staging, 6 * N * 4, cudaMemcpyDefault, h->stream));
  return sync_status(h);
}

int fdtd_fields(fdtd_handle* h, float* out6) { return fdtd_get_fields(h, out6); }

int64_t fdtd_bytes_allocated(fdtd_handle* h) { return h ? h->bytes : -1; }

int64_t fdtd_launch_count(fdtd_handle* h) { return h ? h->launches : -1; }

int fdtd_profile(fdtd_handle* h, int32_t enable, int32_t every) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (enable && every < 1) return fail(FDTD_ERR_INVALID_ARG, "every must be >= 1");
  if (h->gfwd.pending || h->gbwd.pending) TRY(prof_collect(h));
  h->prof_every = enable ? every : 0;
  for (int k = 0; k < FDTD_KERNEL_KINDS; ++k) {
    h->prof_ms[k] = 0;
    h->prof_n[k] = 0;
  }
  return FDTD_OK;
}

int fdtd_profile_read(fdtd_handle* h, double* ms, int64_t* count, int32_t nkinds) {
  if (!h || nkinds < 0) return fail(FDTD_ERR_INVALID_ARG, "bad argument");
  TRY(prof_collect(h));
  for (int k = 0; k < nkinds && k < FDTD_KERNEL_KINDS; ++k) {
    if (ms) ms[k] = h->prof_ms[k];
    if (count) count[k] = h->prof_n[k];
  }
  return FDTD_OK;
}

int fdtd_release_history(fdtd_handle* h) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  dev_free(h, h->face_hist, h->face_cap_steps * h->faces.per_step * 4);
  h->face_hist = nullptr;
  h->face_cap_steps = 0;
  dev_free(h, h->seg_states, h->seg_cap * h->state_floats() * 4);
  h->seg_states = nullptr;
  h->seg_cap = 0;
  // the adjoint state too (allocated again by the next reverse sweep)
  const int64_t pf = h->psi_floats();
  dev_free(h, h->adj, 12 * h->g.vol * 4);
  h->adj = nullptr;
  dev_free(h, h->psibar, pf > 0 ? 4 * pf * 4 : 0);
  h->psibar = nullptr;
  h->recorded = false;
  return FDTD_OK;
}

int fdtd_set_segment_steps(fdtd_handle* h, int32_t steps) {
  if (!h || steps < 0) return fail(FDTD_ERR_INVALID_ARG, "NULL handle or negative segment length");
  h->seg_steps = steps;
  h->recorded = false;  // a history recorded with the old setting is not used
  return FDTD_OK;
}

int fdtd_reverse_kind(const fdtd_grid* grid, const fdtd_pml* pml) {
  if (validate(grid, 0.5, pml) != FDTD_OK) return FDTD_ERR_INVALID_ARG;
  return fused_reverse(make_geo(*grid, *pml, 0.5)) ? 1 : 0;
}

int fdtd_adjoint_frame(const fdtd_grid* grid, const fdtd_pml* pml, int32_t frame[4]) {
  if (!frame || validate(grid, 0.5, pml) != FDTD_OK) return FDTD_ERR_INVALID_ARG;
  int f[4];
  const bool ok = adjoint_frame(make_geo(*grid, *pml, 0.5), f);
  for (int q = 0; q < 4; ++q) frame[q] = f[q];
  return ok ? 1 : 0;
}

int64_t fdtd_adjoint_bytes(const fdtd_grid* grid, const fdtd_pml* pml) {
  if (validate(grid, 0.5, pml) != FDTD_OK) return -1;
  const Geo g = make_geo(*grid, *pml, 0.5);
  return 12 * g.vol * 4 + 4 * psi_bytes(g);
}

int64_t fdtd_history_bytes(const fdtd_grid* grid, const fdtd_pml* pml, int32_t nsteps, int32_t segment_steps) {
  if (validate(grid, 0.5, pml) != FDTD_OK || nsteps < 0 || segment_steps < 0) return -1;
  const Geo g = make_geo(*grid, *pml, 0.5);
  const int64_t per_step = make_faces(g).per_step * 4;
  if (segment_steps == 0 || nsteps <= segment_steps) return per_step * nsteps;
  const int64_t S = (nsteps + segment_steps - 1) / segment_steps;
  const int64_t state = (6 * g.vol + 2 * (psi_bytes(g) / 4)) * 4;
  return per_step * segment_steps + std::max<int64_t>(0, S - 2) * state;
}

int fdtd_wait_probe(int32_t limit_ms, int64_t* waited_ns) {
  if (limit_ms < 1 || limit_ms > 2000 || !waited_ns)
    return fail(FDTD_ERR_INVALID_ARG, "limit_ms in 1..2000 and a waited_ns pointer");
  cudaStream_t st = nullptr;
  int* d_status = nullptr;
  unsigned long long* d_ns = nullptr;
  CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaError_t e = cudaMallocAsync(&d_status, 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_ns, 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, 4, st);
  if (e == cudaSuccess) {
    launch_wait_probe(d_status, d_ns, (unsigned long long)limit_ms * 1000000ull, st);
    e = cudaGetLastError();
  }
  int status = 0;
  unsigned long long ns = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_status, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, d_ns, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (d_status) cudaFreeAsync(d_status, st);
  if (d_ns) cudaFreeAsync(d_ns, st);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (e != cudaSuccess) return fail(FDTD_ERR_CUDA, "wait probe: %s", cudaGetErrorString(e));
  *waited_ns = (int64_t)ns;
  if (status & kStatusTimeout) return fail(FDTD_ERR_TIMEOUT, "the probe's bounded wait gave up after %lld ns", (long long)ns);
  return FDTD_OK;
}

int fdtd_synchronize(fdtd_handle* h) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  return sync_status(h);
}

int fdtd_set_canaries(fdtd_handle* h, int32_t enable) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  h->canary = enable != 0;
  const int64_t rows = (int64_t)h->g.n[1] * h->g.n[2];
  if (h->canary) fill_canaries(h, true, true, true);
  else {  // back to zero padding
    launch_fill_padding(h->g, h->fields, 12 * rows, h->g.n[0], 0.f, h->nsm, h->stream);
    if (h->adj) launch_fill_padding(h->g, h->adj, 12 * rows, h->g.n[0], 0.f, h->nsm, h->stream);
    launch_fill_padding(h->g, h->a, rows, h->g.n[0], 0.f, h->nsm, h->stream);
  }
  CK(cudaGetLastError());
  return FDTD_OK;
}

int fdtd_check_canaries(fdtd_handle* h, int64_t* overwritten) {
  if (!h || !overwritten) return fail(FDTD_ERR_INVALID_ARG, "NULL handle or output");
  if (!h->canary) return fail(FDTD_ERR_STATE, "canaries are off");
  TRY(ensure_staging(h));
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(h->staging);
  CK(cudaMemsetAsync(cnt, 0, 8, h->stream));
  const int64_t rows = (int64_t)h->g.n[1] * h->g.n[2];
  launch_count_padding(h->g, h->fields, 12 * rows, field_canary_x0(h), cnt, h->nsm, h->stream);
  if (h->adj) launch_count_padding(h->g, h->adj, 12 * rows, h->g.n[0], cnt, h->nsm, h->stream);
  launch_count_padding(h->g, h->a, rows, h->g.n[0], cnt, h->nsm, h->stream);
  unsigned long long c = 0;
  CK(cudaMemcpyAsync(&c, cnt, 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *overwritten = (int64_t)c;
  return FDTD_OK;
}

int fdtd_set_graphs(fdtd_handle* h, int32_t enable) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  h->use_graphs = enable != 0;
  return FDTD_OK;
}

int fdtd_set_face_overlap(fdtd_handle* h, int32_t enable) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  h->face_overlap = enable != 0;
  return FDTD_OK;
}

int fdtd_set_check_interval(fdtd_handle* h, int32_t every) {
  if (!h) return fail(FDTD_ERR_INVALID_ARG, "NULL handle");
  if (every < 0) return fail(FDTD_ERR_INVALID_ARG, "every must be >= 0");
  h->check_every = every;
  return FDTD_OK;
}

}  // extern "C"
