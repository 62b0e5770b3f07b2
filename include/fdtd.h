/*
 * fdtd.h: C ABI of the B300 (sm_103a) time-reversible 3D FDTD library (libfdtd.so).
 *
 * The library runs the Yee-grid leapfrog of arXiv 2412.12360 Sec. 2.1 (Faraday Eq. 1 and Ampere
 * Eq. 2 as curl stencils with a per-cell inverse permittivity, a convolutional PML on the outer
 * faces, soft sources and time-integrated detectors) and the reverse-mode gradient of Sec. 2.2:
 * the inverse update step rebuilds the fields backward in time from t+1 to t inside the PML-free
 * region, the tangential H on the six planes enclosing that region is recorded every forward step
 * and replayed in reverse, and adjoint fields are swept alongside to accumulate dL/d(eps) per
 * design cell.
 *
 * Units and conventions (the paper prints only Eqs. 1-2; these are this library's readings):
 *   - normalised units: c = 1, grid spacing 1, H stored as eta0 * H, mu = 1;
 *   - courant = S = c dt / dx, stable for S <= 1/sqrt(3);
 *   - cell (i, j, k), x fastest; Ex at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at (i, j, k+1/2),
 *     Hx at (i, j+1/2, k+1/2), Hy at (i+1/2, j, k+1/2), Hz at (i+1/2, j+1/2, k);
 *   - field order Ex, Ey, Ez, Hx, Hy, Hz; PEC at integer planes 0 and N of every axis;
 *   - one inverse permittivity per cell, applied to that cell's Ex, Ey, Ez;
 *   - CPML: sigma = sigma_max (d/p)^m, kappa = 1 + (kappa_max - 1)(d/p)^m, alpha = alpha_max (1 - d/p),
 *     b = exp(-(sigma/kappa + alpha)), c = sigma / (sigma kappa + kappa^2 alpha) (b - 1), d the depth
 *     of the component's own position into the layer, psi <- b psi + c * difference;
 *   - source waveform g(s) = sin(2 pi (s - t0)/P) exp(-((s - t0)/tau)^2), P = wavelength / S steps,
 *     sampled at s = n + 1/2 and added to E after the E update of step n;
 *   - detectors sample E^{n+1} and H^{n+1/2} after every step n (no interpolation).
 *
 * Memory: every pointer argument marked "host or device" may point to host memory or to device
 * memory of the current CUDA device (the library copies with cudaMemcpyDefault). The handle owns all
 * the device memory it allocates; inputs are copied, outputs are written into caller buffers.
 *
 * Streams: work is enqueued on the stream given at creation (NULL = legacy default stream). Calls
 * that return data to a host pointer synchronise that stream before returning.
 *
 * Errors: every int-returning call returns FDTD_OK (0) or a negative FDTD_ERR_* code and never
 * aborts; fdtd_last_error() gives a message for the calling thread's last failure.
 */
#ifndef FDTD_H_
#define FDTD_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDTD_OK 0
#define FDTD_ERR_INVALID_ARG (-1)
#define FDTD_ERR_UNSTABLE (-2)     /* courant above 1/sqrt(3) */
#define FDTD_ERR_OOM (-3)          /* device allocation failed or a byte budget would be exceeded */
#define FDTD_ERR_CUDA (-4)         /* a CUDA runtime call failed */
#define FDTD_ERR_STATE (-5)        /* call out of order, e.g. backward without a recorded forward */
#define FDTD_ERR_NONFINITE (-6)    /* a non-finite value was found in the fields */
#define FDTD_ERR_TIMEOUT (-7)      /* a bounded device-side wait gave up */

/* fdtd_forward flags */
#define FDTD_RECORD_FACES 1u       /* keep the boundary-face history needed by fdtd_backward */

/* detector kinds */
#define FDTD_DET_POINT_SERIES 0    /* field `component` (0..5) at cell lo, one value per step */
#define FDTD_DET_PLANE_E2_SUM 1    /* per cell of [lo, hi): sum over steps of Ex^2 + Ey^2 + Ez^2 */
#define FDTD_DET_PLANE_FLUX 2      /* per step: sum over [lo, hi) of (E x H)[axis] */
/* Interpolated forms (Sec. 2.1: composite metrics need the staggered components brought to one point
 * in space and time; the paper's evaluation mode). Every component is taken at the cell centre: E_c
 * as the mean of its 4 values around it (offsets 0/1 along the two axes other than c), H_c as the
 * mean of its 2 values (offsets 0/1 along c); the box plus one cell along each axis must lie in the
 * grid (and, for a gradient, in the PML-free region). */
#define FDTD_DET_PLANE_E2_SUM_INTERP 3  /* per cell of [lo, hi): sum over steps of |E^{n+1}(centre)|^2 */
#define FDTD_DET_PLANE_FLUX_INTERP 4    /* per step: sum over [lo, hi) of (E^{n+1/2} x H^{n+1/2})[axis] at the
                                         * centres, E^{n+1/2} = (E^n + E^{n+1}) / 2 */

typedef struct fdtd_handle fdtd_handle;

typedef struct {
  int32_t nx, ny, nz;              /* cells per axis, each >= 2 */
} fdtd_grid;

typedef struct {
  int32_t thickness[6];            /* cells: x-lo, x-hi, y-lo, y-hi, z-lo, z-hi; 0 = bare PEC wall */
  double sigma_max;                /* normalised peak conductivity (sigma dt / eps0) */
  double kappa_max;                /* >= 1 */
  double alpha_max;                /* normalised, >= 0 */
  int32_t grading_m;               /* polynomial grading order, >= 1 */
} fdtd_pml;

/* Source on an E component over the cell box [lo, hi) (Sec. 2.1). Two kinds:
 *   tfsf = 0: additive soft source, E_c += amplitude * profile * g(n + 1/2) after the E update of
 *     step n, g the Gaussian-modulated sine below.
 *   tfsf = +-(d + 1): the plane of a total-field / scattered-field source (Sec. 2.1: the incident
 *     field enters on one side only), a plane wave travelling along axis d in the direction of the
 *     sign. The box must be one cell thick along d (plane index k) and `component` transverse to d.
 *     The incident field is that of a one-dimensional Yee line along d (same Courant number,
 *     permittivity eps_background) driven by a soft source amplitude * g(n + 1/2) on its E four
 *     cells upstream of the plane. E_c on plane k is total field; the H component h (the third
 *     axis) on the adjacent half plane (k - 1/2 for +, k + 1/2 for -) is scattered field, and each
 *     gets the incident value of the other side as a correction, weighted by the profile:
 *       H_h += dir S sH Einc^n(k)  after the H update,  E_c += -dir S a sE Hinc^{n+1/2}  after the E
 *     update, with sE, sH = +-1 the signs of the axis-d derivatives in (curl H)_c and (curl E)_h.
 *     Requires k >= 1 (+) or k <= n_d - 2 (-), and the plane and its H half plane outside the design
 *     box (the E correction uses a there, taken at creation).
 * g(s) = sin(2 pi (s - t0) S / lambda) exp(-((s - t0) / tau)^2), s in steps. */
typedef struct {
  int32_t component;               /* 0, 1, 2 = Ex, Ey, Ez */
  int32_t lo[3], hi[3];            /* cell box, hi exclusive */
  const float* profile;            /* host, box-shaped weights (x fastest) or NULL for 1 */
  double amplitude;
  double wavelength_cells;         /* vacuum wavelength in cells */
  double tau_steps;                /* width of the Gaussian envelope, steps (> 0) */
  double t0_steps;                 /* centre of the envelope, steps */
  int32_t tfsf;                    /* 0 = soft source; +-(axis + 1) = TFSF plane, direction of travel */
  double eps_background;           /* TFSF: permittivity of the incident-field line (> 0) */
} fdtd_source;

/* Detector (Sec. 2.1: detectors record field values at intermediate time steps; composite values
 * use same-index components without interpolation, or the interpolated kinds above). Output sizes:
 * POINT_SERIES and the PLANE_FLUX kinds give nsteps doubles, the PLANE_E2_SUM kinds one double per box
 * cell (x fastest). */
typedef struct {
  int32_t kind;                    /* FDTD_DET_* */
  int32_t component;               /* POINT_SERIES: 0..5 = Ex..Hz */
  int32_t axis;                    /* PLANE_FLUX: normal axis 0, 1, 2 */
  int32_t lo[3], hi[3];            /* cell box, hi exclusive */
} fdtd_detector;

/* Create a solver (Sec. 2.1). eps_inv: host or device, nx*ny*nz floats (x fastest), copied.
 * design_lo/hi: the cell box [lo, hi) whose dL/d(eps) fdtd_backward returns (may be empty).
 * spacing: metres per cell, recorded for reporting only (all arithmetic is in cells).
 * When backward is wanted, detectors and the design box must lie in the PML-free cell box
 * [thickness_lo, n - thickness_hi) of every axis; fdtd_forward with FDTD_RECORD_FACES checks this.
 * Returns INVALID_ARG for malformed input, UNSTABLE for courant > 1/sqrt(3), OOM, CUDA. */
int fdtd_create(fdtd_handle** out, const fdtd_grid* grid, double spacing, double courant,
                const float* eps_inv, const fdtd_source* src, int32_t nsrc, const fdtd_detector* det,
                int32_t ndet, const fdtd_pml* pml, const int32_t design_lo[3], const int32_t design_hi[3],
                void* cuda_stream);

/* Free every device buffer of the handle, in stream order after the work already enqueued on its stream
 * (a handle whose time loops were captured into CUDA graphs first waits for that work). NULL is
 * accepted. */
int fdtd_destroy(fdtd_handle* h);

/* Replace the inverse permittivity on the design box (host or device, box-shaped, x fastest). */
int fdtd_set_design_eps_inv(fdtd_handle* h, const float* eps_inv_box);

/* Design parametrisation eps = eps_lo + (eps_hi - eps_lo) rho on the design box (the density form of
 * the paper's design regions, Sec. 3.2-3.3): sets a = 1/eps from rho (host or device, box-shaped
 * floats in [0, 1], x fastest), with eps rounded to float before the reciprocal. */
int fdtd_set_design_density(fdtd_handle* h, const float* rho_box, double eps_lo, double eps_hi);

/* As fdtd_backward, but writes dL/drho = (eps_hi - eps_lo) dL/deps for the parametrisation of the
 * last fdtd_set_design_density (STATE if there was none). */
int fdtd_backward_density(fdtd_handle* h, const double* dL_ddet, float* dL_drho);

/* One step of the inverse-design loop that drives the forward and gradient solves (Sec. 3.2-3.3:
 * gradient-based optimisation of a design quantised to two materials). The design densities are
 * rho = P(theta), the smoothed Heaviside projection of latent variables theta in [0, 1] that pushes
 * rho towards 0 or 1 as proj_beta grows (binarisation; proj_beta = 0 is the identity):
 *   P(theta) = (tanh(beta eta) + tanh(beta (theta - eta))) / (tanh(beta eta) + tanh(beta (1 - eta))).
 * Given dL/drho at rho = P(theta) (from fdtd_backward_density), the step is Adam (Kingma and Ba):
 *   g = dL/drho P'(theta); m = beta1 m + (1 - beta1) g; v = beta2 v + (1 - beta2) g^2;
 *   theta -= lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps), then clamped to [0, 1];
 *   rho_out = P(theta).
 * All five arrays are DEVICE pointers of design-box cells (x fastest, fp32): dL_drho is read,
 * theta, m and v are updated in place, rho_out is written (it may alias nothing else). The work is
 * enqueued on the solver's stream; t >= 1 is the step count. INVALID_ARG on a NULL or host pointer,
 * t < 1, lr <= 0, beta1 or beta2 outside [0, 1), eps <= 0, proj_beta < 0 or proj_eta outside (0, 1). */
int fdtd_design_adam_step(fdtd_handle* h, const float* dL_drho, float* theta, float* m, float* v, float* rho_out,
                          int32_t t, double lr, double beta1, double beta2, double eps, double proj_beta,
                          double proj_eta);

/* Sec. 2.2's checkpointing alternative to time reversal (for comparison): the same gradient as
 * fdtd_backward for the last forward, but the forward state each adjoint step needs is recomputed
 * from full stored states (fields and CPML memories) instead of rebuilt by the inverse step; no face
 * record is used. method 0: recursive halving (ceil(log2 n) + 1 stored states, (n/2) log2 n extra
 * forward steps for n = 2^j); method 1: treeverse / binomial checkpointing with `slots` stored states
 * (the schedule minimising the forward steps: by dynamic programming up to 4096 steps, from the
 * equal binomial closed form beyond). Each adjoint step re-evaluates
 * its own forward step from its input state, as in revolve. dL_ddet and dL_deps as in fdtd_backward;
 * forward_steps (may be NULL) receives the forward steps evaluated. The stored states are allocated
 * for the call and freed before it returns; afterwards the solver's fields hold an intermediate state.
 * STATE if no forward has run; INVALID_ARG for a bad method, slots < 1 (method 1), a NULL output or a
 * design box in the PML. */
int fdtd_backward_checkpointed(fdtd_handle* h, const double* dL_ddet, float* dL_deps, int32_t method, int32_t slots,
                               int64_t* forward_steps);

/* Forward steps fdtd_backward_checkpointed evaluates for nsteps steps (host only, no GPU); -1 for bad
 * arguments. */
int64_t fdtd_checkpoint_cost(int32_t nsteps, int32_t method, int32_t slots);

/* rho_out = P(theta) with the projection of fdtd_design_adam_step (used when proj_beta changes between
 * steps, and for the first densities). theta and rho_out: DEVICE pointers of design-box cells, fp32,
 * enqueued on the solver's stream. INVALID_ARG on a NULL or host pointer, proj_beta < 0 or proj_eta
 * outside (0, 1). */
int fdtd_design_project(fdtd_handle* h, const float* theta, float* rho_out, double proj_beta, double proj_eta);

/* Set the initial state E^0, H^{-1/2} (host or device, 6*nx*ny*nz floats, field-major, x fastest);
 * NULL restores zero fields. Used for round-trip and eigenmode tests. */
int fdtd_set_initial_fields(fdtd_handle* h, const float* fields6);

/* Sec. 2.1: run nsteps steps from the initial state (a fresh solve each call). With
 * FDTD_RECORD_FACES the tangential H on the six planes enclosing the PML-free region is recorded
 * after every H update (Sec. 2.2), as needed by fdtd_backward. */
int fdtd_forward(fdtd_handle* h, int32_t nsteps, uint32_t flags);

/* Sec. 2.2: reverse-mode gradient of L = sum(dL_ddet * detectors) for the last forward.
 * dL_ddet: host or device, fdtd_detector_total(h) doubles (concatenated in detector order).
 * dL_deps: host or device, design-box-shaped floats (x fastest), written.
 * The primal fields are rebuilt by the inverse update step; after return the handle's fields hold
 * the reconstructed initial state on the PML-free region. STATE if the last forward did not record
 * faces or a backward already consumed it. */
int fdtd_backward(fdtd_handle* h, const double* dL_ddet, float* dL_deps);

/* ---- Grouped forms: several solves advanced by one launch per kernel and time step --------------
 * For serving and batching (the optimisation loops of Sec. 3.2-3.3 solve many designs). The math is
 * that of fdtd_forward / fdtd_backward, so each handle's detectors and dL/deps are bitwise the same
 * as when it is solved alone; what changes is that one launch of the fused forward (or inverse, or
 * adjoint) kernel covers the blocks of every handle of the group, so small grids share the GPU
 * instead of queueing for it. A solve is started with fdtd_begin, its forward advanced by
 * fdtd_group_step until its phase is FDTD_PHASE_FORWARD_DONE (detectors readable), its reverse
 * sweep started with fdtd_begin_backward and advanced the same way until FDTD_PHASE_DONE, and its
 * gradient read with fdtd_finish_backward. Handles may join a group at any step and in either phase
 * (continuous batching). Every handle of a group must have been created on the same stream; at most
 * FDTD_MAX_GROUP handles per call. Grouped steps launch directly (no CUDA graph) and copy the
 * boundary faces in line. */
#define FDTD_MAX_GROUP 8
#define FDTD_PHASE_IDLE 0          /* no incremental solve in progress */
#define FDTD_PHASE_FORWARD 1       /* forward steps remain */
#define FDTD_PHASE_FORWARD_DONE 2  /* the forward has finished: detectors readable, fdtd_begin_backward next */
#define FDTD_PHASE_BACKWARD 3      /* reverse steps remain */
#define FDTD_PHASE_DONE 4          /* the reverse sweep has finished: fdtd_finish_backward next */

/* Move the handle to another stream (NULL = legacy default stream): waits for the work already enqueued
 * on its current stream, then enqueues everything later on cuda_stream. A server creates and prepares
 * a handle on a private stream (set-up calls synchronise their stream) and then moves it onto the
 * stream its group runs on. */
int fdtd_set_stream(fdtd_handle* h, void* cuda_stream);

/* Report what the handle's kernels flagged (as fdtd_synchronize: FDTD_ERR_TIMEOUT, FDTD_ERR_NONFINITE,
 * and clear it) without waiting for the handle's stream: the caller has made sure that the handle's
 * work has completed (an event recorded after it has fired), so that other handles sharing the stream
 * keep running. */
int fdtd_poll_status(fdtd_handle* h);

/* Start a forward solve of nsteps steps (flags as fdtd_forward) that fdtd_group_step advances; no step
 * runs here. INVALID_ARG as fdtd_forward. */
int fdtd_begin(fdtd_handle* h, int32_t nsteps, uint32_t flags);

/* Start the reverse sweep (Sec. 2.2) of a finished recorded forward begun with fdtd_begin; dL_ddet as in
 * fdtd_backward. STATE unless the phase is FDTD_PHASE_FORWARD_DONE and the forward recorded faces. */
int fdtd_begin_backward(fdtd_handle* h, const double* dL_ddet);

/* Advance each of the n handles by up to nsteps steps of its current phase (forward steps, or reverse
 * steps), with one launch per kernel and step for all of them; handles that finish their phase
 * meanwhile drop out of the later steps, handles in another phase are left alone. Enqueued on the
 * handles' common stream; no synchronisation. INVALID_ARG for n outside 1..FDTD_MAX_GROUP, NULL or
 * repeated handles, handles on different streams or nsteps < 0. */
int fdtd_group_step(fdtd_handle* const* hs, int32_t n, int32_t nsteps);

/* The handle's phase (FDTD_PHASE_*) and the steps its phase has left (either may be NULL). */
int fdtd_phase(fdtd_handle* h, int32_t* phase, int32_t* steps_left);

/* Write dL/deps (fdtd_finish_backward) or dL/drho for the density of the last fdtd_set_design_density
 * (fdtd_finish_backward_density) of a finished reverse sweep; host or device buffer as fdtd_backward.
 * Returns the handle to FDTD_PHASE_IDLE. STATE unless the phase is FDTD_PHASE_DONE. */
int fdtd_finish_backward(fdtd_handle* h, float* dL_deps);
int fdtd_finish_backward_density(fdtd_handle* h, float* dL_drho);

/* Whole solves of a group: fdtd_begin of each handle (nsteps[i] steps, flags as fdtd_forward), then
 * grouped steps until every forward has finished (fdtd_group_forward); fdtd_begin_backward of each
 * handle, grouped steps until every reverse sweep has finished, and fdtd_finish_backward of each
 * (fdtd_group_backward, dL_ddet[i] and dL_deps[i] as in fdtd_backward). The handles' last forwards
 * may have different step counts. */
int fdtd_group_forward(fdtd_handle* const* hs, int32_t n, const int32_t* nsteps, uint32_t flags);
int fdtd_group_backward(fdtd_handle* const* hs, int32_t n, const double* const* dL_ddet, float* const* dL_deps);

/* Concatenated detector outputs of the last forward (host or device doubles). */
int fdtd_read_detectors(fdtd_handle* h, double* out);

/* Number of doubles fdtd_read_detectors writes for the last forward (or -1 on error). */
int64_t fdtd_detector_total(fdtd_handle* h);

/* The outputs of detector idx (0-based, in the order given to fdtd_create) of the last forward, into
 * a host or device buffer of fdtd_detector_size(h, idx) doubles: one value per step for the point and
 * flux kinds, one per box cell (x fastest) for the |E|^2 kinds. A host buffer waits for the stream
 * and reports as fdtd_synchronize does. INVALID_ARG for NULL or a bad idx, STATE before a forward. */
int fdtd_read_detector(fdtd_handle* h, int32_t idx, double* out);
int64_t fdtd_detector_size(fdtd_handle* h, int32_t idx);  /* -1 on error */

/* Current fields (host or device, 6*nx*ny*nz floats, field-major, x fastest, pitch removed).
 * fdtd_fields is the same call. */
int fdtd_get_fields(fdtd_handle* h, float* out6);
int fdtd_fields(fdtd_handle* h, float* out6);

/* Bytes of device memory a solve of this size needs (fields, coefficients, adjoint state and a
 * face history for nsteps when record_faces != 0); for admission by HBM footprint. -1 on bad input. */
int64_t fdtd_footprint_bytes(const fdtd_grid* grid, const fdtd_pml* pml, int32_t nsteps,
                             int32_t record_faces, const int32_t design_lo[3], const int32_t design_hi[3]);

/* Face-history segments (bounded memory for the reverse sweep of long or large solves): with steps = L > 0
 * a forward with FDTD_RECORD_FACES of T > L steps keeps the boundary faces (Sec. 2.2) of its last
 * segment only, the steps from (S - 1) L with S = ceil(T / L), and full states (fields and CPML
 * memories) at the starts L, 2L, .., (S - 2) L of the other segments; fdtd_backward then regenerates
 * each earlier segment's faces, when its reverse sweep reaches it, by running that segment's forward
 * again from its start state (the initial state for the first), which costs T - L extra forward steps
 * and leaves the gradient equal to the unsegmented one up to the rounding drift of the inverse step
 * (each segment's reverse sweep starts from the exact forward state). steps = 0 (the default) records
 * every step. Solves with segments run through fdtd_forward / fdtd_backward only (fdtd_begin refuses
 * them). INVALID_ARG for NULL or steps < 0. */
int fdtd_set_segment_steps(fdtd_handle* h, int32_t steps);

/* Bytes of the reverse sweep's history of a solve of nsteps steps with segment length segment_steps
 * (0: the whole face history): the face record it keeps plus the stored segment start states. -1 on
 * bad input. */
int64_t fdtd_history_bytes(const fdtd_grid* grid, const fdtd_pml* pml, int32_t nsteps, int32_t segment_steps);

/* Bytes of the reverse sweep's adjoint state (both adjoint field buffers and their CPML memories), part
 * of fdtd_footprint_bytes, held from a handle's first backward until fdtd_release_history. -1 on bad
 * input. */
int64_t fdtd_adjoint_bytes(const fdtd_grid* grid, const fdtd_pml* pml);

/* The launch plan fdtd_create chooses for a grid, computed on the host (no device work; the
 * environment overrides FDTD_REV_FUSED and FDTD_ADJ_SPLIT that fdtd_create reads are not applied).
 * fdtd_reverse_kind: 1 when the reverse sweep uses the fused pair (the inverse step, then the adjoint
 * step, each in one sweep with double-buffered fields: grids of at least 12 M cells whose 32 x 16
 * column tiles touch an x or y CPML layer in at most 40 % of the cases), 0 for the in-place pair.
 * fdtd_adjoint_frame: writes the frame of the fused adjoint step's tiles that need the x/y CPML loop,
 * frame[0..3] = leading and trailing tile columns, leading and trailing tile rows (32 x 16 tiles), and
 * returns 1 when a rectangle of plain tiles is left inside it (the step then runs as two launches, the
 * frame and the rectangle), 0 when not (one launch). Both: INVALID_ARG for a bad grid or pml (or a
 * NULL frame). */
int fdtd_reverse_kind(const fdtd_grid* grid, const fdtd_pml* pml);
int fdtd_adjoint_frame(const fdtd_grid* grid, const fdtd_pml* pml, int32_t frame[4]);

/* Cap the device bytes any one handle may allocate (-1 = no cap, the default). Allocations past the
 * cap fail with FDTD_ERR_OOM before reaching the CUDA allocator; used to exercise admission and
 * out-of-memory paths without exhausting the GPU. Process-wide. */
int fdtd_set_byte_budget(int64_t bytes);

/* Kernel kinds timed by fdtd_profile_read. */
#define FDTD_KERNEL_UPDATE_H 0     /* forward H half-step */
#define FDTD_KERNEL_UPDATE_E 1     /* forward E half-step */
#define FDTD_KERNEL_REV_E 2        /* reverse: inverse E, adjoint into H-bar, dL/da */
#define FDTD_KERNEL_REV_H 3        /* reverse: inverse H, adjoint into E-bar */
#define FDTD_KERNEL_FUSED_FWD 4    /* forward H and E of one step in one sweep */
#define FDTD_KERNEL_FUSED_REV 5    /* reverse step in one sweep */
#define FDTD_KERNEL_FACE_COPY 6    /* boundary-face record (forward) or replay (reverse) of one step */
#define FDTD_KERNEL_DET_ADJ 7      /* detector adjoints of one reverse step */
#define FDTD_KERNEL_INV_FUSED 8    /* reverse: inverse E and H of one step in one sweep, and dL/da */
#define FDTD_KERNEL_ADJ_FUSED 9    /* reverse: adjoint of one step (Hbar then Ebar) in one sweep */
#define FDTD_KERNEL_KINDS 10

/* Number of kernels this handle has launched since creation (or -1). */
int64_t fdtd_launch_count(fdtd_handle* h);

/* With enable != 0, fdtd_forward and fdtd_backward bracket every `every`-th launch of each stencil
 * kernel with CUDA events on the handle's stream; the events are read (waiting for the stream) at
 * the end of fdtd_backward, before a profiled time loop is replayed again, and by
 * fdtd_profile_read, which reports the device time of those launches. enable = 0 stops it and
 * clears the totals. */
int fdtd_profile(fdtd_handle* h, int32_t enable, int32_t every);

/* Per kernel kind (FDTD_KERNEL_*, up to nkinds): total device milliseconds of the timed launches
 * and how many were timed. Either array may be NULL. */
int fdtd_profile_read(fdtd_handle* h, double* ms, int64_t* count, int32_t nkinds);

/* Device bytes currently held by the handle (or -1). */
int64_t fdtd_bytes_allocated(fdtd_handle* h);

/* Free the reverse sweep's state of the handle (stream-ordered on the handle's stream): the boundary-face
 * history and segment start states of the last recorded forward, and the adjoint fields and their CPML
 * memories (allocated again by the next reverse sweep), for callers that solve many designs one after
 * another and cannot keep every history (batched gradients). A later fdtd_backward then fails with
 * FDTD_ERR_STATE until a new fdtd_forward with FDTD_RECORD_FACES. Returns FDTD_OK, or
 * FDTD_ERR_INVALID_ARG for NULL. */
int fdtd_release_history(fdtd_handle* h);

/* Allocation-free Poynting flux: out = sum over the cell box [lo, hi) of (E x H)[axis] for the fields
 * the caller passes. The paper has no counterpart; this is a library utility for callers that cannot
 * call cudaMalloc (hosts that give the library a fixed memory budget, real-time loops that must not
 * stall on an allocation). It allocates nothing: its partial sums live in a fixed device array of
 * 1024 doubles that the library reserves when it is loaded and that every GPU that loads the library
 * keeps until the process exits, so a box may hold at most 4194304 cells (larger boxes give
 * INVALID_ARG). The sum is a fixed-order two-pass FP64 reduction (per-block partial sums, then one
 * ordered sum): deterministic from call to call, equal to the solver's flux detector to rounding.
 *   fields6: device memory of the current device, 6*nx*ny*nz floats (Ex..Hz, field-major, x fastest,
 *            no row pitch: the layout fdtd_get_fields writes); not modified.
 *   out:     device memory of the current device, one double, written.
 * A host pointer or another GPU's buffer gives INVALID_ARG before anything is launched.
 * Work is enqueued on cuda_stream (NULL = legacy default stream); the call does not synchronise.
 * The first call on a device looks up the array's device address with that device current and keeps
 * it for the life of the process (a cudaDeviceReset after that is not supported). Every call shares
 * the array, so calls whose GPU work overlaps (other streams, other host threads) race and can
 * return wrong sums: serialise them. Each call writes every partial sum it reads, so the array
 * needs no clearing. */
int fdtd_plane_flux_noalloc(const float* fields6, const fdtd_grid* grid, int32_t axis, const int32_t lo[3],
                            const int32_t hi[3], double* out, void* cuda_stream);

/* Wait for all work of the handle's stream, then report what its kernels flagged since the last
 * report (and clear it): FDTD_ERR_TIMEOUT when a bounded device-side wait for a TMA copy gave up,
 * FDTD_ERR_NONFINITE when a field check found a NaN or an infinity (after which the fields, detector
 * outputs and gradients of that work are invalid; the handle stays usable). Calls that return
 * results into host buffers (fdtd_read_detectors, fdtd_backward, fdtd_get_fields, ...) wait and
 * report the same way. */
int fdtd_synchronize(fdtd_handle* h);

/* Diagnostic of the timeout path (failure detection without a fault). Every wait of the stencil
 * kernels for a TMA copy (an mbarrier phase) is bounded: it gives up after 1 s of the GPU's global
 * timer (or 2^30 polls), sets the handle's timeout status and lets the block finish, so a lost copy
 * ends as FDTD_ERR_TIMEOUT from fdtd_synchronize, not as a hang. This call runs that same bounded wait,
 * with a limit of limit_ms milliseconds (1..2000), in a one-block kernel on an mbarrier that nothing
 * arrives on, on a private stream of the current device, and waits for it. It returns FDTD_ERR_TIMEOUT
 * (the expected outcome) with *waited_ns the nanoseconds the wait lasted; FDTD_OK would mean the wait
 * returned without its phase completing. Allocates 12 bytes (stream-ordered) and frees them.
 * INVALID_ARG for a limit out of range or a NULL waited_ns. */
int fdtd_wait_probe(int32_t limit_ms, int64_t* waited_ns);

/* Where the face copies run (default 1): with enable != 0 the per-step face record (forward) and
 * replay (backward) are captured on a second stream beside the stencil kernels, which shortens a
 * step on small grids when the captured loop is replayed many times; with 0 they run in line on the
 * handle's stream, which keeps the captured graph smaller and cheaper to build, the better choice for
 * a handle that solves once (served requests). Results are the same either way. INVALID_ARG for NULL. */
int fdtd_set_face_overlap(fdtd_handle* h, int32_t enable);

/* How the time loops run (default 1): with enable != 0 each forward and backward loop is captured
 * once into a CUDA graph and replayed (the graph is rebuilt when the step count or the buffers
 * change); with 0 its kernels are launched directly on the stream, which spares building a graph
 * for a handle that solves once. Results are the same either way. INVALID_ARG for NULL. */
int fdtd_set_graphs(fdtd_handle* h, int32_t enable);

/* Non-finite field checks: every forward checks the fields after its last step, every backward the
 * rebuilt and the adjoint fields at its end (one read of the arrays, testing the exponent bits of
 * every value). With every > 0 the forward also checks
 * after every `every`-th step, so that a solve that has blown up is caught while it runs. The result
 * is reported by fdtd_synchronize. INVALID_ARG for NULL or every < 0. */
int fdtd_set_check_interval(fdtd_handle* h, int32_t every);

/* Debugging aid against out-of-row accesses. Every row of the field arrays (both buffers), the adjoint
 * fields and a is padded from nx to the pitch (a multiple of 32 cells); no kernel reads the padding
 * or writes it (but see odd nx below). With enable != 0 the padding holds NaN from now on (refilled whenever the arrays are
 * reset), so a kernel that read it would spread NaN into results (caught by the non-finite checks)
 * and one that wrote it leaves a non-NaN value, which fdtd_check_canaries counts (waits for the
 * stream; *overwritten = 0 when every canary is intact). Grids whose nx is a multiple of 32 have no
 * padding. For odd nx the forward kernel, which stores x-adjacent cell pairs, writes zeros into
 * column nx of the field arrays (never read), so their canaries start at column nx + 1.
 * enable = 0 puts zeros back. INVALID_ARG for NULL; fdtd_check_canaries: STATE when off. */
int fdtd_set_canaries(fdtd_handle* h, int32_t enable);
int fdtd_check_canaries(fdtd_handle* h, int64_t* overwritten);

/* Message for the calling thread's last failed call ("" if none). */
const char* fdtd_last_error(void);

/* Library version string. */
const char* fdtd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_H_ */
