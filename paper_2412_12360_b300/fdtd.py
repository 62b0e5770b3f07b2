"""ctypes binding of libfdtd (include/fdtd.h): argument marshalling only.

Every step of the solve runs in the CUDA library. The binding converts scenes, numpy arrays and
torch tensors into the C structures and pointers the ABI takes. Importing this module loads the
library and raises if it has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libfdtd.so")

FDTD_OK = 0
FDTD_ERR_INVALID_ARG = -1
FDTD_ERR_UNSTABLE = -2
FDTD_ERR_OOM = -3
FDTD_ERR_CUDA = -4
FDTD_ERR_STATE = -5
FDTD_ERR_NONFINITE = -6
FDTD_ERR_TIMEOUT = -7
FDTD_RECORD_FACES = 1
KERNEL_NAMES = ["update_H", "update_E", "rev_E", "rev_H", "fused_fwd", "fused_rev", "face_copy", "det_adj",
                "inv_fused", "adj_fused"]

MAX_GROUP = 8
PHASE_IDLE, PHASE_FORWARD, PHASE_FORWARD_DONE, PHASE_BACKWARD, PHASE_DONE = range(5)

ERROR_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "UNSTABLE", -3: "OOM", -4: "CUDA", -5: "STATE",
               -6: "NONFINITE", -7: "TIMEOUT"}


class FDTDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "?"), code, msg))
        self.code = code


class fdtd_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32)]


class fdtd_pml(C.Structure):
    _fields_ = [("thickness", C.c_int32 * 6), ("sigma_max", C.c_double), ("kappa_max", C.c_double),
                ("alpha_max", C.c_double), ("grading_m", C.c_int32)]


class fdtd_source(C.Structure):
    _fields_ = [("component", C.c_int32), ("lo", C.c_int32 * 3), ("hi", C.c_int32 * 3),
                ("profile", C.POINTER(C.c_float)), ("amplitude", C.c_double),
                ("wavelength_cells", C.c_double), ("tau_steps", C.c_double), ("t0_steps", C.c_double),
                ("tfsf", C.c_int32), ("eps_background", C.c_double)]


class fdtd_detector(C.Structure):
    _fields_ = [("kind", C.c_int32), ("component", C.c_int32), ("axis", C.c_int32),
                ("lo", C.c_int32 * 3), ("hi", C.c_int32 * 3)]


_VP = C.c_void_p
_I3 = C.c_int32 * 3

# (name, restype, argtypes) of every symbol include/fdtd.h declares
SIGNATURES = [
    ("fdtd_create", C.c_int, [C.POINTER(_VP), C.POINTER(fdtd_grid), C.c_double, C.c_double, _VP,
                              C.POINTER(fdtd_source), C.c_int32, C.POINTER(fdtd_detector), C.c_int32,
                              C.POINTER(fdtd_pml), _I3, _I3, _VP]),
    ("fdtd_destroy", C.c_int, [_VP]),
    ("fdtd_set_design_eps_inv", C.c_int, [_VP, _VP]),
    ("fdtd_set_initial_fields", C.c_int, [_VP, _VP]),
    ("fdtd_set_design_density", C.c_int, [_VP, _VP, C.c_double, C.c_double]),
    ("fdtd_backward_density", C.c_int, [_VP, _VP, _VP]),
    ("fdtd_design_project", C.c_int, [_VP, _VP, _VP, C.c_double, C.c_double]),
    ("fdtd_backward_checkpointed", C.c_int, [_VP, _VP, _VP, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]),
    ("fdtd_checkpoint_cost", C.c_int64, [C.c_int32, C.c_int32, C.c_int32]),
    ("fdtd_design_adam_step", C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, C.c_int32, C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_double, C.c_double]),
    ("fdtd_forward", C.c_int, [_VP, C.c_int32, C.c_uint32]),
    ("fdtd_backward", C.c_int, [_VP, _VP, _VP]),
    ("fdtd_read_detectors", C.c_int, [_VP, _VP]),
    ("fdtd_detector_total", C.c_int64, [_VP]),
    ("fdtd_get_fields", C.c_int, [_VP, _VP]),
    ("fdtd_fields", C.c_int, [_VP, _VP]),
    ("fdtd_read_detector", C.c_int, [_VP, C.c_int32, _VP]),
    ("fdtd_detector_size", C.c_int64, [_VP, C.c_int32]),
    ("fdtd_footprint_bytes", C.c_int64, [C.POINTER(fdtd_grid), C.POINTER(fdtd_pml), C.c_int32, C.c_int32,
                                         _I3, _I3]),
    ("fdtd_set_byte_budget", C.c_int, [C.c_int64]),
    ("fdtd_bytes_allocated", C.c_int64, [_VP]),
    ("fdtd_release_history", C.c_int, [_VP]),
    ("fdtd_launch_count", C.c_int64, [_VP]),
    ("fdtd_reverse_kind", C.c_int, [C.c_void_p, C.c_void_p]),
    ("fdtd_adjoint_frame", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    ("fdtd_wait_probe", C.c_int, [C.c_int32, C.POINTER(C.c_int64)]),
    ("fdtd_profile", C.c_int, [_VP, C.c_int32, C.c_int32]),
    ("fdtd_profile_read", C.c_int, [_VP, _VP, _VP, C.c_int32]),
    ("fdtd_plane_flux_noalloc", C.c_int, [_VP, C.POINTER(fdtd_grid), C.c_int32, _I3, _I3, _VP, _VP]),
    ("fdtd_synchronize", C.c_int, [_VP]),
    ("fdtd_set_stream", C.c_int, [_VP, _VP]),
    ("fdtd_poll_status", C.c_int, [_VP]),
    ("fdtd_set_segment_steps", C.c_int, [_VP, C.c_int32]),
    ("fdtd_adjoint_bytes", C.c_int64, [C.POINTER(fdtd_grid), C.POINTER(fdtd_pml)]),
    ("fdtd_history_bytes", C.c_int64, [C.POINTER(fdtd_grid), C.POINTER(fdtd_pml), C.c_int32, C.c_int32]),
    ("fdtd_begin", C.c_int, [_VP, C.c_int32, C.c_uint32]),
    ("fdtd_begin_backward", C.c_int, [_VP, _VP]),
    ("fdtd_group_step", C.c_int, [C.POINTER(_VP), C.c_int32, C.c_int32]),
    ("fdtd_phase", C.c_int, [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    ("fdtd_finish_backward", C.c_int, [_VP, _VP]),
    ("fdtd_finish_backward_density", C.c_int, [_VP, _VP]),
    ("fdtd_group_forward", C.c_int, [C.POINTER(_VP), C.c_int32, C.POINTER(C.c_int32), C.c_uint32]),
    ("fdtd_group_backward", C.c_int, [C.POINTER(_VP), C.c_int32, C.POINTER(_VP), C.POINTER(_VP)]),
    ("fdtd_set_check_interval", C.c_int, [_VP, C.c_int32]),
    ("fdtd_set_face_overlap", C.c_int, [_VP, C.c_int32]),
    ("fdtd_set_graphs", C.c_int, [_VP, C.c_int32]),
    ("fdtd_set_canaries", C.c_int, [_VP, C.c_int32]),
    ("fdtd_check_canaries", C.c_int, [_VP, C.POINTER(C.c_int64)]),
    ("fdtd_last_error", C.c_char_p, []),
    ("fdtd_version", C.c_char_p, []),
]

_lib = None


def lib():
    """The loaded libfdtd (raises if the in-tree build is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libfdtd.so is not built (%s); run __graft_entry__.build() or "
                              "python paper_2412_12360_b300/csrc/build.py" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().fdtd_last_error().decode()


def checkpoint_cost(nsteps: int, method: int, slots: int = 0) -> int:
    """Forward steps the checkpointing gradient evaluates (host only)."""
    return int(lib().fdtd_checkpoint_cost(int(nsteps), int(method), int(slots)))


def check(rc):
    if rc != FDTD_OK:
        raise FDTDError(rc, last_error())
    return rc


def _ptr(x):
    """Raw address of a numpy array or torch tensor (host or device), or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data


def make_grid(n):
    return fdtd_grid(int(n[0]), int(n[1]), int(n[2]))


def make_pml(scene):
    p = fdtd_pml()
    for f in range(6):
        p.thickness[f] = int(scene.pml[f])
    p.sigma_max = float(scene.sigma_max)
    p.kappa_max = float(scene.kappa_max)
    p.alpha_max = float(scene.alpha_max)
    p.grading_m = int(scene.grading_m)
    return p


def footprint_bytes(scene, nsteps: Optional[int] = None, record_faces: bool = True) -> int:
    g = make_grid(scene.n)
    p = make_pml(scene)
    ns = scene.nsteps if nsteps is None else nsteps
    return int(lib().fdtd_footprint_bytes(C.byref(g), C.byref(p), int(ns), int(record_faces),
                                          _I3(*scene.design_lo), _I3(*scene.design_hi)))


def history_bytes(scene, nsteps: Optional[int] = None, segment_steps: int = 0) -> int:
    """Device bytes of a solve's reverse-sweep history (faces kept plus segment start states)."""
    g = make_grid(scene.n)
    p = make_pml(scene)
    ns = scene.nsteps if nsteps is None else nsteps
    return int(lib().fdtd_history_bytes(C.byref(g), C.byref(p), int(ns), int(segment_steps)))


def adjoint_bytes(scene) -> int:
    """Device bytes of a handle's reverse-sweep adjoint state (freed by fdtd_release_history)."""
    g = make_grid(scene.n)
    p = make_pml(scene)
    return int(lib().fdtd_adjoint_bytes(C.byref(g), C.byref(p)))


def reverse_kind(scene) -> int:
    """1 when fdtd_create gives this scene's grid the fused reverse pair, 0 for the in-place pair."""
    g, p = make_grid(scene.n), make_pml(scene)
    rc = lib().fdtd_reverse_kind(C.byref(g), C.byref(p))
    if rc < 0:
        raise FDTDError(rc, last_error())
    return rc


def adjoint_frame(scene):
    """(split, (xl, xh, yl, yh)): whether the fused adjoint step of this grid runs as a frame launch and
    a plain-rectangle launch, and the frame's leading/trailing tile columns and rows."""
    g, p = make_grid(scene.n), make_pml(scene)
    f = (C.c_int32 * 4)()
    rc = lib().fdtd_adjoint_frame(C.byref(g), C.byref(p), f)
    if rc < 0:
        raise FDTDError(rc, last_error())
    return rc, tuple(int(v) for v in f)


def wait_probe(limit_ms: int):
    """Run one bounded device-side wait that nothing completes (fdtd_wait_probe): returns (code, the
    nanoseconds it waited); the code is FDTD_ERR_TIMEOUT when the wait gave up as it should."""
    ns = C.c_int64(0)
    rc = lib().fdtd_wait_probe(int(limit_ms), C.byref(ns))
    return rc, int(ns.value)


def set_byte_budget(nbytes: int):
    check(lib().fdtd_set_byte_budget(int(nbytes)))


def _handles(solvers):
    arr = (_VP * len(solvers))()
    for r, s in enumerate(solvers):
        arr[r] = s.h
    return arr


def group_step(solvers, nsteps: int):
    """fdtd_group_step: advance every solver's current phase by up to nsteps steps, one launch per
    kernel and step for the whole group (the solvers must share one stream)."""
    check(lib().fdtd_group_step(_handles(solvers), len(solvers), int(nsteps)))


def group_forward(solvers, nsteps, record_faces: bool = False):
    """fdtd_group_forward: whole forwards of a group (nsteps: one count per solver, or one for all)."""
    ns = [int(nsteps)] * len(solvers) if np.isscalar(nsteps) else [int(v) for v in nsteps]
    check(lib().fdtd_group_forward(_handles(solvers), len(solvers), (C.c_int32 * len(ns))(*ns),
                                   FDTD_RECORD_FACES if record_faces else 0))
    for s, n in zip(solvers, ns):
        s.nsteps = n


def group_backward(solvers, dL_ddet, dL_deps):
    """fdtd_group_backward: the reverse sweeps of a group (lists of per-solver buffers)."""
    g = (_VP * len(solvers))(*[_ptr(x) for x in dL_ddet])
    o = (_VP * len(solvers))(*[_ptr(x) for x in dL_deps])
    check(lib().fdtd_group_backward(_handles(solvers), len(solvers), g, o))


class Solver:
    """One solver handle (fdtd_create ... fdtd_destroy) built from a scene description.

    eps_inv may be given as a torch CUDA tensor or a numpy array; by default the scene's array.
    """

    def __init__(self, scene, stream=None, eps_inv=None, spacing: float = 0.0):
        L = lib()
        self.scene = scene
        self._keep = []
        srcs = (fdtd_source * max(1, len(scene.sources)))()
        for q, s in enumerate(scene.sources):
            srcs[q].component = int(s.component)
            for d in range(3):
                srcs[q].lo[d] = int(s.lo[d])
                srcs[q].hi[d] = int(s.hi[d])
            if s.profile is not None:
                prof = np.ascontiguousarray(np.asarray(s.profile, dtype=np.float32)).ravel()
                self._keep.append(prof)
                srcs[q].profile = prof.ctypes.data_as(C.POINTER(C.c_float))
            srcs[q].amplitude = float(s.amplitude)
            srcs[q].wavelength_cells = float(s.wavelength_cells)
            srcs[q].tau_steps = float(s.tau_steps)
            srcs[q].t0_steps = float(s.t0_steps)
            srcs[q].tfsf = int(getattr(s, "tfsf", 0))
            srcs[q].eps_background = float(getattr(s, "eps_background", 1.0))
        dets = (fdtd_detector * max(1, len(scene.detectors)))()
        for q, dt in enumerate(scene.detectors):
            dets[q].kind = int(dt.kind)
            dets[q].component = int(dt.component)
            dets[q].axis = int(dt.axis)
            for d in range(3):
                dets[q].lo[d] = int(dt.lo[d])
                dets[q].hi[d] = int(dt.hi[d])
        if eps_inv is None:
            eps_inv = np.ascontiguousarray(np.asarray(scene.eps_inv, dtype=np.float32))
        self._keep.append(eps_inv)
        g = make_grid(scene.n)
        p = make_pml(scene)
        h = _VP()
        stream_ptr = None
        if stream is not None:
            stream_ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        check(L.fdtd_create(C.byref(h), C.byref(g), float(spacing), float(scene.courant), _ptr(eps_inv),
                            srcs, len(scene.sources), dets, len(scene.detectors), C.byref(p),
                            _I3(*scene.design_lo), _I3(*scene.design_hi), stream_ptr))
        self.h = h
        self.nsteps = None
        self.stream = stream  # the stream given at creation (None: the legacy default stream)

    def close(self):
        if getattr(self, "h", None):
            lib().fdtd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- ABI calls -----------------------------------------------------------------------------
    def fdtd_forward(self, nsteps: int, record_faces: bool = False):
        check(lib().fdtd_forward(self.h, int(nsteps), FDTD_RECORD_FACES if record_faces else 0))
        self.nsteps = int(nsteps)

    def fdtd_backward(self, dL_ddet, dL_deps):
        check(lib().fdtd_backward(self.h, _ptr(dL_ddet), _ptr(dL_deps)))

    def fdtd_read_detectors(self, out):
        check(lib().fdtd_read_detectors(self.h, _ptr(out)))

    def fdtd_detector_total(self) -> int:
        return int(lib().fdtd_detector_total(self.h))

    def fdtd_get_fields(self, out6):
        check(lib().fdtd_get_fields(self.h, _ptr(out6)))

    def fdtd_read_detector(self, idx: int, out):
        check(lib().fdtd_read_detector(self.h, int(idx), _ptr(out)))

    def fdtd_detector_size(self, idx: int) -> int:
        n = int(lib().fdtd_detector_size(self.h, int(idx)))
        if n < 0:
            raise FDTDError(n, last_error())
        return n

    def detector(self, idx: int) -> np.ndarray:
        out = np.zeros(max(1, self.fdtd_detector_size(idx)), dtype=np.float64)
        self.fdtd_read_detector(idx, out)
        return out[: self.fdtd_detector_size(idx)]

    def fdtd_set_initial_fields(self, fields6):
        check(lib().fdtd_set_initial_fields(self.h, _ptr(fields6)))

    def fdtd_set_design_eps_inv(self, box):
        check(lib().fdtd_set_design_eps_inv(self.h, _ptr(box)))

    def fdtd_set_design_density(self, rho_box, eps_lo: float, eps_hi: float):
        check(lib().fdtd_set_design_density(self.h, _ptr(rho_box), float(eps_lo), float(eps_hi)))

    def fdtd_backward_density(self, dL_ddet, dL_drho):
        check(lib().fdtd_backward_density(self.h, _ptr(dL_ddet), _ptr(dL_drho)))

    def fdtd_design_adam_step(self, dL_drho, theta, m, v, rho_out, t: int, lr: float, beta1: float = 0.9,
                              beta2: float = 0.999, eps: float = 1e-8, proj_beta: float = 0.0,
                              proj_eta: float = 0.5):
        check(lib().fdtd_design_adam_step(self.h, _ptr(dL_drho), _ptr(theta), _ptr(m), _ptr(v), _ptr(rho_out),
                                          int(t), float(lr), float(beta1), float(beta2), float(eps),
                                          float(proj_beta), float(proj_eta)))

    def fdtd_backward_checkpointed(self, dL_ddet, dL_deps, method: int = 0, slots: int = 0) -> int:
        """Checkpointing gradient of the last forward (method 0 recursive halving, 1 treeverse with
        `slots` stored states); returns the forward steps it evaluated."""
        n = C.c_int64(0)
        check(lib().fdtd_backward_checkpointed(self.h, _ptr(dL_ddet), _ptr(dL_deps), int(method), int(slots),
                                               C.byref(n)))
        return int(n.value)

    def fdtd_design_project(self, theta, rho_out, proj_beta: float = 0.0, proj_eta: float = 0.5):
        check(lib().fdtd_design_project(self.h, _ptr(theta), _ptr(rho_out), float(proj_beta), float(proj_eta)))

    def fdtd_synchronize(self):
        check(lib().fdtd_synchronize(self.h))

    def fdtd_set_segment_steps(self, steps: int):
        """Keep the faces of the last `steps`-step segment only, regenerating the others (0: all)."""
        check(lib().fdtd_set_segment_steps(self.h, int(steps)))

    def fdtd_poll_status(self):
        """Raise what the kernels flagged, without waiting for the stream (its work must be done)."""
        check(lib().fdtd_poll_status(self.h))

    def fdtd_set_stream(self, stream):
        """Move the handle to another stream (a torch stream, a raw handle or None)."""
        ptr = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        check(lib().fdtd_set_stream(self.h, ptr))
        self.stream = stream

    def fdtd_begin(self, nsteps: int, record_faces: bool = False):
        check(lib().fdtd_begin(self.h, int(nsteps), FDTD_RECORD_FACES if record_faces else 0))
        self.nsteps = int(nsteps)

    def fdtd_begin_backward(self, dL_ddet):
        check(lib().fdtd_begin_backward(self.h, _ptr(dL_ddet)))

    def fdtd_phase(self):
        """(phase, steps left in it)."""
        ph, left = C.c_int32(0), C.c_int32(0)
        check(lib().fdtd_phase(self.h, C.byref(ph), C.byref(left)))
        return int(ph.value), int(left.value)

    def fdtd_finish_backward(self, dL_deps):
        check(lib().fdtd_finish_backward(self.h, _ptr(dL_deps)))

    def fdtd_finish_backward_density(self, dL_drho):
        check(lib().fdtd_finish_backward_density(self.h, _ptr(dL_drho)))

    def fdtd_set_check_interval(self, every: int):
        """Check the fields for NaN / infinity every `every` forward steps too (0: at sweep ends only)."""
        check(lib().fdtd_set_check_interval(self.h, int(every)))

    def fdtd_set_face_overlap(self, enable: bool):
        """Face copies beside the stencil kernels (True, for handles that solve repeatedly) or in line."""
        check(lib().fdtd_set_face_overlap(self.h, 1 if enable else 0))

    def fdtd_set_graphs(self, enable: bool):
        """Time loops captured into CUDA graphs (True, for repeated solves) or launched directly."""
        check(lib().fdtd_set_graphs(self.h, 1 if enable else 0))

    def fdtd_set_canaries(self, enable: bool):
        """NaN canaries in the arrays' pitch padding (a debugging aid)."""
        check(lib().fdtd_set_canaries(self.h, 1 if enable else 0))

    def fdtd_check_canaries(self) -> int:
        """Padding entries some kernel overwrote since the canaries were set (0: all intact)."""
        n = C.c_int64(0)
        check(lib().fdtd_check_canaries(self.h, C.byref(n)))
        return int(n.value)

    def fdtd_bytes_allocated(self) -> int:
        return int(lib().fdtd_bytes_allocated(self.h))

    def fdtd_release_history(self):
        check(lib().fdtd_release_history(self.h))

    def fdtd_launch_count(self) -> int:
        return int(lib().fdtd_launch_count(self.h))

    def fdtd_profile(self, enable: bool, every: int = 16):
        check(lib().fdtd_profile(self.h, int(bool(enable)), int(every)))

    def fdtd_profile_read(self):
        """{kernel name: (total ms of the timed launches, number timed)}."""
        nk = len(KERNEL_NAMES)
        ms = np.zeros(nk, dtype=np.float64)
        cnt = np.zeros(nk, dtype=np.int64)
        check(lib().fdtd_profile_read(self.h, ms.ctypes.data, cnt.ctypes.data, nk))
        return {KERNEL_NAMES[k]: (float(ms[k]), int(cnt[k])) for k in range(nk) if cnt[k] > 0}

    # --- numpy conveniences (host buffers) ------------------------------------------------------
    def detectors(self) -> np.ndarray:
        out = np.zeros(max(1, self.fdtd_detector_total()), dtype=np.float64)
        self.fdtd_read_detectors(out)
        return out[: self.fdtd_detector_total()]

    def fields(self) -> np.ndarray:
        nx, ny, nz = self.scene.n
        out = np.zeros((6, nz, ny, nx), dtype=np.float32)
        self.fdtd_get_fields(out)
        return out

    def gradient(self, dL_ddet) -> np.ndarray:
        shape = self.scene.design_shape()
        out = np.zeros(shape, dtype=np.float32)
        g = np.ascontiguousarray(np.asarray(dL_ddet, dtype=np.float64))
        self.fdtd_backward(g, out)
        return out
