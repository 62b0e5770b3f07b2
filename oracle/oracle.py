"""ctypes wrapper of the FP64 oracle (yee_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the bench's CPU-baseline leg,
never by the product path. It takes a scene object by duck typing (attributes listed in
`_SceneArgs`) and shares no code with the CUDA library.

Functions follow arXiv 2412.12360: `forward` is the Yee leapfrog of Sec. 2.1 (Eqs. 1-2) with CPML,
soft sources and detectors; `roundtrip` is the inverse update step of Sec. 2.2; `gradient` is the
reverse-mode derivative of Sec. 2.2 by store-all, checkpointing or time reversal; `complex_step` is
an independent derivative check.
"""
import ctypes as C

import numpy as np

from . import build as _build


class _Source(C.Structure):
    _fields_ = [("component", C.c_int32), ("lo", C.c_int32 * 3), ("hi", C.c_int32 * 3),
                ("profile", C.POINTER(C.c_double)), ("amplitude", C.c_double),
                ("wavelength_cells", C.c_double), ("tau_steps", C.c_double), ("t0_steps", C.c_double),
                ("tfsf", C.c_int32), ("eps_background", C.c_double)]


class _Detector(C.Structure):
    _fields_ = [("kind", C.c_int32), ("component", C.c_int32), ("axis", C.c_int32),
                ("lo", C.c_int32 * 3), ("hi", C.c_int32 * 3)]


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("courant", C.c_double), ("pml", C.c_int32 * 6),
                ("sigma_max", C.c_double), ("kappa_max", C.c_double), ("alpha_max", C.c_double),
                ("grading_m", C.c_int32), ("eps_inv", C.POINTER(C.c_double)),
                ("nsrc", C.c_int32), ("src", C.POINTER(_Source)),
                ("ndet", C.c_int32), ("det", C.POINTER(_Detector)),
                ("design_lo", C.c_int32 * 3), ("design_hi", C.c_int32 * 3)]


_LIB = None


def load(path):
    """The oracle library at `path` with its entry points typed (lib() loads the built one)."""
    L = C.CDLL(path)
    P = C.POINTER
    d = P(C.c_double)
    L.orc_detector_total.argtypes = [P(_Scene), C.c_int32]
    L.orc_detector_total.restype = C.c_int64
    L.orc_face_count.argtypes = [P(_Scene)]
    L.orc_face_count.restype = C.c_int64
    L.orc_forward.argtypes = [P(_Scene), C.c_int32, d, d, d]
    L.orc_roundtrip.argtypes = [P(_Scene), C.c_int32, d, d, d]
    L.orc_gradient.argtypes = [P(_Scene), C.c_int32, d, C.c_int32, C.c_int32, d, d, d]
    L.orc_gradient_from.argtypes = [P(_Scene), C.c_int32, d, d, C.c_int32, C.c_int32, d, d, d]
    L.orc_complex_step.argtypes = [P(_Scene), C.c_int32, d, C.c_int32, P(C.c_int32), C.c_double, d]
    L.orc_cpml_tables.argtypes = [P(_Scene), C.c_int32, d]
    L.orc_sample.argtypes = [P(_Scene), d, d, d]
    L.orc_waveform.argtypes = [P(_Scene), C.c_int32, C.c_double]
    L.orc_waveform.restype = C.c_double
    return L


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load(_build.build())
    return _LIB


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


class _SceneArgs:
    """Marshals a scene object into the oracle's C structures (and keeps the arrays alive).

    Expected attributes: n (nx, ny, nz), courant, pml (6 ints), sigma_max, kappa_max, alpha_max,
    grading_m, eps_inv (array (nz, ny, nx)), sources (component, lo, hi, profile or None, amplitude,
    wavelength_cells, tau_steps, t0_steps, and optionally tfsf and eps_background), detectors (kind,
    component, axis, lo, hi),
    design_lo, design_hi.
    """

    def __init__(self, scene):
        self.scene = scene
        self.n = tuple(int(v) for v in scene.n)
        nx, ny, nz = self.n
        self.eps_inv = np.ascontiguousarray(np.asarray(scene.eps_inv, dtype=np.float64).reshape(nz, ny, nx))
        self._profiles = []
        srcs = (_Source * max(1, len(scene.sources)))()
        for q, s in enumerate(scene.sources):
            srcs[q].component = int(s.component)
            for d in range(3):
                srcs[q].lo[d] = int(s.lo[d])
                srcs[q].hi[d] = int(s.hi[d])
            if s.profile is not None:
                prof = np.ascontiguousarray(np.asarray(s.profile, dtype=np.float64)).ravel()
                self._profiles.append(prof)
                srcs[q].profile = _dptr(prof)
            srcs[q].amplitude = float(s.amplitude)
            srcs[q].wavelength_cells = float(s.wavelength_cells)
            srcs[q].tau_steps = float(s.tau_steps)
            srcs[q].t0_steps = float(s.t0_steps)
            srcs[q].tfsf = int(getattr(s, "tfsf", 0))
            srcs[q].eps_background = float(getattr(s, "eps_background", 1.0))
        dets = (_Detector * max(1, len(scene.detectors)))()
        for q, dt in enumerate(scene.detectors):
            dets[q].kind = int(dt.kind)
            dets[q].component = int(dt.component)
            dets[q].axis = int(dt.axis)
            for d in range(3):
                dets[q].lo[d] = int(dt.lo[d])
                dets[q].hi[d] = int(dt.hi[d])
        self._srcs, self._dets = srcs, dets
        sc = _Scene()
        for d in range(3):
            sc.n[d] = self.n[d]
            sc.design_lo[d] = int(scene.design_lo[d])
            sc.design_hi[d] = int(scene.design_hi[d])
        sc.courant = float(scene.courant)
        for f in range(6):
            sc.pml[f] = int(scene.pml[f])
        sc.sigma_max = float(scene.sigma_max)
        sc.kappa_max = float(scene.kappa_max)
        sc.alpha_max = float(scene.alpha_max)
        sc.grading_m = int(scene.grading_m)
        sc.eps_inv = _dptr(self.eps_inv)
        sc.nsrc = len(scene.sources)
        sc.src = srcs
        sc.ndet = len(scene.detectors)
        sc.det = dets
        self.c = sc

    @property
    def ptr(self):
        return C.byref(self.c)

    @property
    def N(self):
        nx, ny, nz = self.n
        return nx * ny * nz

    def design_shape(self):
        s = self.scene
        return tuple(int(s.design_hi[d]) - int(s.design_lo[d]) for d in (2, 1, 0))


def detector_total(scene, nsteps):
    a = _SceneArgs(scene)
    return int(lib().orc_detector_total(a.ptr, nsteps))


def face_count(scene):
    a = _SceneArgs(scene)
    return int(lib().orc_face_count(a.ptr))


def _fields_in(a, init):
    if init is None:
        return None
    arr = np.ascontiguousarray(np.asarray(init, dtype=np.float64)).reshape(6 * a.N)
    return arr


def forward(scene, nsteps, init=None):
    """Run nsteps steps. Returns (fields (6, nz, ny, nx): E^n then H^{n-1/2}, detector vector)."""
    a = _SceneArgs(scene)
    nx, ny, nz = a.n
    init_arr = _fields_in(a, init)
    out = np.zeros(6 * a.N)
    det = np.zeros(max(1, int(lib().orc_detector_total(a.ptr, nsteps))))
    rc = lib().orc_forward(a.ptr, int(nsteps), _dptr(init_arr), _dptr(out), _dptr(det))
    assert rc == 0
    return out.reshape(6, nz, ny, nx), det[: int(lib().orc_detector_total(a.ptr, nsteps))]


def roundtrip(scene, nsteps, init=None):
    """Forward nsteps with face recording, then nsteps inverse steps. Returns (after_fwd, after_back)."""
    a = _SceneArgs(scene)
    nx, ny, nz = a.n
    init_arr = _fields_in(a, init)
    fwd = np.zeros(6 * a.N)
    back = np.zeros(6 * a.N)
    rc = lib().orc_roundtrip(a.ptr, int(nsteps), _dptr(init_arr), _dptr(fwd), _dptr(back))
    assert rc == 0
    return fwd.reshape(6, nz, ny, nx), back.reshape(6, nz, ny, nx)


METHOD_STORE_ALL, METHOD_CHECKPOINT, METHOD_TIME_REVERSAL = 0, 1, 2


def gradient(scene, nsteps, dL_ddet, method=METHOD_TIME_REVERSAL, interval=16, full=False, init=None):
    """dL/deps on the design box (shape (dz, dy, dx)) for L = sum(dL_ddet * detectors), for the forward
    from `init` (fields (6, nz, ny, nx): E^0, H^{-1/2}; None: zero fields).

    Returns (dL_deps, dL_da over the whole grid or None, detector vector).
    """
    a = _SceneArgs(scene)
    nx, ny, nz = a.n
    ntot = int(lib().orc_detector_total(a.ptr, nsteps))
    g = np.ascontiguousarray(np.asarray(dL_ddet, dtype=np.float64)).ravel()
    assert g.size == ntot
    out = np.zeros(max(1, int(np.prod(a.design_shape()))))
    full_arr = np.zeros(a.N) if (full and method != METHOD_TIME_REVERSAL) else None
    det = np.zeros(max(1, ntot))
    init_arr = _fields_in(a, init)
    rc = lib().orc_gradient_from(a.ptr, int(nsteps), _dptr(init_arr), _dptr(g), int(method), int(interval),
                                 _dptr(out), _dptr(full_arr), _dptr(det))
    assert rc == 0
    dshape = a.design_shape()
    grad = out[: int(np.prod(dshape))].reshape(dshape)
    return grad, (full_arr.reshape(nz, ny, nx) if full_arr is not None else None), det[:ntot]


def complex_step(scene, nsteps, dL_ddet, voxels, h=1e-20):
    """Complex-step dL/deps at voxels [(i, j, k), ...]."""
    a = _SceneArgs(scene)
    g = np.ascontiguousarray(np.asarray(dL_ddet, dtype=np.float64)).ravel()
    vox = np.ascontiguousarray(np.asarray(voxels, dtype=np.int32)).ravel()
    out = np.zeros(len(voxels))
    rc = lib().orc_complex_step(a.ptr, int(nsteps), _dptr(g), len(voxels),
                                vox.ctypes.data_as(C.POINTER(C.c_int32)), float(h), _dptr(out))
    assert rc == 0
    return out


def sample(scene, state6, prev6=None):
    """Detector outputs of one step sampled from given fields: state6 = (E^{n+1}, H^{n+1/2}) as
    (6, nz, ny, nx), prev6 (optional) supplies E^n in its first three arrays."""
    a = _SceneArgs(scene)
    st = np.ascontiguousarray(np.asarray(state6, dtype=np.float64))
    pv = None if prev6 is None else np.ascontiguousarray(np.asarray(prev6, dtype=np.float64))
    out = np.zeros(detector_total(scene, 1))
    lib().orc_sample(a.ptr, _dptr(pv), _dptr(st), _dptr(out))
    return out


def cpml_tables(scene, axis):
    """(b_int, c_int, kappa_int, b_half, c_half, kappa_half) of one axis."""
    a = _SceneArgs(scene)
    N = a.n[axis]
    out = np.zeros(6 * N)
    lib().orc_cpml_tables(a.ptr, int(axis), _dptr(out))
    return out.reshape(6, N)


def waveform(scene, q, step):
    a = _SceneArgs(scene)
    return float(lib().orc_waveform(a.ptr, int(q), float(step)))
