"""The C ABI library loads, exports every symbol the header declares, and validates its input on the
host (no GPU needed: these calls fail before any CUDA work)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_2412_12360_b300 import fdtd as F
from paper_2412_12360_b300 import scenes as S
from paper_2412_12360_b300.csrc import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return F.lib()


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|int64_t|char\s*\*|void)\s*\**\s*(fdtd_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(L):
    names = _declared_symbols()
    assert "fdtd_create" in names and "fdtd_backward" in names and len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    bound = {s[0] for s in F.SIGNATURES}
    assert names <= bound, names - bound


def test_version_and_error_string(L):
    assert b"sm_103a" in L.fdtd_version()
    assert isinstance(F.last_error(), str)


def _create(scene, courant=None, pml=None, src=None, det=None, design=None):
    """Call fdtd_create with possibly broken arguments; return (rc, message)."""
    sc = scene
    g = F.make_grid(sc.n)
    p = F.make_pml(sc)
    if pml is not None:
        for f in range(6):
            p.thickness[f] = pml[f]
    srcs = (F.fdtd_source * 2)()
    ns = 0
    for s in (src if src is not None else sc.sources):
        srcs[ns].component = s[0] if isinstance(s, tuple) else s.component
        lo, hi = (s[1], s[2]) if isinstance(s, tuple) else (s.lo, s.hi)
        srcs[ns].tfsf = s[3] if isinstance(s, tuple) and len(s) > 3 else 0
        srcs[ns].eps_background = s[4] if isinstance(s, tuple) and len(s) > 4 else 1.0
        for d in range(3):
            srcs[ns].lo[d] = lo[d]
            srcs[ns].hi[d] = hi[d]
        srcs[ns].amplitude = 1.0
        srcs[ns].wavelength_cells = 20.0
        srcs[ns].tau_steps = 30.0
        srcs[ns].t0_steps = 90.0
        ns += 1
    dets = (F.fdtd_detector * 2)()
    nd = 0
    for d in (det if det is not None else []):
        dets[nd].kind, dets[nd].component, dets[nd].axis = d[0], d[1], d[2]
        for k in range(3):
            dets[nd].lo[k] = d[3][k]
            dets[nd].hi[k] = d[4][k]
        nd += 1
    eps = np.ones(sc.n[::-1], dtype=np.float32)
    dlo, dhi = design if design is not None else (sc.design_lo, sc.design_hi)
    h = C.c_void_p()
    rc = F.lib().fdtd_create(C.byref(h), C.byref(g), 0.0, float(sc.courant if courant is None else courant),
                             eps.ctypes.data, srcs, ns, dets, nd, C.byref(p), F._I3(*dlo), F._I3(*dhi), None)
    return rc, F.last_error()


def test_create_rejects_bad_input_before_any_device_work(L):
    sc = S.cavity_32(10)
    rc, msg = _create(sc, courant=0.6)
    assert rc == F.FDTD_ERR_UNSTABLE and "stability" in msg
    rc, _ = _create(sc, courant=-1.0)
    assert rc == F.FDTD_ERR_INVALID_ARG
    rc, msg = _create(sc, pml=(16, 16, 0, 0, 0, 0))
    assert rc == F.FDTD_ERR_INVALID_ARG and "PML" in msg
    rc, msg = _create(sc, src=[(3, (1, 1, 1), (2, 2, 2))])
    assert rc == F.FDTD_ERR_INVALID_ARG and "component" in msg
    rc, msg = _create(sc, src=[(2, (30, 1, 1), (33, 2, 2))])
    assert rc == F.FDTD_ERR_INVALID_ARG and "box" in msg
    rc, msg = _create(sc, det=[(7, 0, 0, (1, 1, 1), (2, 2, 2))])
    assert rc == F.FDTD_ERR_INVALID_ARG and "kind" in msg
    rc, msg = _create(sc, det=[(0, 6, 0, (1, 1, 1), (2, 2, 2))])
    assert rc == F.FDTD_ERR_INVALID_ARG
    rc, msg = _create(sc, det=[(2, 0, 3, (1, 1, 1), (2, 2, 2))])
    assert rc == F.FDTD_ERR_INVALID_ARG and "axis" in msg
    rc, msg = _create(sc, design=((4, 4, 4), (40, 8, 8)))
    assert rc == F.FDTD_ERR_INVALID_ARG and "design" in msg


def test_create_rejects_grids_beyond_the_index_range(L):
    """Per-array offsets are 32-bit: a grid whose pitch-padded field array reaches 2^31 cells, or an
    axis outside [2, 65536], is refused before any device work."""
    sc = S.cavity_32(10)
    for n, what in (((2048, 1024, 1024), "2^31"), ((1, 32, 32), "range"), ((70000, 4, 4), "range")):
        g = F.make_grid(n)
        p = F.make_pml(sc)
        eps = np.ones(1, dtype=np.float32)
        h = C.c_void_p()
        rc = F.lib().fdtd_create(C.byref(h), C.byref(g), 0.0, float(sc.courant), eps.ctypes.data, None, 0, None, 0,
                                 C.byref(p), F._I3(0, 0, 0), F._I3(0, 0, 0), None)
        assert rc == F.FDTD_ERR_INVALID_ARG and what in F.last_error(), (n, F.last_error())


def test_create_rejects_bad_tfsf_and_interpolated_detectors(L):
    sc = S.cavity_32(10)
    design = ((10, 10, 10), (20, 20, 20))
    ok = (0, (4, 4, 8), (28, 28, 9), 3)  # Ex plane at z = 8, travelling +z
    rc, msg = _create(sc, src=[(2, (4, 4, 8), (28, 28, 9), 3)], design=design)
    assert rc == F.FDTD_ERR_INVALID_ARG and "transverse" in msg
    rc, msg = _create(sc, src=[(0, (4, 4, 8), (28, 28, 10), 3)], design=design)
    assert rc == F.FDTD_ERR_INVALID_ARG and "thick" in msg
    rc, msg = _create(sc, src=[(0, (4, 4, 0), (28, 28, 1), 3)], design=design)
    assert rc == F.FDTD_ERR_INVALID_ARG and "scattered" in msg
    rc, msg = _create(sc, src=[(0, (4, 4, 31), (28, 28, 32), -3)], design=design)
    assert rc == F.FDTD_ERR_INVALID_ARG and "scattered" in msg
    rc, msg = _create(sc, src=[(0, (4, 4, 8), (28, 28, 9), 4)], design=design)
    assert rc == F.FDTD_ERR_INVALID_ARG and "tfsf" in msg
    rc, msg = _create(sc, src=[ok[:4] + (0.0,)], design=design)
    assert rc == F.FDTD_ERR_INVALID_ARG and "eps_background" in msg
    rc, msg = _create(sc, src=[(0, (4, 4, 15), (28, 28, 16), 3)], design=design)  # the plane in the box
    assert rc == F.FDTD_ERR_INVALID_ARG and "design" in msg
    rc, msg = _create(sc, src=[(0, (4, 4, 20), (28, 28, 21), 3)], design=design)  # H half plane 19 in the box
    assert rc == F.FDTD_ERR_INVALID_ARG and "design" in msg
    rc, msg = _create(sc, det=[(3, 0, 0, (4, 4, 20), (32, 28, 21))], design=design)
    assert rc == F.FDTD_ERR_INVALID_ARG and "interpolated" in msg
    rc, msg = _create(sc, det=[(4, 0, 5, (4, 4, 20), (28, 28, 21))], design=design)
    assert rc == F.FDTD_ERR_INVALID_ARG and "axis" in msg
    rc, msg = _create(sc, det=[(5, 0, 0, (4, 4, 20), (28, 28, 21))], design=design)
    assert rc == F.FDTD_ERR_INVALID_ARG and "kind" in msg


def test_checkpoint_cost_rejects_bad_arguments(L):
    assert L.fdtd_checkpoint_cost(-1, 0, 0) == -1
    assert L.fdtd_checkpoint_cost(10, 2, 3) == -1
    assert L.fdtd_checkpoint_cost(10, 1, 0) == -1
    assert L.fdtd_checkpoint_cost(0, 1, 3) == 0


def test_null_handle_calls_fail_cleanly(L):
    assert L.fdtd_forward(None, 10, 0) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_backward(None, None, None) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_destroy(None) == F.FDTD_OK
    assert L.fdtd_bytes_allocated(None) == -1
    assert L.fdtd_synchronize(None) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_set_check_interval(None, 8) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_set_canaries(None, 1) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_check_canaries(None, None) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_read_detector(None, 0, None) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_detector_size(None, 0) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_fields(None, None) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_set_face_overlap(None, 0) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_set_graphs(None, 0) == F.FDTD_ERR_INVALID_ARG


def test_wait_probe_rejects_bad_arguments_before_any_device_work(L):
    ns = C.c_int64(-5)
    assert L.fdtd_wait_probe(0, C.byref(ns)) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_wait_probe(2001, C.byref(ns)) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_wait_probe(10, None) == F.FDTD_ERR_INVALID_ARG
    assert ns.value == -5


def test_noalloc_flux_refuses_host_buffers_before_any_launch(L):
    """The allocation-free flux call takes device memory of the current device only: host buffers (or,
    with no GPU, anything) are refused with INVALID_ARG before a kernel is launched."""
    grid = F.make_grid((4, 4, 4))
    fields = np.zeros(6 * 64, dtype=np.float32)
    out = np.zeros(1, dtype=np.float64)
    rc = L.fdtd_plane_flux_noalloc(fields.ctypes.data, C.byref(grid), 2, F._I3(0, 0, 1), F._I3(4, 4, 2),
                                   out.ctypes.data, None)
    assert rc == F.FDTD_ERR_INVALID_ARG
    assert "device memory" in F.last_error()
    assert out[0] == 0.0


def test_footprint_grows_with_steps_and_faces(L):
    sc = S.design_96(2000)
    f0 = F.footprint_bytes(sc, 2000, record_faces=False)
    f1 = F.footprint_bytes(sc, 2000, record_faces=True)
    f2 = F.footprint_bytes(sc, 4000, record_faces=True)
    assert 0 < f0 < f1 < f2
    # face history: 2 tangential H per face cell per step, fp32, on 6 planes of 77 x 77
    per_step = 6 * 2 * 77 * 77 * 4
    assert f2 - f1 == 2000 * per_step
    # fields (6) + a + adjoint fields (6), each 96^3 fp32 (pitch 96)
    assert f0 >= 13 * 96 ** 3 * 4


def test_missing_library_fails_loudly():
    """Without the built library the binding raises at first use: there is no CPU fallback."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2412_12360_b300 import fdtd, scenes\n"
            "fdtd.LIB_PATH = '/nonexistent/libfdtd.so'\n"
            "try:\n"
            "    fdtd.Solver(scenes.cavity_32(10))\n"
            "except ImportError as e:\n"
            "    print('raised:', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(3)\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "not built" in r.stdout, (r.returncode, r.stdout, r.stderr)


def test_product_and_oracle_are_separate():
    """The product package and the CUDA library neither import nor include the oracle, and the oracle
    neither imports nor includes the product (the seeded input builders in scenes.py hold no method
    arithmetic and are the one module both use)."""
    pkg = os.path.join(ROOT, "paper_2412_12360_b300")
    product = glob.glob(os.path.join(pkg, "*.py")) + glob.glob(os.path.join(pkg, "csrc", "*.*")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    for f in product:
        text = open(f).read()
        assert not re.search(r"^\s*(from|import)\s+oracle\b|#include\s*[<\"].*oracle", text, re.M), f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.*")):
        if not f.endswith((".py", ".cpp", ".h", ".c")):
            continue
        text = open(f).read()
        assert not re.search(r"paper_2412_12360_b300\.(fdtd|serve|autograd|design|ranks)|csrc|fdtd_internal|libfdtd",
                             text), f
