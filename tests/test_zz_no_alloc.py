"""The allocation-free flux entry point (fdtd_plane_flux_noalloc) against the solver's flux detector.

Callers that cannot allocate device memory (a fixed memory budget, real-time loops) use
fdtd_plane_flux_noalloc, whose scratch is a fixed array reserved at load time. Its result must
match the existing path: the flux detector of fdtd_forward, whose last sample is the flux of the
final fields. This file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2412_12360_b300 import scenes as S
from tests import _helpers as H

pytestmark = pytest.mark.gpu


def _scene(nsteps):
    n = (40, 36, 44)
    nx, ny, nz = n
    rng = np.random.default_rng(71)
    eps_inv = np.ones((nz, ny, nx), dtype=np.float32)
    eps_inv[14:30, 12:24, 14:26] = S.inv(1.0 + 11.1 * rng.random((16, 12, 12)))
    src = H.point_source(S.EZ, (20, 18, 10), wavelength=10.0)
    dets = [S.Detector(S.DET_PLANE_FLUX, (6, 6, 33), (34, 30, 34), axis=2),
            S.Detector(S.DET_PLANE_FLUX, (28, 6, 6), (29, 30, 38), axis=0),
            S.Detector(S.DET_PLANE_FLUX, (6, 25, 6), (34, 26, 38), axis=1)]
    return H.box_scene(n, pml=(6,) * 6, eps_inv=eps_inv, sources=[src], detectors=dets, nsteps=nsteps,
                       name="noalloc")


def test_noalloc_flux_matches_detector_on_two_calls_in_a_row(cuda_ok):
    import torch
    from paper_2412_12360_b300 import fdtd

    L = fdtd.lib()
    nsteps = 150
    sc = _scene(nsteps)
    nx, ny, nz = sc.n
    with fdtd.Solver(sc) as s:
        s.fdtd_forward(nsteps)
        det = s.detectors()
        fields = torch.zeros((6, nz, ny, nx), dtype=torch.float32, device="cuda")
        s.fdtd_get_fields(fields)
    torch.cuda.synchronize()
    f64 = fields.double().cpu().numpy()
    grid = fdtd.make_grid(sc.n)
    out = torch.zeros(2, len(sc.detectors), dtype=torch.float64, device="cuda")
    for call in range(2):
        for q, d in enumerate(sc.detectors):
            rc = L.fdtd_plane_flux_noalloc(fields.data_ptr(), C.byref(grid), d.axis, fdtd._I3(*d.lo),
                                           fdtd._I3(*d.hi), out[call, q].data_ptr(), None)
            assert rc == fdtd.FDTD_OK, fdtd.last_error()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for q, d in enumerate(sc.detectors):
        ref_det = det[q * nsteps + nsteps - 1]              # the detector's last sample
        a1, a2 = (d.axis + 1) % 3, (d.axis + 2) % 3
        sl = (slice(d.lo[2], d.hi[2]), slice(d.lo[1], d.hi[1]), slice(d.lo[0], d.hi[0]))
        ref_np = np.sum(f64[a1][sl] * f64[3 + a2][sl] - f64[a2][sl] * f64[3 + a1][sl])
        scale = np.sum(np.abs(f64[a1][sl] * f64[3 + a2][sl]) + np.abs(f64[a2][sl] * f64[3 + a1][sl]))
        assert scale > 0
        for call in range(2):
            assert abs(got[call, q] - ref_det) <= 1e-10 * scale, (q, call, got[call, q], ref_det)
            assert abs(got[call, q] - ref_np) <= 1e-10 * scale
        assert got[0, q] == got[1, q]


def test_noalloc_flux_rejects_oversized_and_bad_boxes(cuda_ok):
    import torch
    from paper_2412_12360_b300 import fdtd

    L = fdtd.lib()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = fdtd.make_grid((2048, 2048, 2))  # 8388608 cells in the box: above the 4194304-cell maximum
    dummy = torch.zeros(8, dtype=torch.float32, device="cuda")
    rc = L.fdtd_plane_flux_noalloc(dummy.data_ptr(), C.byref(big), 2, fdtd._I3(0, 0, 0), fdtd._I3(2048, 2048, 2),
                                   out.data_ptr(), None)
    assert rc == fdtd.FDTD_ERR_INVALID_ARG and "maximum" in fdtd.last_error()
    small = fdtd.make_grid((4, 4, 4))
    rc = L.fdtd_plane_flux_noalloc(dummy.data_ptr(), C.byref(small), 3, fdtd._I3(0, 0, 0), fdtd._I3(1, 1, 1),
                                   out.data_ptr(), None)
    assert rc == fdtd.FDTD_ERR_INVALID_ARG
    rc = L.fdtd_plane_flux_noalloc(dummy.data_ptr(), C.byref(small), 0, fdtd._I3(0, 0, 0), fdtd._I3(5, 1, 1),
                                   out.data_ptr(), None)
    assert rc == fdtd.FDTD_ERR_INVALID_ARG
