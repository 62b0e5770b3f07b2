"""Full-size checks in the configurations bench.py times.

design_96 (the bench workload: 96^3, 10-cell CPML, 40^3 design box, 2000 steps): the whole detector
plane and the whole dL/deps against the FP64 oracle. waveguide_600 (600^3, 216 M cells): properties
that hold at any size, on the full grid for a shortened run: the fp32 time-reversal round trip
returns to the (zero) initial state, and dL/drho agrees with a central difference along a uniform
density shift.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_12360_b300 import scenes as S

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / np.linalg.norm(np.asarray(b, float)))


def test_design96_full_run_matches_oracle(cuda_ok):
    from paper_2412_12360_b300 import fdtd
    sc = S.design_96()
    g = np.ones(O.detector_total(sc, sc.nsteps))
    grad_o, _, det_o = O.gradient(sc, sc.nsteps, g, O.METHOD_TIME_REVERSAL)
    with fdtd.Solver(sc) as s:
        s.fdtd_forward(sc.nsteps, record_faces=True)
        det_g = s.detectors()
        grad_g = s.gradient(g)
    e_det, e_grad = rel(det_g, det_o), rel(grad_g, grad_o)
    print("design_96 2000 steps: detector rel L2 %.2e, dL/deps rel L2 %.2e" % (e_det, e_grad))
    assert e_det < 1e-4
    assert e_grad < 1e-3


def test_waveguide600_roundtrip_and_directional_derivative(cuda_ok):
    import torch
    from paper_2412_12360_b300 import fdtd
    nsteps = 1600
    sc = S.waveguide_600(nsteps)
    # the guided pulse (about 0.16 cells per step in the Si core) reaches the design box (x >= 200) after
    # ~1100 steps; its reflection is back at the x = 150 plane within 1600 steps
    sc.detectors = [S.Detector(S.DET_PLANE_FLUX, (150, 12, 12), (151, 588, 588), axis=0)]
    lo, hi = sc.extra["eps_lo"], sc.extra["eps_hi"]
    rho = torch.from_numpy(sc.extra["rho"]).cuda()
    v = torch.ones_like(rho)                 # direction: a uniform shift of the density
    with fdtd.Solver(sc) as s:
        s.fdtd_set_design_density(rho, lo, hi)
        s.fdtd_forward(nsteps, record_faces=True)
        det = s.detectors()
        peak = float(np.abs(s.fields()).max())
        g = np.ones(s.fdtd_detector_total())
        grad = torch.empty_like(rho)
        s.fdtd_backward_density(torch.from_numpy(g).cuda(), grad)
        torch.cuda.synchronize()
        back = s.fields()                     # reconstructed initial state on R (zero initially)
        nx, ny, nz = sc.n
        p = sc.pml
        rbox = back[:, p[4] + 1:nz - p[5] - 1, p[2] + 1:ny - p[3] - 1, p[0] + 1:nx - p[1] - 1]
        drift = float(np.abs(rbox).max()) / peak
        print("600^3 %d steps: round-trip residual / peak field %.2e" % (nsteps, drift))
        assert drift < 1e-4
        dd = float((grad.double() * v.double()).sum())
        delta = 1e-3
        L = []
        for sgn in (1, -1):
            s.fdtd_set_design_density((rho + sgn * delta * v).clamp(-1.0, 2.0).contiguous(), lo, hi)
            s.fdtd_forward(nsteps)
            L.append(float(s.detectors().sum()))
    fd = (L[0] - L[1]) / (2 * delta)
    print("600^3 directional derivative: adjoint %.6e, central difference %.6e" % (dd, fd))
    assert abs(fd - dd) <= 2e-2 * abs(dd)
