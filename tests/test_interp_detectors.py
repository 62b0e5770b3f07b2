"""Interpolated detectors (arXiv 2412.12360 Sec. 2.1: composite metrics such as energy and Poynting
flux need the staggered components interpolated in space and time; the paper's evaluation mode).

Every component is taken at the cell centre (E_c: mean of its 4 values around the centre, H_c: mean
of its 2), and the flux uses E^{n+1/2} = (E^n + E^{n+1}) / 2.

Oracle pins (CPU): the interpolation is exact for fields affine in space (the detector equals the
closed form at the cell centres), and the gradient through interpolated detectors equals the
complex-step derivative (independent of the adjoint code) and agrees between store-all and time
reversal. GPU (CUDA fp32) against the oracle: detector outputs and dL/deps.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_12360_b300 import scenes as S
from tests import _helpers as H


def affine_fields(n, coef):
    """(6, nz, ny, nx) fields with F_c(x) = coef[c] . (1, x, y, z) at each component's Yee position."""
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.zeros((6, nz, ny, nx))
    for f in range(6):
        c = f % 3
        off = np.full(3, 0.5) if f >= 3 else np.zeros(3)
        off[c] += 0.5 if f < 3 else -0.5                         # E_c at +1/2 along c; H_c at 0 along c
        pos = (x + off[0], y + off[1], z + off[2])
        a = coef[f]
        out[f] = a[0] + a[1] * pos[0] + a[2] * pos[1] + a[3] * pos[2]
    return out


def centre_value(coef, f, p):
    a = coef[f]
    return a[0] + a[1] * (p[0] + 0.5) + a[2] * (p[1] + 0.5) + a[3] * (p[2] + 0.5)


def test_interpolation_exact_for_affine_fields():
    n = (12, 11, 10)
    rng = np.random.default_rng(2)
    c1, c0 = rng.standard_normal((6, 4)), rng.standard_normal((6, 4))
    st, prev = affine_fields(n, c1), affine_fields(n, c0)
    lo, hi = (2, 3, 4), (9, 8, 7)
    sc = H.box_scene(n, detectors=[S.Detector(S.DET_PLANE_E2_SUM_INTERP, lo, hi),
                                   S.Detector(S.DET_PLANE_FLUX_INTERP, lo, hi, axis=1)], nsteps=1)
    out = O.sample(sc, st, prev)
    cells = [(i, j, k) for k in range(lo[2], hi[2]) for j in range(lo[1], hi[1]) for i in range(lo[0], hi[0])]
    e2 = np.array([sum(centre_value(c1, c, p) ** 2 for c in range(3)) for p in cells])
    a1, a2 = 2, 0  # axis y: (E x H)_y = Ez Hx - Ex Hz
    flux = sum(0.5 * (centre_value(c1, a1, p) + centre_value(c0, a1, p)) * centre_value(c1, 3 + a2, p) -
               0.5 * (centre_value(c1, a2, p) + centre_value(c0, a2, p)) * centre_value(c1, 3 + a1, p) for p in cells)
    assert np.max(np.abs(out[:len(cells)] - e2)) <= 1e-12 * np.max(np.abs(e2))
    assert abs(out[len(cells)] - flux) <= 1e-12 * abs(flux)


def interp_scene(nsteps=80):
    n = (22, 20, 24)
    rng = np.random.default_rng(19)
    eps_inv = np.ones((n[2], n[1], n[0]), dtype=np.float32)
    dlo, dhi = (8, 7, 9), (14, 13, 14)
    eps_inv[dlo[2]:dhi[2], dlo[1]:dhi[1], dlo[0]:dhi[0]] = S.inv(1.0 + 11.1 * rng.random((5, 6, 6)))
    src = H.point_source(S.EY, (10, 10, 6), wavelength=8.0)
    dets = [S.Detector(S.DET_PLANE_E2_SUM_INTERP, (6, 6, 16), (15, 14, 17)),
            S.Detector(S.DET_PLANE_FLUX_INTERP, (6, 6, 17), (15, 14, 18), axis=2),
            S.Detector(S.DET_PLANE_FLUX_INTERP, (12, 6, 8), (13, 14, 16), axis=0)]
    return H.box_scene(n, pml=(5,) * 6, eps_inv=eps_inv, sources=[src], detectors=dets, design=(dlo, dhi),
                       nsteps=nsteps, name="interp")


def test_interpolated_detector_gradient_complex_step():
    sc = interp_scene(80)
    g = np.random.default_rng(5).standard_normal(O.detector_total(sc, 80))
    gt, _, _ = O.gradient(sc, 80, g, O.METHOD_TIME_REVERSAL)
    gs, _, _ = O.gradient(sc, 80, g, O.METHOD_STORE_ALL)
    assert np.linalg.norm(gt - gs) <= 1e-10 * np.linalg.norm(gs)
    vox = [(9, 8, 10), (12, 11, 12), (8, 12, 13)]
    cs = O.complex_step(sc, 80, g, vox)
    dlo = sc.design_lo
    for v, c in zip(vox, cs):
        a = gs[v[2] - dlo[2], v[1] - dlo[1], v[0] - dlo[0]]
        assert abs(a - c) <= 1e-9 * max(abs(c), 1e-30), (v, a, c)


# ---------------------------------------------------------------- GPU against the oracle --------

@pytest.fixture(scope="module")
def F(cuda_ok):
    from paper_2412_12360_b300 import fdtd
    fdtd.lib()
    return fdtd


@pytest.mark.gpu
def test_gpu_interpolated_detectors_and_gradient(F):
    sc = interp_scene(300)
    g = np.random.default_rng(6).standard_normal(O.detector_total(sc, 300))
    grad_o, _, det_o = O.gradient(sc, 300, g, O.METHOD_TIME_REVERSAL)
    with F.Solver(sc) as s:
        s.fdtd_forward(300, record_faces=True)
        det_g = s.detectors()
        grad_g = s.gradient(g)
    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))
    print("interpolated detectors rel %.3e, dL/deps rel %.3e" % (rel(det_g, det_o), rel(grad_g, grad_o)))
    assert rel(det_g, det_o) < 1e-4
    assert rel(grad_g, grad_o) < 1e-3


@pytest.mark.gpu
def test_gpu_interpolated_detectors_checkpointed_gradient(F):
    """The checkpointing gradient takes E^n of the interpolated flux from the recomputed state."""
    sc = interp_scene(120)
    g = np.random.default_rng(7).standard_normal(O.detector_total(sc, 120))
    grad_o, _, _ = O.gradient(sc, 120, g, O.METHOD_TIME_REVERSAL)
    with F.Solver(sc) as s:
        s.fdtd_forward(120)
        d = np.zeros(sc.design_shape(), dtype=np.float32)
        s.fdtd_backward_checkpointed(g, d, 1, 5)
    e = float(np.linalg.norm(d - grad_o) / np.linalg.norm(grad_o))
    print("interpolated detectors, treeverse gradient rel %.3e" % e)
    assert e < 1e-3
