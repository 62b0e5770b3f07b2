"""One-sided total-field / scattered-field plane source (arXiv 2412.12360 Sec. 2.1: the incident
field enters on one side only).

Oracle pins (CPU): the wave leaves the plane on the total-field side only (time-integrated |E|^2 a
few cells behind the plane against the same distance ahead; a soft sheet with the same profile
radiates equally both ways), for each axis and both directions; the inverse step returns the initial
state on R with TFSF sources present; the time-reversal gradient equals the store-all gradient.
GPU (CUDA fp32) against the oracle: fields and detectors after a forward, and dL/deps.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_12360_b300 import scenes as S
from tests import _helpers as H


def tfsf_scene(axis, tfsf, comp, n=(40, 36, 44), ks=20, p=7, nsteps=140, w0=6.0, design=None, eps_inv=None,
               extra_sources=()):
    """A TFSF plane at index ks along `axis` over the PML-free cross-section (Gaussian profile) and
    |E|^2 planes 7 cells behind and ahead of it."""
    nx = list(n)
    lo, hi = [p, p, p], [n[0] - p, n[1] - p, n[2] - p]
    lo[axis], hi[axis] = ks, ks + 1
    t1, t2 = [d for d in range(3) if d != axis]
    prof2 = S.gaussian_sheet((hi[t2] - lo[t2], hi[t1] - lo[t1]), w0)
    shape = [hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0]]  # (z, y, x)
    prof = prof2.reshape(shape)
    src = S.default_pulse(S.Source(comp, tuple(lo), tuple(hi), prof, 1.0, 11.0, tfsf=tfsf),
                          S.courant_from_factor())
    dets = []
    for off in (-7, 7):
        dlo, dhi = list(lo), list(hi)
        dlo[axis], dhi[axis] = ks + off, ks + off + 1
        dets.append(S.Detector(S.DET_PLANE_E2_SUM, tuple(dlo), tuple(dhi)))
    return H.box_scene(tuple(nx), pml=(p,) * 6, eps_inv=eps_inv, sources=[src] + list(extra_sources),
                       detectors=dets, design=design, nsteps=nsteps, name="tfsf")


def back_ahead(sc):
    _, d = O.forward(sc, sc.nsteps)
    m = len(d) // 2
    return d[:m].sum(), d[m:].sum()


@pytest.mark.parametrize("axis,comp", [(2, 0), (2, 1), (0, 1), (1, 2)])
def test_tfsf_radiates_to_one_side(axis, comp):
    b, a = back_ahead(tfsf_scene(axis, axis + 1, comp))
    assert b / a < 1e-2, b / a          # travel +: the field behind the plane stays small
    b, a = back_ahead(tfsf_scene(axis, -(axis + 1), comp))
    assert a / b < 1e-2, a / b          # travel -: mirrored
    b, a = back_ahead(tfsf_scene(axis, 0, comp))
    assert 0.9 < b / a < 1.1, b / a     # a soft sheet radiates both ways


def tfsf_design_scene(nsteps=120):
    n = (30, 28, 40)
    rng = np.random.default_rng(17)
    eps_inv = np.ones((n[2], n[1], n[0]), dtype=np.float32)
    dlo, dhi = (10, 9, 22), (20, 19, 30)
    eps_inv[dlo[2]:dhi[2], dlo[1]:dhi[1], dlo[0]:dhi[0]] = S.inv(1.0 + 11.1 * rng.random((8, 10, 10)))
    pt = H.point_source(S.EY, (12, 14, 31), wavelength=10.0, amplitude=0.3)
    sc = tfsf_scene(2, 3, 0, n=n, ks=14, p=6, nsteps=nsteps, design=(dlo, dhi), eps_inv=eps_inv, extra_sources=[pt])
    sc.detectors.append(S.Detector(S.DET_PLANE_FLUX, (7, 7, 32), (23, 21, 33), axis=2))
    return sc


def test_tfsf_roundtrip_returns_initial_state_on_R():
    sc = tfsf_design_scene(150)
    init = S.random_fields(sc, 2).astype(np.float64)
    fwd, back = O.roundtrip(sc, 150, init)
    m = H.r_masks(sc)
    assert np.linalg.norm(fwd[m] - init[m]) > 0.1 * np.linalg.norm(init[m])
    assert np.linalg.norm(back[m] - init[m]) <= 1e-12 * np.linalg.norm(init[m])


def test_tfsf_time_reversal_gradient_equals_store_all():
    sc = tfsf_design_scene(100)
    g = np.random.default_rng(4).standard_normal(O.detector_total(sc, 100))
    gt, _, _ = O.gradient(sc, 100, g, O.METHOD_TIME_REVERSAL)
    gs, _, _ = O.gradient(sc, 100, g, O.METHOD_STORE_ALL)
    assert np.linalg.norm(gt - gs) <= 1e-10 * np.linalg.norm(gs)


# ---------------------------------------------------------------- GPU against the oracle --------

@pytest.fixture(scope="module")
def F(cuda_ok):
    from paper_2412_12360_b300 import fdtd
    fdtd.lib()
    return fdtd


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.gpu
@pytest.mark.parametrize("axis,tfsf,comp", [(2, 3, 0), (0, -1, 2), (1, 2, 0)])
def test_gpu_tfsf_forward_matches_oracle(F, axis, tfsf, comp):
    # 110 steps: the pulse is still inside the grid (once it has left through the layers only fp32
    # rounding noise of the total/incident cancellation is left, ~1e-7 of the peak field)
    sc = tfsf_scene(axis, tfsf, comp, n=(67, 45, 38), ks=19, nsteps=110)
    f_o, d_o = O.forward(sc, 110)
    with F.Solver(sc) as s:
        s.fdtd_forward(110)
        f_g = s.fields()
        d_g = s.detectors()
    print("tfsf axis %d dir %d: fields rel L2 %.3e, detectors %.3e" % (axis, tfsf, rel(f_g, f_o), rel(d_g, d_o)))
    assert rel(f_g, f_o) < 1e-4
    assert rel(d_g, d_o) < 1e-4


@pytest.mark.gpu
def test_gpu_tfsf_gradient_and_roundtrip(F):
    sc = tfsf_design_scene(300)
    g = np.random.default_rng(6).standard_normal(O.detector_total(sc, 300))
    grad_o, _, det_o = O.gradient(sc, 300, g, O.METHOD_TIME_REVERSAL)
    init = S.random_fields(sc, 8)
    with F.Solver(sc) as s:
        s.fdtd_forward(300, record_faces=True)
        det_g = s.detectors()
        grad_g = s.gradient(g)
        s.fdtd_set_initial_fields(init)
        s.fdtd_forward(300, record_faces=True)
        s.gradient(np.zeros(s.fdtd_detector_total()))
        back = s.fields()
    m = H.r_masks(sc)
    print("tfsf gradient rel L2 %.3e, detectors %.3e, round-trip drift %.3e" % (
        rel(grad_g, grad_o), rel(det_g, det_o), rel(back[m], init[m])))
    assert rel(det_g, det_o) < 1e-4
    assert rel(grad_g, grad_o) < 1e-3
    assert rel(back[m], init[m]) < 1e-4


@pytest.mark.gpu
def test_gpu_tfsf_with_interpolated_flux_and_checkpointing(F):
    """TFSF plane, interpolated flux detector and the treeverse gradient together, against the oracle."""
    sc = tfsf_design_scene(160)
    sc.detectors = [S.Detector(S.DET_PLANE_FLUX_INTERP, (7, 7, 30), (22, 20, 31), axis=2),
                    S.Detector(S.DET_PLANE_E2_SUM_INTERP, (7, 7, 32), (22, 20, 33))]
    g = np.random.default_rng(10).standard_normal(O.detector_total(sc, 160))
    grad_o, _, det_o = O.gradient(sc, 160, g, O.METHOD_TIME_REVERSAL)
    with F.Solver(sc) as s:
        s.fdtd_forward(160, record_faces=True)
        det_g = s.detectors()
        grad_tr = s.gradient(g)
        s.fdtd_forward(160)
        grad_ck = np.zeros(sc.design_shape(), dtype=np.float32)
        s.fdtd_backward_checkpointed(g, grad_ck, 1, 6)
    print("tfsf + interpolated detectors: detectors %.3e, time reversal %.3e, treeverse %.3e" % (
        rel(det_g, det_o), rel(grad_tr, grad_o), rel(grad_ck, grad_o)))
    assert rel(det_g, det_o) < 1e-4
    assert rel(grad_tr, grad_o) < 1e-3
    assert rel(grad_ck, grad_o) < 1e-3
