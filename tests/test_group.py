"""Grouped solves (fdtd_group_step / fdtd_group_forward / fdtd_group_backward): several handles advanced
by one launch per kernel and time step give each handle bitwise the detectors, dL/deps and fields it
gets when solved alone, also when handles join the group at different steps and in different phases,
and one of them matches the FP64 oracle within the parity bars."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_12360_b300 import scenes as S
from tests import _helpers as H


def group_scenes():
    """Four scenes of different shapes, CPML widths, sources, detectors and step counts."""
    out = [S.design_box_scene((40, 36, 44), 6, 12, 150, 71, name="g0"),
           S.design_box_scene((64, 64, 64), 10, 32, 110, 72, name="g1", tfsf=True),
           S.design_box_scene((45, 38, 41), 6, 12, 130, 73, name="g2", interp=True)]
    n = (67, 37, 29)
    nx, ny, nz = n
    rng = np.random.default_rng(74)
    eps_inv = np.ones((nz, ny, nx), dtype=np.float32)
    dlo, dhi = (41, 9, 8), (60, 28, 21)
    eps_inv[dlo[2]:dhi[2], dlo[1]:dhi[1], dlo[0]:dhi[0]] = S.inv(
        1.0 + 11.1 * rng.random((dhi[2] - dlo[2], dhi[1] - dlo[1], dhi[0] - dlo[0])))
    pt = H.point_source(S.EZ, (30, 18, 14), wavelength=9.0)
    dets = [H.point_probe(S.EZ, (52, 18, 16)), H.point_probe(S.HY, (20, 20, 12)),
            S.Detector(S.DET_PLANE_FLUX, (42, 6, 6), (44, 31, 23), axis=0),
            S.Detector(S.DET_PLANE_E2_SUM, (8, 6, 20), (60, 31, 21))]
    out.append(H.box_scene(n, pml=(5, 7, 4, 6, 6, 3), eps_inv=eps_inv, sources=[pt], detectors=dets,
                           design=(dlo, dhi), nsteps=140, name="g3"))
    return out


def _gvec(sc, seed):
    return np.random.default_rng(seed).standard_normal(O.detector_total(sc, sc.nsteps))


def _alone(F, sc, g):
    with F.Solver(sc) as s:
        s.fdtd_forward(sc.nsteps, record_faces=True)
        det = s.detectors()
        grad = s.gradient(g)
        fields = s.fields()
    return det, grad, fields


def test_group_abi_rejects_bad_groups_on_the_host():
    from paper_2412_12360_b300 import fdtd as F
    L = F.lib()
    assert L.fdtd_group_step(None, 1, 1) == F.FDTD_ERR_INVALID_ARG
    arr = (C.c_void_p * 9)()
    assert L.fdtd_group_step(arr, 0, 1) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_group_step(arr, 9, 1) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_group_step(arr, 2, 1) == F.FDTD_ERR_INVALID_ARG  # NULL handles
    assert L.fdtd_phase(None, None, None) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_begin(None, 10, 0) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_finish_backward(None, None) == F.FDTD_ERR_INVALID_ARG


def _solvers(F, scs, stream, monkeypatch, kinds):
    """Solvers on one stream; kinds[r] the reverse kind of solver r (the in-place pair, or the fused
    kernels), so a group holds both."""
    out = []
    for sc, kind in zip(scs, kinds):
        monkeypatch.setenv("FDTD_REV_FUSED", kind)
        out.append(F.Solver(sc, stream=stream))
    monkeypatch.delenv("FDTD_REV_FUSED")
    return out


@pytest.mark.gpu
def test_group_solves_equal_standalone_solves_bitwise(cuda_ok, monkeypatch):
    import torch
    from paper_2412_12360_b300 import fdtd as F
    scs = group_scenes()
    gs = [_gvec(sc, 80 + r) for r, sc in enumerate(scs)]
    kinds = ["1", "0", "1", "0"]
    alone = []
    for sc, g, kind in zip(scs, gs, kinds):
        monkeypatch.setenv("FDTD_REV_FUSED", kind)
        alone.append(_alone(F, sc, g))
    stream = torch.cuda.Stream()
    solvers = _solvers(F, scs, stream, monkeypatch, kinds)
    F.group_forward(solvers, [sc.nsteps for sc in scs], record_faces=True)
    dets = [s.detectors() for s in solvers]
    grads = [np.zeros(sc.design_shape(), dtype=np.float32) for sc in scs]
    F.group_backward(solvers, gs, grads)
    for s in solvers:
        s.fdtd_synchronize()
    for r, (sc, s) in enumerate(zip(scs, solvers)):
        a_det, a_grad, a_fields = alone[r]
        assert np.array_equal(dets[r], a_det), sc.name
        assert np.array_equal(grads[r], a_grad), sc.name
        assert np.array_equal(s.fields(), a_fields), sc.name
        assert s.fdtd_phase()[0] == F.PHASE_IDLE
        s.close()


@pytest.mark.gpu
def test_group_with_handles_joining_in_different_phases(cuda_ok, monkeypatch):
    """Continuous batching: a handle starts alone, others join while it runs (one in its forward phase,
    one after another has reached its reverse sweep), and a finished one leaves; every result is the
    standalone result bitwise, and the first one matches the oracle."""
    import torch
    from paper_2412_12360_b300 import fdtd as F
    scs = group_scenes()
    gs = [_gvec(sc, 90 + r) for r, sc in enumerate(scs)]
    kinds = ["0", "1", "0", "1"]
    alone = []
    for sc, g, kind in zip(scs, gs, kinds):
        monkeypatch.setenv("FDTD_REV_FUSED", kind)
        alone.append(_alone(F, sc, g))
    stream = torch.cuda.Stream()
    solvers = _solvers(F, scs, stream, monkeypatch, kinds)
    grads = [np.zeros(sc.design_shape(), dtype=np.float32) for sc in scs]
    dets = [None] * len(scs)
    active = []
    joins = {0: 0, 1: 37, 2: 90, 3: 200}   # tick at which each request arrives
    tick = 0
    done, started = set(), set()
    while len(done) < len(scs):
        for r, t in joins.items():
            if t <= tick and r not in started:
                solvers[r].fdtd_begin(scs[r].nsteps, record_faces=True)
                active.append(r)
                started.add(r)
        # handles whose forward finished: read the detectors and start the reverse sweep
        for r in list(active):
            ph, _ = solvers[r].fdtd_phase()
            if ph == F.PHASE_FORWARD_DONE:
                dets[r] = solvers[r].detectors()
                solvers[r].fdtd_begin_backward(gs[r])
            elif ph == F.PHASE_DONE:
                solvers[r].fdtd_finish_backward(grads[r])
                solvers[r].fdtd_synchronize()
                active.remove(r)
                done.add(r)
        if active:
            F.group_step([solvers[r] for r in active], 7)
        tick += 7 if active else 1
        assert tick < 10000
    for r, sc in enumerate(scs):
        assert np.array_equal(dets[r], alone[r][0]), sc.name
        assert np.array_equal(grads[r], alone[r][1]), sc.name
    sc = scs[0]
    grad_o, _, det_o = O.gradient(sc, sc.nsteps, gs[0], O.METHOD_TIME_REVERSAL)
    assert np.linalg.norm(grads[0] - grad_o) / np.linalg.norm(grad_o) < 1e-3
    assert np.linalg.norm(dets[0] - det_o) / np.linalg.norm(det_o) < 1e-4
    for s in solvers:
        s.close()


@pytest.mark.gpu
def test_group_step_refuses_handles_on_different_streams(cuda_ok):
    import torch
    from paper_2412_12360_b300 import fdtd as F
    scs = group_scenes()[:2]
    a = F.Solver(scs[0], stream=torch.cuda.Stream())
    b = F.Solver(scs[1], stream=torch.cuda.Stream())
    a.fdtd_begin(10)
    b.fdtd_begin(10)
    with pytest.raises(F.FDTDError) as e:
        F.group_step([a, b], 1)
    assert e.value.code == F.FDTD_ERR_INVALID_ARG
    with pytest.raises(F.FDTDError) as e:
        F.group_step([a, a], 1)
    assert e.value.code == F.FDTD_ERR_INVALID_ARG
    a.close()
    b.close()
