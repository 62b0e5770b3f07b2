"""Face-history segments (fdtd_set_segment_steps): the reverse sweep of a forward that kept only its last
segment's faces, regenerating the earlier segments from stored start states, gives the gradient of the
whole-history sweep (to the inverse step's rounding drift, which segments reset) and of the FP64
oracle, with either reverse-step kind, several segment lengths and a TFSF plane; and the history it
holds is the bounded size the library reports."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_12360_b300 import scenes as S
from tests import _helpers as H


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def test_history_bytes_of_segments_on_the_host():
    from paper_2412_12360_b300 import fdtd as F
    sc = S.design_box_scene((40, 36, 44), 6, 12, 300, 71, name="seg")
    whole = F.history_bytes(sc, 300, 0)
    seg = F.history_bytes(sc, 300, 50)                  # 6 segments: 50 steps of faces, 4 start states
    per_step = whole // 300
    assert F.history_bytes(sc, 300, 300) == whole and F.history_bytes(sc, 300, 400) == whole
    assert seg > 50 * per_step and (seg - 50 * per_step) % 4 == 0
    assert F.history_bytes(sc, 300, -1) == -1


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["0", "1"])
@pytest.mark.parametrize("seg", [1, 37, 50, 149])
def test_segmented_gradient_equals_whole_history_gradient(cuda_ok, kind, seg, monkeypatch):
    from paper_2412_12360_b300 import fdtd as F
    monkeypatch.setenv("FDTD_REV_FUSED", kind)
    sc = S.design_box_scene((40, 36, 44), 6, 12, 150, 71, name="seg", tfsf=seg == 37)
    g = np.random.default_rng(5).standard_normal(O.detector_total(sc, sc.nsteps))
    with F.Solver(sc) as s:
        s.fdtd_forward(sc.nsteps, record_faces=True)
        det0 = s.detectors()
        grad0 = s.gradient(g)
        held0 = s.fdtd_bytes_allocated()
    with F.Solver(sc) as s:
        s.fdtd_set_segment_steps(seg)
        for _ in range(2):  # the second solve replays the captured loops
            s.fdtd_forward(sc.nsteps, record_faces=True)
            det1 = s.detectors()
            grad1 = s.gradient(g)
        held1 = s.fdtd_bytes_allocated()
    grad_o, _, det_o = O.gradient(sc, sc.nsteps, g, O.METHOD_TIME_REVERSAL)
    e01, e1o = _rel(grad1, grad0), _rel(grad1, grad_o)
    print("segments of %d steps (reverse kind %s): dL/deps vs whole history %.2e, vs oracle %.2e; device bytes "
          "%d -> %d" % (seg, kind, e01, e1o, held0, held1))
    assert np.array_equal(det1, det0)            # the forward and its detectors are unchanged
    assert e01 <= 1e-4 and e1o < 1e-3
    whole = F.history_bytes(sc, sc.nsteps, 0)
    assert held1 - held0 == F.history_bytes(sc, sc.nsteps, seg) - whole


@pytest.mark.gpu
def test_segmented_backward_is_refused_by_the_grouped_form(cuda_ok):
    from paper_2412_12360_b300 import fdtd as F
    sc = S.design_box_scene((40, 36, 44), 6, 12, 100, 71, name="seg")
    with F.Solver(sc) as s:
        s.fdtd_set_segment_steps(30)
        with pytest.raises(F.FDTDError) as e:
            s.fdtd_begin(100, record_faces=True)
        assert e.value.code == F.FDTD_ERR_INVALID_ARG
        s.fdtd_begin(20, record_faces=True)      # a single segment is an ordinary whole history


def test_history_plan_keeps_segments_or_recomputes_by_budget():
    """autograd.history_plan: whole histories while they fit, then the longest segments that fit, then
    recomputation; the extra forward steps are T - L per segmented design and T per recomputed one."""
    import torch  # noqa: F401  (autograd imports torch)
    from paper_2412_12360_b300 import autograd, fdtd as F
    T = 300
    scs = [S.design_box_scene((40, 36, 44), 6, 12, T, 71 + b, name="p%d" % b) for b in range(3)]
    adj = [F.adjoint_bytes(sc) for sc in scs]
    base = sum(F.footprint_bytes(sc, T, record_faces=False) for sc in scs) - sum(adj) + max(adj)
    whole = F.history_bytes(scs[0], T, 0)
    plan, extra = autograd.history_plan(scs, T, base + 3 * whole)
    assert plan == [0, 0, 0] and extra == 0
    seg2 = F.history_bytes(scs[0], T, 150)
    plan, extra = autograd.history_plan(scs, T, base + whole + seg2)
    assert plan == [0, 150, -1]
    assert extra == (T - 150) + T
    plan, extra = autograd.history_plan(scs, T, base)
    assert plan == [-1, -1, -1] and extra == 3 * T
