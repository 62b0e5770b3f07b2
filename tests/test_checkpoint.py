"""Checkpointing gradient, the recomputation alternative to time reversal (arXiv 2412.12360 Sec. 2.2).

Host pins (CPU, from a dry run of the schedule the GPU runs): recursive halving evaluates
n + (n/2) log2 n forward steps for n = 2^j (the paper's
"n/2 log2 n additional forward function calls" beyond the n taped ones); the treeverse schedule
matches the binomial-checkpointing closed form T = r l - C(c + r - 1, c + 1), r the least integer with
l <= C(c + r - 1, c), for c stored states (c = 1 gives l (l + 1) / 2, c >= l gives 2 l - 1).
GPU: both schedules give the time-reversal gradient and the FP64 oracle's, and evaluate exactly the
forward steps their schedule predicts.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_12360_b300 import fdtd


def test_recursive_halving_forward_steps():
    for j in range(0, 13):
        n = 2 ** j
        assert fdtd.checkpoint_cost(n, 0) == n + (n // 2) * j


def binomial_cost(l, c):
    r = 1
    while math.comb(c + r - 1, c) < l:
        r += 1
    return r * l - math.comb(c + r - 1, c + 1)


def test_treeverse_binomial_closed_form():
    for c in (1, 2, 3, 5, 8):
        for l in list(range(1, 60)) + [97, 200, 333]:
            assert fdtd.checkpoint_cost(l, 1, c) == binomial_cost(l, c), (l, c)
    # long runs (the paper's 5 nm and 2.5 nm cases have 20980 and 41960 steps) use the closed form
    # for the splits; the schedule they give still evaluates the closed-form count
    for l, c in ((4097, 5), (20980, 10), (41960, 30), (9999, 3)):
        assert fdtd.checkpoint_cost(l, 1, c) == binomial_cost(l, c), (l, c)
    assert fdtd.checkpoint_cost(50, 1, 1) == 50 * 51 // 2
    assert fdtd.checkpoint_cost(40, 1, 40) == 79
    for n in (64, 100, 256):  # with as many states as halving uses, treeverse never does worse
        depth = math.ceil(math.log2(n)) + 1
        assert fdtd.checkpoint_cost(n, 1, depth) <= fdtd.checkpoint_cost(n, 0)


@pytest.fixture(scope="module")
def F(cuda_ok):
    fdtd.lib()
    return fdtd


@pytest.mark.gpu
def test_gpu_checkpointed_gradient_equals_time_reversal(F):
    from tests.test_gpu_parity import ragged_scene
    sc = ragged_scene(200)
    g = np.random.default_rng(12).standard_normal(O.detector_total(sc, 200))
    grad_o, _, _ = O.gradient(sc, 200, g, O.METHOD_TIME_REVERSAL)
    with F.Solver(sc) as s:
        s.fdtd_forward(200, record_faces=True)
        grad_tr = s.gradient(g)
        out = {}
        for method, slots in ((0, 0), (1, 4), (1, 1)):
            s.fdtd_forward(200)
            d = np.zeros(sc.design_shape(), dtype=np.float32)
            steps = s.fdtd_backward_checkpointed(g, d, method, slots)
            assert steps == fdtd.checkpoint_cost(200, method, slots)
            out[(method, slots)] = d
    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))
    for key, d in out.items():
        print("checkpointed %s: rel to time reversal %.3e, to oracle %.3e" % (key, rel(d, grad_tr), rel(d, grad_o)))
        assert rel(d, grad_tr) < 1e-4
        assert rel(d, grad_o) < 1e-3
