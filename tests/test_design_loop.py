"""Inverse-design loop (arXiv 2412.12360 Sec. 3.2-3.3): the FP64 reference pinned to closed forms
(CPU), and the CUDA projection, Adam step and whole loop against it (GPU).

Pins: the projection's end points, its beta -> 0 limit (identity) and large-beta limit (a step), its
derivative against central differences; Adam's first step from zero moments, which is
-lr g / (|g| + eps), and its repeat under a constant gradient; clamping to [0, 1]; a first design
iteration with a small step lowering the loss (descent).
"""
import math

import numpy as np
import pytest

from oracle import design as D
from oracle import oracle as O
from paper_2412_12360_b300 import scenes as S


# ---------------------------------------------------------------- oracle pins (CPU) ------------

def test_projection_end_points_and_limits():
    th = np.linspace(0.0, 1.0, 101)
    for beta in (1.0, 8.0, 64.0):
        for eta in (0.3, 0.5, 0.7):
            p = D.projection(th, beta, eta)
            assert abs(p[0]) < 1e-15 and abs(p[-1] - 1.0) < 1e-15
            assert np.all(np.diff(p) >= 0) and (beta > 8.0 or np.all(np.diff(p) > 0))  # saturates in fp64
    assert abs(D.projection(0.5, 8.0, 0.5) - 0.5) < 1e-15          # symmetric about eta = 1/2
    assert np.max(np.abs(D.projection(th, 1e-4, 0.4) - th)) < 1e-8  # beta -> 0: identity
    assert np.array_equal(D.projection(th, 0.0, 0.4), th)
    p = D.projection(th, 400.0, 0.5)                                # beta -> inf: a step at eta
    assert np.all(p[th < 0.45] < 1e-6) and np.all(p[th > 0.55] > 1 - 1e-6)


def test_projection_derivative_central_differences():
    th = np.linspace(0.02, 0.98, 49)
    h = 1e-6
    for beta, eta in ((0.0, 0.5), (2.0, 0.5), (8.0, 0.35), (30.0, 0.6)):
        fd = (D.projection(th + h, beta, eta) - D.projection(th - h, beta, eta)) / (2 * h)
        an = D.projection_grad(th, beta, eta)
        assert np.max(np.abs(fd - an)) <= 1e-7 * max(1.0, np.max(np.abs(an)))


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(3)
    th0 = rng.uniform(0.3, 0.7, 200)
    g = rng.standard_normal(200) * 10.0 ** rng.uniform(-3, 3, 200)
    lr, eps = 1e-2, 1e-8
    th1, m1, v1, rho1 = D.adam_step(th0, 0.0, 0.0, g, 1, lr, 0.9, 0.999, eps)
    # bias-corrected moments after one step are g and g^2
    assert np.allclose(th1, th0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g, rtol=1e-15) and np.allclose(v1, 0.001 * g * g, rtol=1e-15)
    assert np.array_equal(rho1, th1)                                # beta = 0
    th2, _, _, _ = D.adam_step(th1, m1, v1, g, 2, lr, 0.9, 0.999, eps)
    assert np.allclose(th2 - th1, th1 - th0, rtol=1e-12, atol=1e-15)  # constant gradient: same step
    # clamped to [0, 1]
    th, _, _, rho = D.adam_step(np.array([0.001, 0.999]), 0.0, 0.0, np.array([1.0, -1.0]), 1, 0.1, proj_beta=8.0)
    assert np.array_equal(th, [0.0, 1.0]) and abs(rho[0]) < 1e-15 and abs(rho[1] - 1.0) < 1e-15


def tiny_design_scene(nsteps=160):
    return S.design_box_scene((26, 24, 28), 5, 8, nsteps, 21, 1.0, 12.1, 10.0, "design_tiny")


def neg_sum(det):
    return -float(np.sum(det)), -np.ones_like(det)


def test_first_design_iteration_descends():
    sc = tiny_design_scene()
    theta0 = np.full(sc.design_shape(), 0.5)
    losses, _ = D.design_loop(sc, sc.nsteps, theta0, 2, neg_sum, 1e-3, 1.0, 12.1)
    assert losses[1] < losses[0]


# ---------------------------------------------------------------- GPU against the oracle --------

@pytest.fixture(scope="module")
def F(cuda_ok):
    from paper_2412_12360_b300 import fdtd
    fdtd.lib()
    return fdtd


@pytest.mark.gpu
def test_gpu_projection_and_adam_step(F):
    import torch
    sc = tiny_design_scene()
    shp = sc.design_shape()
    rng = np.random.default_rng(5)
    th = rng.uniform(0, 1, shp).astype(np.float32)
    m = (rng.standard_normal(shp) * 1e-2).astype(np.float32)
    v = (rng.uniform(0, 1, shp) * 1e-3).astype(np.float32)
    g = (rng.standard_normal(shp) * 0.1).astype(np.float32)
    dev = torch.device("cuda")
    T = {k: torch.from_numpy(x.copy()).to(dev) for k, x in (("th", th), ("m", m), ("v", v), ("g", g))}
    rho = torch.empty_like(T["th"])
    with F.Solver(sc) as s:
        s.fdtd_design_project(T["th"], rho, 6.0, 0.45)
        torch.cuda.synchronize()
        assert np.max(np.abs(rho.cpu().numpy() - D.projection(th, 6.0, 0.45))) < 2e-6
        s.fdtd_design_adam_step(T["g"], T["th"], T["m"], T["v"], rho, 3, 0.05, 0.9, 0.999, 1e-8, 6.0, 0.45)
        torch.cuda.synchronize()
        s.fdtd_design_adam_step(T["g"], T["th"], T["m"], T["v"], rho, 3, 0.05, 0.9, 0.999, 1e-8, 0.0, 0.45)
        torch.cuda.synchronize()
    t1, m1, v1, _ = D.adam_step(th, m, v, g, 3, 0.05, 0.9, 0.999, 1e-8, 6.0, 0.45)
    t2, m2, v2, r2 = D.adam_step(t1, m1, v1, g, 3, 0.05, 0.9, 0.999, 1e-8, 0.0, 0.45)
    assert np.max(np.abs(T["th"].cpu().numpy() - t2)) < 1e-5
    assert np.max(np.abs(rho.cpu().numpy() - r2)) < 1e-5
    assert np.max(np.abs(T["m"].cpu().numpy() - m2)) <= 1e-5 * np.max(np.abs(m2))
    assert np.max(np.abs(T["v"].cpu().numpy() - v2)) <= 1e-5 * np.max(np.abs(v2))


@pytest.mark.gpu
def test_gpu_design_loop_matches_oracle(F):
    import torch
    from paper_2412_12360_b300 import design
    sc = tiny_design_scene()
    iters, lr = 4, 0.02
    beta_of = lambda it: 0.0 if it < 2 else 4.0
    theta0 = np.random.default_rng(11).uniform(0.3, 0.7, sc.design_shape())
    th32 = theta0.astype(np.float32)
    with F.Solver(sc) as s:
        loop = design.DesignLoop(s, torch.from_numpy(th32.copy()).cuda(), 1.0, 12.1, sc.nsteps,
                                 lambda det: (-det.sum(), -torch.ones_like(det)), lr=lr, beta_of=beta_of)
        losses_g = loop.run(iters)
        theta_g = loop.theta.cpu().numpy()
    losses_o, theta_o = D.design_loop(sc, sc.nsteps, th32.astype(np.float64), iters, neg_sum, lr, 1.0, 12.1, beta_of)
    print("design loop losses gpu %s oracle %s" % (losses_g, losses_o))
    for a, b in zip(losses_g, losses_o):
        assert abs(a - b) <= 1e-4 * abs(b)
    assert losses_g[-1] < losses_g[0]
    # Adam moves every variable by about lr per step whatever the size of its gradient, so variables
    # whose gradient is near fp32 noise may move the other way; those stay within 2 lr per step
    d = np.abs(theta_g - theta_o)
    assert np.max(d) <= 2 * lr * iters + 1e-6
    assert np.mean(d < 1e-4) > 0.97, np.mean(d < 1e-4)
