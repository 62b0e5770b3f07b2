"""Served (continuous-batching) solves and the autograd Function on the GPU.

Each served request gives bitwise the same detectors and dL/deps alone and in the mix; the memory
budget bounds what runs at once; FDTDSolve's dL/drho matches the FP64 oracle's dL/deps scaled by
deps/drho, in both its keep and recompute modes.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_12360_b300 import scenes as S

pytestmark = pytest.mark.gpu


def _mix(n=6):
    rng = np.random.default_rng(5)
    out = []
    sizes = [(40, 40, 40), (48, 40, 56), (56, 56, 56), (40, 48, 40)]
    for r in range(n):
        nn = sizes[r % len(sizes)]
        out.append(S.design_box_scene(nn, 6, 12, int(rng.integers(150, 260)), 900 + r, name="mix%d" % r))
    return out


def test_served_results_equal_alone_and_in_the_mix(cuda_ok):
    from paper_2412_12360_b300 import serve
    scenes = _mix(6)
    alone = serve.run_sequential(scenes)
    with serve.Server(max_inflight=4) as srv:
        futs = [srv.submit(sc) for sc in scenes]
        res = [f.result(timeout=600) for f in futs]
        peak = srv.peak_inflight
    assert peak >= 2
    for (d0, g0), r in zip(alone, res):
        assert np.array_equal(d0, r.detectors)
        assert np.array_equal(g0, r.dL_deps)


def test_served_cancellation_and_failure_reporting(cuda_ok):
    """A queued request the client cancels is never admitted; one whose fields blow up (a NaN in its
    design permittivity, an input) fails with NONFINITE; the others complete with their standalone
    results."""
    from concurrent.futures import CancelledError

    from paper_2412_12360_b300 import fdtd, serve
    scenes = _mix(3)
    bad = _mix(1)[0]
    bad.eps_inv = bad.eps_inv.copy()
    lo, hi = bad.design_lo, bad.design_hi
    bad.eps_inv[(lo[2] + hi[2]) // 2, (lo[1] + hi[1]) // 2, (lo[0] + hi[0]) // 2] = np.nan
    alone = serve.run_sequential([scenes[0], scenes[2]])
    with serve.Server(max_inflight=1) as srv:
        f0 = srv.submit(scenes[0])
        f1 = srv.submit(scenes[1])
        fb = srv.submit(bad)
        f2 = srv.submit(scenes[2])
        assert f1.cancel()  # one slot: the first request runs, the rest wait
        r0, r2 = f0.result(timeout=600), f2.result(timeout=600)
        with pytest.raises(fdtd.FDTDError) as e:
            fb.result(timeout=600)
        assert "NONFINITE" in str(e.value)
        with pytest.raises(CancelledError):
            f1.result(timeout=1)
        assert srv.cancelled == 1
    for (d0, g0), r in zip(alone, (r0, r2)):
        assert np.array_equal(d0, r.detectors)
        assert np.array_equal(g0, r.dL_deps)


def test_served_admission_bounded_by_budget(cuda_ok):
    from paper_2412_12360_b300 import fdtd, serve
    scenes = _mix(5)
    fps = [fdtd.footprint_bytes(sc, sc.nsteps) for sc in scenes]
    budget = sum(sorted(fps)[-2:])  # room for the two largest at most
    with serve.Server(budget_bytes=budget, max_inflight=8) as srv:
        res = [f.result(timeout=600) for f in [srv.submit(sc) for sc in scenes]]
        peak = srv.peak_inflight
    assert len(res) == 5 and 1 <= peak <= 3
    lat = serve.latency_stats(res)
    assert lat["p99_s"] >= lat["p50_s"] > 0


@pytest.mark.parametrize("mode", ["keep", "recompute", 1, [40, -1], [0, 55]])
def test_autograd_density_gradient_matches_oracle(cuda_ok, mode):
    import torch
    from paper_2412_12360_b300 import autograd, fdtd
    scenes = [S.design_box_scene((40, 36, 44), 6, 12, 160, 31 + b, name="ad%d" % b) for b in range(2)]
    eps_lo, eps_hi = scenes[0].extra["eps_lo"], scenes[0].extra["eps_hi"]
    rho = torch.stack([torch.from_numpy(sc.extra["rho"]) for sc in scenes]).cuda().requires_grad_(True)
    solvers = [fdtd.Solver(sc) for sc in scenes]
    det = autograd.solve(rho, solvers, eps_lo, eps_hi, 160, mode)
    w = torch.linspace(0.5, 1.5, det.shape[1], dtype=torch.float64, device="cuda")
    loss = (det * w).sum()
    loss.backward()
    grad = rho.grad.cpu().numpy()
    for b, sc in enumerate(scenes):
        g = w.cpu().numpy()
        grad_o, _, det_o = O.gradient(sc, 160, g, O.METHOD_TIME_REVERSAL)
        ref = (eps_hi - eps_lo) * grad_o
        e = np.linalg.norm(grad[b] - ref) / np.linalg.norm(ref)
        assert e < 1e-3, e
        assert np.linalg.norm(det[b].detach().cpu().numpy() - det_o) / np.linalg.norm(det_o) < 1e-4
    for s in solvers:
        s.close()


def test_autograd_orders_solver_streams_against_torch_streams(cuda_ok):
    """Solvers on streams of their own, the call made under another torch stream: the inputs are
    produced on torch's current stream right before the call and the loss reads the outputs right
    after it, so a missing ordering between the streams would show as wrong values."""
    import torch
    from paper_2412_12360_b300 import autograd, fdtd
    scenes = [S.design_box_scene((40, 36, 44), 6, 12, 160, 31 + b, name="as%d" % b) for b in range(2)]
    eps_lo, eps_hi = scenes[0].extra["eps_lo"], scenes[0].extra["eps_hi"]
    solver_streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    solvers = [fdtd.Solver(sc, stream=st) for sc, st in zip(scenes, solver_streams)]
    caller = torch.cuda.Stream()
    rho0 = torch.stack([torch.from_numpy(sc.extra["rho"]) for sc in scenes]).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(caller):
        big = torch.empty(64 * 1024 * 1024, device="cuda").uniform_()   # keeps the caller's stream busy
        rho = (rho0 + 0.0 * big[: rho0.numel()].view_as(rho0)).requires_grad_(True)
        det = autograd.solve(rho, solvers, eps_lo, eps_hi, 160, "keep")
        w = torch.linspace(0.5, 1.5, det.shape[1], dtype=torch.float64, device="cuda")
        loss = (det * w).sum()
        loss.backward()
    torch.cuda.synchronize()
    grad = rho.grad.cpu().numpy()
    for b, sc in enumerate(scenes):
        grad_o, _, det_o = O.gradient(sc, 160, w.cpu().numpy(), O.METHOD_TIME_REVERSAL)
        ref = (eps_hi - eps_lo) * grad_o
        assert np.linalg.norm(grad[b] - ref) / np.linalg.norm(ref) < 1e-3
        assert np.linalg.norm(det[b].detach().cpu().numpy() - det_o) / np.linalg.norm(det_o) < 1e-4
    for s in solvers:
        s.close()
