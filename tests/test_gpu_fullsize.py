"""Full-size checks in the configurations bench.py times.

design_96 (the bench workload: 96^3, 10-cell CPML, 40^3 design box, 2000 steps): the whole detector
plane and the whole dL/deps against the FP64 oracle. waveguide_600 (600^3, 216 M cells): properties
that hold at any size, on the full grid for a shortened run: the fp32 time-reversal round trip
returns to the (zero) initial state, and dL/drho agrees with a central difference along a uniform
density shift. waveguide_600, the 240x240x960 batch member and the two largest served grids:
element-wise parity of fields, probe series and dL/deps at sampled points, from the oracle's solve
of each point's light cone.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_12360_b300 import scenes as S
from tests import _helpers as H

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


@pytest.mark.parametrize("config", ["waveguide_600", "waveguide_batch_member", "served_200", "served_128x128x256"])
def test_full_size_light_cone_parity(cuda_ok, config):
    """Element-wise parity on the full grids of the large configurations, in the launch configuration
    the bench times (same grid, so the same tiles, z-chunks and stage rings): from a seeded random
    state on the PML-free region, n steps forward and the time-reversal gradient. In n steps a Yee
    update moves information at most one cell per step, so the fields within r cells of a probe point
    q, the probe's series and dL/deps on the box of radius r around q depend only on the state and the
    permittivity within n + r cells of q (the adjoint of the probe reaches the box within n steps
    too). The FP64 oracle solves that sub-box (PEC walls n + r + 3 cells away, too far to matter) from
    the same state and gives those values exactly. Probe points sit on tile and z-chunk boundaries and
    in the random-density design region."""
    import torch
    from paper_2412_12360_b300 import fdtd
    n_steps, r = 12, 3
    M = n_steps + r + 3
    if config == "waveguide_600":
        sc = S.waveguide_600(n_steps)
        probes = [(300, 300, 300), (64, 48, 60), (543, 561, 541)]
    elif config == "waveguide_batch_member":
        sc = S.waveguide_batch_member(0, n_steps)
        probes = [(120, 120, 480), (32, 64, 240), (207, 200, 928)]
    elif config == "served_200":  # the largest grid of the served stream
        sc = S.design_box_scene((200, 200, 200), 10, 100, n_steps, 10007)
        probes = [(100, 100, 100), (32, 48, 30), (171, 160, 170)]
    else:
        sc = S.design_box_scene((128, 128, 256), 10, 64, n_steps, 10003)
        probes = [(64, 64, 128), (96, 32, 40), (33, 96, 227)]
    nx, ny, nz = sc.n
    p = sc.pml
    for q in probes:  # the sub-boxes stay inside the PML-free region
        for d in range(3):
            assert p[2 * d] <= q[d] - M and q[d] + M < sc.n[d] - p[2 * d + 1], (q, d)
    q0 = probes[0]
    sc.sources = []
    sc.detectors = [S.Detector(S.DET_POINT_SERIES, q, tuple(v + 1 for v in q), component=S.EZ) for q in probes]
    sc.design_lo = tuple(v - r for v in q0)
    sc.design_hi = tuple(v + r + 1 for v in q0)
    dev = torch.device("cuda")
    gen = torch.Generator(device=dev).manual_seed(77)
    init = torch.zeros((6, nz, ny, nx), dtype=torch.float32, device=dev)
    init[:, p[4]:nz - p[5], p[2]:ny - p[3], p[0]:nx - p[1]] = (
        2 * torch.rand((6, nz - p[4] - p[5], ny - p[2] - p[3], nx - p[0] - p[1]), generator=gen, device=dev) - 1)
    g = np.random.default_rng(78).standard_normal(len(probes) * n_steps)
    fields = torch.empty_like(init)
    with fdtd.Solver(sc) as s:
        s.fdtd_set_initial_fields(init)
        s.fdtd_forward(n_steps, record_faces=True)
        s.fdtd_get_fields(fields)
        det_g = s.detectors()
        grad_g = s.gradient(g)
    for qi, q in enumerate(probes):
        lo = [v - M for v in q]
        sl = (slice(None), slice(lo[2], lo[2] + 2 * M + 1), slice(lo[1], lo[1] + 2 * M + 1),
              slice(lo[0], lo[0] + 2 * M + 1))
        sub_init = init[sl].double().cpu().numpy()
        eps_sub = np.ascontiguousarray(sc.eps_inv[sl[1:]])
        c = (M, M, M)
        sub = H.box_scene((2 * M + 1,) * 3, eps_inv=eps_sub, courant=sc.courant,
                          detectors=[S.Detector(S.DET_POINT_SERIES, c, (M + 1,) * 3, component=S.EZ)],
                          design=((M - r,) * 3, (M + r + 1,) * 3), nsteps=n_steps)
        g_sub = g[qi * n_steps:(qi + 1) * n_steps]
        grad_o, _, det_o = O.gradient(sub, n_steps, g_sub, O.METHOD_STORE_ALL, init=sub_init)
        f_o, _ = O.forward(sub, n_steps, init=sub_init)
        blk = (slice(None), slice(M - r, M + r + 1), slice(M - r, M + r + 1), slice(M - r, M + r + 1))
        f_g = fields[(slice(None), slice(q[2] - r, q[2] + r + 1), slice(q[1] - r, q[1] + r + 1),
                      slice(q[0] - r, q[0] + r + 1))].double().cpu().numpy()
        e_f = float(np.max(np.abs(f_g - f_o[blk])) / np.max(np.abs(f_o[blk])))
        e_d = float(np.max(np.abs(det_g[qi * n_steps:(qi + 1) * n_steps] - det_o)) / np.max(np.abs(det_o)))
        msg = "%s probe %s: fields %.2e, probe series %.2e" % (config, q, e_f, e_d)
        if qi == 0:
            e_g = rel(grad_g, grad_o)
            msg += ", dL/deps %.2e" % e_g
            assert e_g < 1e-4, msg
        print(msg)
        assert e_f < 1e-5 and e_d < 1e-5, msg
