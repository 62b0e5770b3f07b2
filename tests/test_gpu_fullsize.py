"""Full-size checks in the configurations bench.py times.

design_96 (the bench workload: 96^3, 10-cell CPML, 40^3 design box, 2000 steps): the whole detector
plane and the whole dL/deps against the FP64 oracle. waveguide_600 (600^3, 216 M cells): properties
that hold at any size, on the full grid for a shortened run: the fp32 time-reversal round trip
returns to the (zero) initial state, and dL/drho agrees with a central difference along a uniform
density shift. design_96_tfsf and design_96_interp (400 steps): detectors and dL/deps against the
oracle. waveguide_600, the 240x240x960 batch member and the two largest served grids:
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


@pytest.mark.parametrize("variant", ["tfsf", "interp"])
def test_design96_variants_match_oracle(cuda_ok, variant):
    """The bench's design_96_tfsf and design_96_interp workloads (the same 96^3 grid and launch
    configuration), shortened to 400 steps so that the beam has crossed the detector plane: the
    whole detector output and dL/deps against the FP64 oracle."""
    from paper_2412_12360_b300 import fdtd
    nsteps = 400
    sc = S.design_box_scene((96, 96, 96), 10, 40, nsteps, 1234, 1.0, 12.1, 20.0, "design_96_" + variant,
                            tfsf=variant == "tfsf", interp=variant == "interp")
    g = np.random.default_rng(79).standard_normal(O.detector_total(sc, nsteps))
    grad_o, _, det_o = O.gradient(sc, nsteps, g, O.METHOD_TIME_REVERSAL)
    with fdtd.Solver(sc) as s:
        s.fdtd_forward(nsteps, record_faces=True)
        det_g = s.detectors()
        grad_g = s.gradient(g)
    e_det, e_grad = rel(det_g, det_o), rel(grad_g, grad_o)
    print("design_96_%s %d steps: detector rel L2 %.2e, dL/deps rel L2 %.2e" % (variant, nsteps, e_det, e_grad))
    assert np.max(np.abs(det_o)) > 0 and np.max(np.abs(grad_o)) > 0
    assert e_det < 1e-4
    assert e_grad < 1e-3


def _window(sc, q, M):
    """The sub-box of the cells within M of q, clipped to the grid, and its CPML: the grid's layer on
    each face the sub-box shares with the grid (the graded coefficients depend only on the distance
    to that face), none on the faces inside the grid (walls M cells from q, too far to matter)."""
    lo = [max(0, q[d] - M) for d in range(3)]
    hi = [min(sc.n[d], q[d] + M + 1) for d in range(3)]
    pml = []
    for d in range(3):
        pml += [sc.pml[2 * d] if lo[d] == 0 else 0, sc.pml[2 * d + 1] if hi[d] == sc.n[d] else 0]
    return lo, hi, tuple(pml)


def _light_cone_check(sc, probes, n_steps, r, label):
    """From a seeded random state on the PML-free region, n steps forward and the time-reversal
    gradient on the full grid (the launch configuration of that grid). probes[0] carries a point
    detector and the design box of radius r; every probe compares the fields of its block of radius
    r. In n steps a Yee update moves information at most one cell per step, so those values depend
    only on the state, the permittivity and the CPML within n + r cells of the probe: the FP64
    oracle's solve of that window from the same state gives them exactly."""
    import torch
    from paper_2412_12360_b300 import fdtd
    M = n_steps + r + 3
    nx, ny, nz = sc.n
    p = sc.pml
    q0 = probes[0]
    for d in range(3):  # the detector and the design box lie in the PML-free region
        assert p[2 * d] <= q0[d] - r and q0[d] + r < sc.n[d] - p[2 * d + 1]
    sc.sources = []
    sc.detectors = [S.Detector(S.DET_POINT_SERIES, q0, tuple(v + 1 for v in q0), component=S.EZ)]
    sc.design_lo = tuple(v - r for v in q0)
    sc.design_hi = tuple(v + r + 1 for v in q0)
    dev = torch.device("cuda")
    gen = torch.Generator(device=dev).manual_seed(77)
    init = torch.zeros((6, nz, ny, nx), dtype=torch.float32, device=dev)
    init[:, p[4]:nz - p[5], p[2]:ny - p[3], p[0]:nx - p[1]] = (
        2 * torch.rand((6, nz - p[4] - p[5], ny - p[2] - p[3], nx - p[0] - p[1]), generator=gen, device=dev) - 1)
    g = np.random.default_rng(78).standard_normal(n_steps)
    fields = torch.empty_like(init)
    with fdtd.Solver(sc) as s:
        s.fdtd_set_initial_fields(init)
        s.fdtd_forward(n_steps, record_faces=True)
        s.fdtd_get_fields(fields)
        det_g = s.detectors()
        grad_g = s.gradient(g)
    for qi, q in enumerate(probes):
        lo, hi, pm = _window(sc, q, M)
        sl = (slice(None),) + tuple(slice(lo[d], hi[d]) for d in (2, 1, 0))
        c = tuple(q[d] - lo[d] for d in range(3))
        nsub = tuple(hi[d] - lo[d] for d in range(3))
        extra = {}
        if qi == 0:
            extra = dict(detectors=[S.Detector(S.DET_POINT_SERIES, c, tuple(v + 1 for v in c), component=S.EZ)],
                         design=(tuple(v - r for v in c), tuple(v + r + 1 for v in c)))
        sub = H.box_scene(nsub, pml=pm, eps_inv=np.ascontiguousarray(sc.eps_inv[sl[1:]]), courant=sc.courant,
                          sigma_max=sc.sigma_max, nsteps=n_steps, **extra)
        sub_init = init[sl].double().cpu().numpy()
        f_o, _ = O.forward(sub, n_steps, init=sub_init)
        bl = [(max(0, c[d] - r), min(nsub[d], c[d] + r + 1)) for d in range(3)]
        blk = (slice(None),) + tuple(slice(*bl[d]) for d in (2, 1, 0))
        gblk = (slice(None),) + tuple(slice(bl[d][0] + lo[d], bl[d][1] + lo[d]) for d in (2, 1, 0))
        f_g = fields[gblk].double().cpu().numpy()
        e_f = float(np.max(np.abs(f_g - f_o[blk])) / np.max(np.abs(f_o[blk])))
        msg = "%s probe %s (window CPML %s): fields %.2e" % (label, q, pm, e_f)
        if qi == 0:
            grad_o, _, det_o = O.gradient(sub, n_steps, g, O.METHOD_STORE_ALL, init=sub_init)
            e_d = float(np.max(np.abs(det_g - det_o)) / np.max(np.abs(det_o)))
            e_g = rel(grad_g, grad_o)
            msg += ", probe series %.2e, dL/deps %.2e" % (e_d, e_g)
            assert e_d < 1e-5 and e_g < 1e-4, msg
        print(msg)
        assert e_f < 1e-5, msg


@pytest.mark.parametrize("config", ["waveguide_600", "waveguide_batch_member", "served_200", "served_128x128x256"])
def test_full_size_light_cone_parity(cuda_ok, config):
    """Element-wise parity on the full grids of the large configurations, in their launch
    configurations (same grid, so the same tiles, z-chunks and stage rings): probe points inside the
    PML-free region on tile and z-chunk boundaries and in the random-density design region."""
    n_steps, r = 12, 3
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
    _light_cone_check(sc, probes, n_steps, r, config)


@pytest.mark.parametrize("config", ["waveguide_600", "served_200"])
def test_full_size_light_cone_parity_in_the_cpml(cuda_ok, config):
    """The same at probes in the CPML layers (faces, an edge, a corner) and at a detector and design box
    next to a layer, so that the adjoint sweep runs through it: the windows reach the grid's faces and
    carry the layers of those faces."""
    n_steps, r = 12, 3
    if config == "waveguide_600":
        sc = S.waveguide_600(n_steps)
        probes = [(16, 300, 300), (6, 6, 6), (593, 300, 580), (300, 590, 300), (300, 300, 595)]
    else:
        sc = S.design_box_scene((200, 200, 200), 10, 100, n_steps, 10007)
        probes = [(186, 100, 13), (3, 100, 100), (197, 197, 5), (100, 192, 100), (50, 4, 196)]
    _light_cone_check(sc, probes, n_steps, r, config + "_cpml")
