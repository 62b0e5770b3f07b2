"""GPU (CUDA, fp32 fields, fp64 accumulators) against the FP64 oracle on the same seeded inputs.

Bars: fields after the run within 1e-4 relative L2; detector outputs within 1e-4 relative; dL/deps
within 1e-3 relative L2 over the design box (and the max error is reported). Grids span several
column tiles of both the forward (32 x 16) and the reverse (32 x 8) kernels with ragged tails, one
with an odd x extent (the forward kernel's last cell pair then has one cell in the grid); layers
differ per face.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_12360_b300 import scenes as S
from tests import _helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F(cuda_ok):
    from paper_2412_12360_b300 import fdtd
    fdtd.lib()
    return fdtd


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def ragged_scene(nsteps=600, seed=41):
    n = (70, 45, 38)
    pml = (6, 5, 7, 6, 5, 8)
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    eps_inv = np.ones((nz, ny, nx), dtype=np.float32)
    dlo, dhi = (20, 14, 12), (46, 33, 27)
    eps_inv[dlo[2]:dhi[2], dlo[1]:dhi[1], dlo[0]:dhi[0]] = S.inv(
        1.0 + 11.1 * rng.random((dhi[2] - dlo[2], dhi[1] - dlo[1], dhi[0] - dlo[0])))
    prof = S.gaussian_sheet((ny - 12, nx - 11), 12.0)[None]
    sheet = S.default_pulse(S.Source(S.EX, (6, 7, 10), (nx - 5, ny - 5, 11), prof, 1.0, 12.0), S.courant_from_factor())
    pt = H.point_source(S.EZ, (30, 10, 20), wavelength=10.0, amplitude=0.5)
    dets = [H.point_probe(S.HY, (50, 30, 25)),
            S.Detector(S.DET_PLANE_E2_SUM, (6, 7, 28), (64, 39, 29)),
            S.Detector(S.DET_PLANE_FLUX, (58, 7, 8), (59, 39, 30), axis=0),
            S.Detector(S.DET_PLANE_FLUX, (6, 7, 29), (64, 39, 30), axis=2)]
    return H.box_scene(n, pml=pml, eps_inv=eps_inv, sources=[sheet, pt], detectors=dets, design=(dlo, dhi),
                       nsteps=nsteps, name="ragged")


def odd_scene(nsteps=400, seed=43, pml=(5, 7, 4, 6, 6, 3)):
    """Odd nx, sources, detectors and the design box reaching the last x column, and a two-cell-thick
    x-normal flux box whose cells fall in two different cell pairs."""
    n = (67, 37, 29)
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    eps_inv = np.ones((nz, ny, nx), dtype=np.float32)
    dlo, dhi = (41, 9, 8), (67, 30, 22)
    eps_inv[dlo[2]:dhi[2], dlo[1]:dhi[1], dlo[0]:dhi[0]] = S.inv(
        1.0 + 11.1 * rng.random((dhi[2] - dlo[2], dhi[1] - dlo[1], dhi[0] - dlo[0])))
    prof = S.gaussian_sheet((ny - 10, nx - 5), 10.0)[None]
    sheet = S.default_pulse(S.Source(S.EY, (5, 5, 8), (nx, ny - 5, 9), prof, 1.0, 12.0), S.courant_from_factor())
    pt = H.point_source(S.EZ, (66, 20, 14), wavelength=9.0, amplitude=0.5)
    dets = [H.point_probe(S.EZ, (66, 18, 16)),
            S.Detector(S.DET_PLANE_E2_SUM, (50, 6, 20), (67, 31, 21)),
            S.Detector(S.DET_PLANE_FLUX, (41, 6, 6), (43, 31, 23), axis=0),
            S.Detector(S.DET_PLANE_FLUX, (5, 6, 23), (66, 31, 24), axis=2)]
    return H.box_scene(n, pml=pml, eps_inv=eps_inv, sources=[sheet, pt], detectors=dets, design=(dlo, dhi),
                       nsteps=nsteps, name="odd_x")


def wide_scene(nsteps=150, seed=47):
    """A grid whose adjoint-step tiles form a frame of x/y CPML tiles (first and last two columns, first
    and last two rows) around a rectangle of plain tiles, with ragged tails in x and y, unequal
    layers, and detectors and a design box in both parts."""
    n = (133, 99, 36)
    pml = (6, 5, 7, 4, 5, 6)
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    eps_inv = np.ones((nz, ny, nx), dtype=np.float32)
    dlo, dhi = (10, 12, 9), (120, 90, 28)
    eps_inv[dlo[2]:dhi[2], dlo[1]:dhi[1], dlo[0]:dhi[0]] = S.inv(
        1.0 + 11.1 * rng.random((dhi[2] - dlo[2], dhi[1] - dlo[1], dhi[0] - dlo[0])))
    prof = S.gaussian_sheet((ny - 11, nx - 11), 20.0)[None]
    sheet = S.default_pulse(S.Source(S.EX, (6, 7, 6), (nx - 5, ny - 4, 7), prof, 1.0, 14.0), S.courant_from_factor())
    pt = H.point_source(S.EZ, (70, 40, 18), wavelength=10.0, amplitude=0.5)
    dets = [H.point_probe(S.HY, (125, 50, 20)), H.point_probe(S.EY, (8, 92, 15)),
            S.Detector(S.DET_PLANE_E2_SUM, (6, 7, 25), (128, 95, 26)),
            S.Detector(S.DET_PLANE_FLUX, (126, 7, 8), (127, 95, 29), axis=0)]
    return H.box_scene(n, pml=pml, eps_inv=eps_inv, sources=[sheet, pt], detectors=dets, design=(dlo, dhi),
                       nsteps=nsteps, name="wide")


def test_split_adjoint_step_equals_one_launch(F, monkeypatch):
    """The fused adjoint step as two launches (the frame of tiles that need the x/y CPML loop, then the
    rectangle of plain tiles, each with its own z-chunks) gives bitwise the detectors, dL/deps and
    fields of one launch over all tiles, also with other z-chunks, and matches the oracle."""
    sc = wide_scene()
    g = np.random.default_rng(16).standard_normal(O.detector_total(sc, sc.nsteps))
    monkeypatch.setenv("FDTD_REV_FUSED", "1")
    out = {}
    for name, split, tz in (("one", "0", None), ("split", "1", None), ("split_tz5", "1", "5")):
        monkeypatch.setenv("FDTD_ADJ_SPLIT", split)
        if tz is None:
            monkeypatch.delenv("FDTD_TZ", raising=False)
        else:
            monkeypatch.setenv("FDTD_TZ", tz)
        with F.Solver(sc) as s:
            s.fdtd_forward(sc.nsteps, record_faces=True)
            det = s.detectors()
            l0 = s.fdtd_launch_count()
            grad = s.gradient(g)
            out[name] = (det, grad, s.fields(), s.fdtd_launch_count() - l0)
    assert out["split"][3] == out["one"][3] + sc.nsteps  # one more launch per reverse step
    for name in ("split", "split_tz5"):
        for a, b in zip(out[name][:3], out["one"][:3]):
            assert np.array_equal(a, b), name
    grad_o, _, det_o = O.gradient(sc, sc.nsteps, g, O.METHOD_TIME_REVERSAL)
    e, ed = rel_l2(out["split"][1], grad_o), rel_l2(out["split"][0], det_o)
    print("split adjoint step: dL/deps rel L2 %.3e, detectors %.3e" % (e, ed))
    assert e < 1e-3 and ed < 1e-4


def test_bounded_wait_ends_with_a_timeout_status_and_the_context_stays_usable(F):
    """The stencil kernels' bounded wait, run on an mbarrier that nothing completes, gives up after its
    limit and reports FDTD_ERR_TIMEOUT instead of hanging; the process then solves a scene to the
    oracle's result (no GPU fault is involved: the wait only polls its own shared-memory barrier)."""
    for limit_ms in (20, 200):
        rc, ns = F.wait_probe(limit_ms)
        print("wait probe, limit %d ms: code %d after %.1f ms" % (limit_ms, rc, ns / 1e6))
        assert rc == F.FDTD_ERR_TIMEOUT
        assert limit_ms * 1e6 <= ns < limit_ms * 1e6 + 50e6
    sc = S.cavity_32(200)
    f_o, d_o = O.forward(sc, 200)
    with F.Solver(sc) as s:
        s.fdtd_forward(200)
        assert rel_l2(s.detectors(), d_o) < 1e-4


def test_forward_pec_cavity_1000_steps(F):
    sc = S.cavity_32(1000)
    f_o, d_o = O.forward(sc, 1000)
    with F.Solver(sc) as s:
        s.fdtd_forward(1000)
        f_g = s.fields()
        d_g = s.detectors()
    e = rel_l2(f_g, f_o)
    print("cavity_32 1000 steps: fields rel L2 %.3e" % e)
    assert e < 1e-4
    assert rel_l2(d_g, d_o) < 1e-4


def test_forward_cpml_ragged_grid(F):
    sc = ragged_scene(600)
    f_o, d_o = O.forward(sc, 600)
    with F.Solver(sc) as s:
        s.fdtd_forward(600)
        f_g = s.fields()
        d_g = s.detectors()
    e = rel_l2(f_g, f_o)
    print("ragged 600 steps: fields rel L2 %.3e" % e)
    assert e < 1e-4
    off = 0
    for d in sc.detectors:
        m = 600 if d.kind != S.DET_PLANE_E2_SUM else int(np.prod([d.hi[k] - d.lo[k] for k in range(3)]))
        ed = rel_l2(d_g[off:off + m], d_o[off:off + m])
        print("  detector kind %d rel %.3e" % (d.kind, ed))
        assert ed < 1e-4
        off += m


def test_forward_and_gradient_odd_x_extent(F):
    sc = odd_scene(400)
    f_o, d_o = O.forward(sc, 400)
    with F.Solver(sc) as s:
        s.fdtd_forward(400)
        f_g = s.fields()
        d_g = s.detectors()
        per = [s.detector(q) for q in range(len(sc.detectors))]  # one detector at a time
        with pytest.raises(F.FDTDError):
            s.fdtd_detector_size(len(sc.detectors))
    assert np.array_equal(np.concatenate(per), d_g)
    e = rel_l2(f_g, f_o)
    print("odd_x 400 steps: fields rel L2 %.3e" % e)
    assert e < 1e-4
    off = 0
    for d in sc.detectors:
        m = 400 if d.kind != S.DET_PLANE_E2_SUM else int(np.prod([d.hi[k] - d.lo[k] for k in range(3)]))
        ed = rel_l2(d_g[off:off + m], d_o[off:off + m])
        print("  detector kind %d rel %.3e" % (d.kind, ed))
        assert ed < 1e-4
        off += m
    # the gradient needs its detectors off the layers: no layer on the high x face (a PEC wall there)
    sc = odd_scene(300, pml=(5, 0, 4, 6, 6, 3))
    g = np.random.default_rng(9).standard_normal(O.detector_total(sc, 300))
    grad_o, _, _ = O.gradient(sc, 300, g, O.METHOD_TIME_REVERSAL)
    with F.Solver(sc) as s:
        s.fdtd_forward(300, record_faces=True)
        grad_g = s.gradient(g)
    e = rel_l2(grad_g, grad_o)
    print("odd_x 300 steps: dL/deps rel L2 %.3e" % e)
    assert e < 1e-3


def test_forward_from_initial_state_and_zero_steps(F):
    sc = S.cavity_32(200)
    init = S.random_fields(sc, 3)
    with F.Solver(sc) as s:
        s.fdtd_set_initial_fields(init)
        s.fdtd_forward(0)
        assert np.array_equal(s.fields(), init)
        s.fdtd_forward(200)
        f_g = s.fields()
    f_o, _ = O.forward(sc, 200, init.astype(np.float64))
    assert rel_l2(f_g, f_o) < 1e-4


def test_time_reversal_roundtrip_drift(F):
    """Forward then the inverse update step (inside backward) returns the initial state on R."""
    for sc in (S.cavity_32(500), ragged_scene(500)):
        init = S.random_fields(sc, 5)
        with F.Solver(sc) as s:
            s.fdtd_set_initial_fields(init)
            s.fdtd_forward(500, record_faces=True)
            fwd = s.fields()
            s.gradient(np.zeros(s.fdtd_detector_total()))
            back = s.fields()
        m = H.r_masks(sc)
        drift = rel_l2(back[m], init[m])
        print("%s: fp32 round-trip drift after 500+500 steps: rel L2 %.3e, max %.3e" % (
            sc.name, drift, np.max(np.abs(back[m] - init[m]))))
        assert rel_l2(fwd[m], init[m]) > 0.1
        assert drift < 1e-4


def test_gradient_matches_oracle_ragged(F):
    sc = ragged_scene(400)
    rng = np.random.default_rng(7)
    g = rng.standard_normal(O.detector_total(sc, 400))
    grad_o, _, det_o = O.gradient(sc, 400, g, O.METHOD_TIME_REVERSAL)
    with F.Solver(sc) as s:
        s.fdtd_forward(400, record_faces=True)
        det_g = s.detectors()
        grad_g = s.gradient(g)
    e = rel_l2(grad_g, grad_o)
    print("ragged 400 steps: dL/deps rel L2 %.3e, max abs err / max %.3e" % (
        e, np.max(np.abs(grad_g - grad_o)) / np.max(np.abs(grad_o))))
    assert rel_l2(det_g, det_o) < 1e-4
    assert e < 1e-3


def folded_scene(all_folded, nsteps=300, seed=45):
    """Detectors whose adjoints the reverse H kernel adds (points on E components, |E|^2 planes, two of
    them overlapping), alone or with more of them than it takes and with H-point and flux detectors
    that keep launches of their own."""
    sc = ragged_scene(nsteps, seed)
    dets = [H.point_probe(S.EX, (40, 20, 24)),
            S.Detector(S.DET_PLANE_E2_SUM, (8, 9, 26), (60, 36, 27)),
            S.Detector(S.DET_PLANE_E2_SUM, (30, 20, 25), (50, 30, 28)),
            H.point_probe(S.EY, (12, 33, 29))]
    if not all_folded:
        dets += [S.Detector(S.DET_PLANE_E2_SUM, (10, 8, 27), (30, 20, 29)),
                 H.point_probe(S.HZ, (44, 12, 26)),
                 S.Detector(S.DET_PLANE_FLUX, (58, 7, 8), (59, 39, 30), axis=0)]
    sc.detectors = dets
    return sc


@pytest.mark.parametrize("all_folded", [True, False])
def test_gradient_folded_detector_adjoints(F, all_folded):
    sc = folded_scene(all_folded)
    rng = np.random.default_rng(10)
    g = rng.standard_normal(O.detector_total(sc, sc.nsteps))
    grad_o, _, _ = O.gradient(sc, sc.nsteps, g, O.METHOD_TIME_REVERSAL)
    with F.Solver(sc) as s:
        s.fdtd_forward(sc.nsteps, record_faces=True)
        grad_g = s.gradient(g)
        # the checkpointed gradient adds every detector adjoint by its own launch
        out = np.zeros(sc.design_shape(), dtype=np.float32)
        s.fdtd_backward_checkpointed(g, out, 0)
    e, e_c = rel_l2(grad_g, grad_o), rel_l2(grad_g, out)
    print("folded detector adjoints (all folded: %s): dL/deps rel L2 %.3e vs oracle, %.3e vs checkpointed"
          % (all_folded, e, e_c))
    assert e < 1e-3
    assert e_c < 1e-4


@pytest.mark.parametrize("nstage", ["3", "4"])
@pytest.mark.parametrize("scene", ["ragged", "odd_x"])
def test_gradient_three_and_four_stage_reverse_kernels(F, scene, nstage, monkeypatch):
    """Both ring sizes of the reverse kernels (the fused inverse and adjoint steps of time reversal,
    and the reverse kernels of the checkpointing gradient) on small scenes: each size is what some grid
    runs by default."""
    monkeypatch.setenv("FDTD_REV_NSTAGE", nstage)
    sc = ragged_scene(300) if scene == "ragged" else odd_scene(300, pml=(5, 0, 4, 6, 6, 3))
    g = np.random.default_rng(11).standard_normal(O.detector_total(sc, 300))
    grad_o, _, _ = O.gradient(sc, 300, g, O.METHOD_TIME_REVERSAL)
    with F.Solver(sc) as s:
        s.fdtd_forward(300, record_faces=True)
        grad_g = s.gradient(g)
        grad_c = np.zeros(sc.design_shape(), dtype=np.float32)
        s.fdtd_forward(300)
        s.fdtd_backward_checkpointed(g, grad_c, 1, 6)
    e, e_c = rel_l2(grad_g, grad_o), rel_l2(grad_c, grad_o)
    print("%s 300 steps, %s-stage reverse: dL/deps rel L2 %.3e (time reversal), %.3e (checkpointing)"
          % (scene, nstage, e, e_c))
    assert e < 1e-3 and e_c < 1e-3


@pytest.mark.parametrize("kind", ["0", "1"])
@pytest.mark.parametrize("scene", ["ragged", "odd_x", "tfsf_interp"])
def test_gradient_with_each_reverse_kind(F, scene, kind, monkeypatch):
    """Both reverse-step kinds (the in-place pair rev_E + rev_H, and the fused inverse + adjoint
    kernels that large grids use) against the oracle, on scenes with unequal layers, an odd x extent,
    a TFSF plane and interpolated detectors."""
    monkeypatch.setenv("FDTD_REV_FUSED", kind)
    sc = ragged_scene(250) if scene == "ragged" else (odd_scene(250, pml=(5, 0, 4, 6, 6, 3)) if scene == "odd_x"
                                                       else S.design_box_scene((45, 38, 41), 6, 12, 250, 21,
                                                                               name="kinds", tfsf=True, interp=True))
    g = np.random.default_rng(15).standard_normal(O.detector_total(sc, sc.nsteps))
    grad_o, _, det_o = O.gradient(sc, sc.nsteps, g, O.METHOD_TIME_REVERSAL)
    with F.Solver(sc) as s:
        s.fdtd_forward(sc.nsteps, record_faces=True)
        det = s.detectors()
        grad = s.gradient(g)
    e, ed = rel_l2(grad, grad_o), rel_l2(det, det_o)
    print("%s, reverse kind %s: dL/deps rel L2 %.3e, detectors %.3e" % (scene, kind, e, ed))
    assert e < 1e-3 and ed < 1e-4


@pytest.mark.parametrize("kind", ["0", "1"])
@pytest.mark.parametrize("scene", ["ragged", "tfsf_interp"])
def test_results_do_not_depend_on_the_z_chunk(F, scene, kind, monkeypatch):
    """The z-marching kernels recompute the plane next to their chunk with the same arithmetic as the
    block that owns it, so the z-planes per block leave fields, detectors and gradients bitwise the same
    (flux detectors, whose per-block partial sums follow the chunks, to FP64 rounding)."""
    sc = ragged_scene(120) if scene == "ragged" else S.design_box_scene(
        (45, 38, 41), 6, 12, 120, 21, name="tz", tfsf=True, interp=True)
    g = np.random.default_rng(14).standard_normal(O.detector_total(sc, sc.nsteps))
    out = []
    monkeypatch.setenv("FDTD_REV_FUSED", kind)
    for tz in (None, "3", "7"):
        if tz is None:
            monkeypatch.delenv("FDTD_TZ", raising=False)
        else:
            monkeypatch.setenv("FDTD_TZ", tz)
        with F.Solver(sc) as s:
            s.fdtd_forward(sc.nsteps, record_faces=True)
            det = s.detectors()
            f_fwd = s.fields()
            out.append((det, f_fwd, s.gradient(g), s.fields()))
    flux = np.zeros(out[0][0].shape, dtype=bool)
    off = 0
    for d in sc.detectors:
        n = int(np.prod([d.hi[k] - d.lo[k] for k in range(3)])) if d.kind in (1, 3) else sc.nsteps
        if d.kind in (2, 4):
            flux[off:off + n] = True
        off += n
    for o in out[1:]:
        assert np.array_equal(o[0][~flux], out[0][0][~flux])
        assert np.allclose(o[0][flux], out[0][0][flux], rtol=1e-12, atol=1e-12 * np.abs(out[0][0]).max())
        for a, b in zip(o[1:], out[0][1:]):
            assert np.array_equal(a, b)


def test_gradient_pec_point_detectors(F):
    sc = S.cavity_32(300)
    rng = np.random.default_rng(8)
    g = rng.standard_normal(O.detector_total(sc, 300))
    grad_o, _, _ = O.gradient(sc, 300, g, O.METHOD_TIME_REVERSAL)
    with F.Solver(sc) as s:
        s.fdtd_forward(300, record_faces=True)
        grad_g = s.gradient(g)
    e = rel_l2(grad_g, grad_o)
    print("cavity_32 300 steps: dL/deps rel L2 %.3e" % e)
    assert e < 1e-3


def test_device_and_host_buffers_agree_and_runs_are_deterministic(F):
    import torch
    sc = ragged_scene(150)
    g = np.random.default_rng(9).standard_normal(O.detector_total(sc, 150))
    outs = []
    for _ in range(2):
        with F.Solver(sc, eps_inv=torch.from_numpy(sc.eps_inv).cuda()) as s:
            s.fdtd_forward(150, record_faces=True)
            det_d = torch.zeros(s.fdtd_detector_total(), dtype=torch.float64, device="cuda")
            s.fdtd_read_detectors(det_d)
            gd = torch.from_numpy(g).cuda()
            out_d = torch.zeros(sc.design_shape(), dtype=torch.float32, device="cuda")
            s.fdtd_backward(gd, out_d)
            torch.cuda.synchronize()
            outs.append((det_d.cpu().numpy(), out_d.cpu().numpy()))
    with F.Solver(sc) as s:
        s.fdtd_forward(150, record_faces=True)
        det_h = s.detectors()
        out_h = s.gradient(g)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][0], det_h) and np.array_equal(outs[0][1], out_h)


def test_nonfinite_fields_are_reported_and_the_handle_recovers(F):
    """A NaN in the initial state (an input, not a device fault) spreads through the solve; the field
    checks flag it, fdtd_synchronize and the host-buffer reads report NONFINITE, and the same handle
    then solves a clean problem to the oracle's result. The periodic check changes no result."""
    sc = ragged_scene(120)
    nx, ny, nz = sc.n
    init = np.zeros((6, nz, ny, nx), dtype=np.float32)
    init[2, 20, 22, 35] = np.nan
    f_o, d_o = O.forward(sc, 120)
    with F.Solver(sc) as s:
        s.fdtd_set_initial_fields(init)
        s.fdtd_forward(120, record_faces=True)
        with pytest.raises(F.FDTDError) as e:
            s.fdtd_synchronize()
        assert "NONFINITE" in str(e.value)
        s.fdtd_synchronize()  # reported once, then cleared
        s.fdtd_forward(120, record_faces=True)
        with pytest.raises(F.FDTDError) as e:
            s.detectors()  # a host-buffer read reports it too
        assert "NONFINITE" in str(e.value)
        # a NaN in dL/d(outputs) poisons the adjoint fields: the backward reports it
        s.fdtd_set_initial_fields(None)
        s.fdtd_forward(120, record_faces=True)
        s.fdtd_synchronize()
        g = np.ones(O.detector_total(sc, 120))
        g[5] = np.nan
        with pytest.raises(F.FDTDError) as e:
            s.gradient(g)
        assert "NONFINITE" in str(e.value)
        # clean again, with a check every 7 steps: results equal the oracle's and the unchecked run's
        s.fdtd_forward(120)
        plain = s.fields()
        s.fdtd_set_check_interval(7)
        s.fdtd_forward(120)
        checked = s.fields()
        s.fdtd_synchronize()
    assert np.array_equal(plain, checked)
    assert rel_l2(checked, f_o) < 1e-4


@pytest.mark.parametrize("scene", ["ragged", "odd_x", "tfsf_interp"])
def test_pitch_padding_canaries_stay_intact(F, scene):
    """NaN canaries in the pitch padding of every field, adjoint and permittivity row: a forward with the
    face record, the time-reversal and the checkpointing gradients leave every canary in place, read
    none (no NaN reaches a result) and give bitwise the results of the same runs without canaries."""
    if scene == "ragged":
        sc = ragged_scene(150)
    elif scene == "odd_x":
        sc = odd_scene(150, pml=(5, 0, 4, 6, 6, 3))
    else:
        sc = S.design_box_scene((45, 38, 41), 6, 12, 150, 21, name="canary", tfsf=True, interp=True)
    assert sc.n[0] % 32 != 0  # a grid with pitch padding
    g = np.random.default_rng(12).standard_normal(O.detector_total(sc, sc.nsteps))
    out = []
    for canary in (False, True):
        with F.Solver(sc) as s:
            if canary:
                s.fdtd_set_canaries(True)
            s.fdtd_forward(sc.nsteps, record_faces=True)
            det = s.detectors()
            grad = s.gradient(g)
            ck = np.zeros(sc.design_shape(), dtype=np.float32)
            s.fdtd_backward_checkpointed(g, ck, 1, 3)
            fields = s.fields()
            if canary:
                assert s.fdtd_check_canaries() == 0
            s.fdtd_synchronize()
        out.append((det, grad, ck, fields))
    for a, b in zip(*out):
        assert np.all(np.isfinite(b))
        assert np.array_equal(a, b)


@pytest.mark.parametrize("kind", ["0", "1"])
@pytest.mark.parametrize("scene", ["ragged", "tfsf_interp"])
def test_face_copies_and_graphs_on_or_off_give_the_same_results(F, scene, kind, monkeypatch):
    """Face copies overlapped or in line, time loops captured into graphs or launched directly (with
    the per-launch profiling events on): bitwise the same detectors, gradients and fields, with either
    reverse-step kind."""
    monkeypatch.setenv("FDTD_REV_FUSED", kind)
    sc = ragged_scene(150) if scene == "ragged" else S.design_box_scene(
        (45, 38, 41), 6, 12, 150, 21, name="ovl", tfsf=True, interp=True)
    g = np.random.default_rng(13).standard_normal(O.detector_total(sc, sc.nsteps))
    out = []
    for ovl, graphs in ((True, True), (False, True), (True, False), (False, False)):
        with F.Solver(sc) as s:
            s.fdtd_set_face_overlap(ovl)
            s.fdtd_set_graphs(graphs)
            s.fdtd_profile(True, 16)
            for _ in range(2):  # the second solve replays (or relaunches) the loops
                s.fdtd_forward(sc.nsteps, record_faces=True)
                r = (s.detectors(), s.gradient(g), s.fields())
            prof = s.fdtd_profile_read()
        rev = ("inv_fused", "adj_fused") if kind == "1" else ("rev_E", "rev_H")
        assert prof["fused_fwd"][1] > 0 and prof[rev[0]][1] > 0 and prof[rev[1]][1] > 0
        out.append(r)
    for o in out[1:]:
        for a, b in zip(out[0], o):
            assert np.array_equal(a, b)


def test_degenerate_solves(F):
    """No sources (everything stays zero), no detectors (nothing to differentiate), an empty design box
    (backward writes nothing), and the shortest solves (1 and 2 steps: the first reverse step's
    detector adjoint by its own launch, the later ones folded into the reverse H kernel) against the
    oracle."""
    quiet = ragged_scene(50)
    quiet.sources = []
    with F.Solver(quiet) as s:
        s.fdtd_forward(50, record_faces=True)
        assert not np.any(s.fields()) and not np.any(s.detectors())
        g = np.ones(O.detector_total(quiet, 50))
        assert not np.any(s.gradient(g))
    blind = ragged_scene(50)
    blind.detectors = []
    with F.Solver(blind) as s:
        s.fdtd_forward(50, record_faces=True)
        assert s.fdtd_detector_total() == 0
        assert not np.any(s.gradient(np.zeros(0)))
    nodesign = ragged_scene(50)
    nodesign.design_lo = nodesign.design_hi = (30, 20, 20)
    with F.Solver(nodesign) as s:
        s.fdtd_forward(50, record_faces=True)
        out = s.gradient(np.ones(O.detector_total(nodesign, 50)))
        assert out.size == 0
    for nsteps in (1, 2, 3):
        sc = ragged_scene(nsteps)
        # a source in the design box that is already on at the first steps, probes beside it
        sc.sources = [H.point_source(S.EZ, (30, 20, 20), wavelength=4.0)]
        sc.sources[0].t0_steps = 1.5
        sc.detectors = [H.point_probe(S.EZ, (30, 20, 20)), H.point_probe(S.EX, (30, 20, 21)),
                        S.Detector(S.DET_PLANE_E2_SUM, (26, 16, 20), (35, 25, 21)),
                        S.Detector(S.DET_PLANE_FLUX, (26, 16, 21), (35, 25, 22), axis=2)]
        g = np.random.default_rng(14).standard_normal(O.detector_total(sc, nsteps))
        grad_o, _, det_o = O.gradient(sc, nsteps, g, O.METHOD_TIME_REVERSAL)
        with F.Solver(sc) as s:
            s.fdtd_forward(nsteps, record_faces=True)
            det_g = s.detectors()
            grad_g = s.gradient(g)
        assert np.max(np.abs(det_o)) > 0, nsteps
        assert rel_l2(det_g, det_o) < 1e-5, nsteps
        if nsteps == 1:  # E^1 is the source alone (H^{1/2} = 0): nothing depends on eps yet
            assert not np.any(grad_o) and not np.any(grad_g)
        else:
            assert np.max(np.abs(grad_o)) > 0 and rel_l2(grad_g, grad_o) < 1e-5, nsteps


def test_state_errors_and_byte_budget(F):
    sc = S.cavity_32(20)
    with F.Solver(sc) as s:
        s.fdtd_forward(20)
        with pytest.raises(F.FDTDError) as ei:
            s.gradient(np.zeros(s.fdtd_detector_total()))
        assert ei.value.code == F.FDTD_ERR_STATE
        s.fdtd_forward(20, record_faces=True)
        s.gradient(np.zeros(s.fdtd_detector_total()))
        with pytest.raises(F.FDTDError) as ei:
            s.gradient(np.zeros(s.fdtd_detector_total()))
        assert ei.value.code == F.FDTD_ERR_STATE
    F.set_byte_budget(1 << 20)
    try:
        with pytest.raises(F.FDTDError) as ei:
            F.Solver(sc)
        assert ei.value.code == F.FDTD_ERR_OOM
    finally:
        F.set_byte_budget(-1)


def test_backward_rejects_detectors_in_the_pml(F):
    sc = ragged_scene(10)
    sc.detectors = [S.Detector(S.DET_PLANE_E2_SUM, (1, 7, 28), (64, 40, 29))]
    with F.Solver(sc) as s:
        s.fdtd_forward(10)  # plain forward is fine
        with pytest.raises(F.FDTDError) as ei:
            s.fdtd_forward(10, record_faces=True)
        assert ei.value.code == F.FDTD_ERR_INVALID_ARG
