"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: closed-form discrete dispersion of
a PEC cavity, convergence to the continuum cavity frequency, exact invariants of the Yee leapfrog
(energy, Gauss law), exact inverse stepping (Sec. 2.2), independent derivatives (complex step and
finite differences), reciprocity, the paper's printed step and cell counts (Table 2, Sec. 3.1-3.3),
and CPML reflection (Sec. 2.1).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_12360_b300 import scenes as S
from tests import _helpers as H


# ------------------------------------------------------------------------------------------------
# Table 2 (Sec. 3.1) and the step/cell counts of Sec. 3.2-3.3
# ------------------------------------------------------------------------------------------------

def _golden_table2():
    rows = []
    with open(__file__.replace("test_oracle_pins.py", "golden/table2_steps_cells.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_table2_step_and_cell_counts():
    rows = _golden_table2()
    assert len(rows) == 7
    for sx, sy, sz, dx_nm, t_fs, steps, cells in rows:
        n = S.grid_for((float(sx) * 1e-6, float(sy) * 1e-6, float(sz) * 1e-6), float(dx_nm) * 1e-9)
        assert S.steps_for(float(t_fs) * 1e-15, float(dx_nm) * 1e-9) == int(steps)
        got = n[0] * n[1] * n[2]
        # the paper prints cell counts to 2-3 significant digits
        assert abs(got - float(cells)) / float(cells) < 0.01, (n, cells)


# ------------------------------------------------------------------------------------------------
# Yee update, PEC and Courant number: exact discrete cavity eigenmodes
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,m,a", [((10, 9, 8), (1, 1, 1), 1.0),
                                   ((12, 7, 9), (2, 1, 3), 1.0),
                                   ((9, 11, 10), (3, 2, 0), 1.0 / 2.25),
                                   ((8, 8, 12), (0, 1, 4), 0.5)])
def test_eigenmode_frequency(n, m, a):
    nx, ny, nz = n
    eps_inv = np.full((nz, ny, nx), a, dtype=np.float32)
    cells = [(2, 3, 3), (3, 1, 2), (1, 2, 5), (5, 5, 1), (1, 5, 7)]
    probes = [H.point_probe(c, cell) for cell in cells for c in range(3)]
    sc = H.box_scene(n, eps_inv=eps_inv, detectors=probes)
    init = H.mode_fields(n, m)
    nsteps = 300
    _, det = O.forward(sc, nsteps, init)
    theta = H.discrete_theta(n, m, sc.courant, float(np.float32(a)))  # the float32 value the scene holds
    series = [det[q * nsteps:(q + 1) * nsteps] for q in range(len(probes))]
    used = 0
    for e in series:
        if np.max(np.abs(e)) < 1e-2:
            continue
        used += 1
        c = H.fit_cos_theta(e)
        assert abs(math.acos(c) - theta) < 1e-10, (math.acos(c), theta)
    assert used >= 3
    # the probe series are also pure sinusoids: residual of the recurrence at rounding level
    e = max(series, key=lambda v: np.max(np.abs(v)))
    c = math.cos(theta)
    assert np.max(np.abs(e[2:] + e[:-2] - 2 * c * e[1:-1])) < 1e-12 * np.max(np.abs(e))


def test_broadband_spectrum_peaks_sit_on_the_discrete_modes():
    """A short pulse rings every cavity mode it couples to: after it ends, the FFT peaks of two probe
    series in a PEC box sit within one bin of the Yee dispersion relation's mode frequencies
    theta_mnp (all (m, n, p) with at least two nonzero indices, oblique ones included). A 1 % error
    in the Courant number or in the curl weights would move the peaks by ~20 bins."""
    n = (10, 8, 6)
    nx, ny, nz = n
    src = H.point_source(S.EZ, (3, 2, 2), wavelength=3.0)
    src.tau_steps, src.t0_steps = 2.5, 8.0
    sc = H.box_scene(n, sources=[src], detectors=[H.point_probe(S.EZ, (6, 5, 3)), H.point_probe(S.EX, (4, 6, 4))])
    N, skip = 8192, 512
    _, det = O.forward(sc, N)
    thetas = np.array(sorted({H.discrete_theta(n, (a, b, c), sc.courant, 1.0)
                              for a in range(nx) for b in range(ny) for c in range(nz)
                              if (a > 0) + (b > 0) + (c > 0) >= 2}))
    matched = set()
    for k in range(2):
        e = det[k * N + skip:(k + 1) * N]
        F = np.abs(np.fft.rfft(e * np.hanning(e.size)))
        binw = 2 * math.pi / e.size
        peaks = [i for i in range(1, F.size - 1) if F[i] > F[i - 1] and F[i] >= F[i + 1] and F[i] > 1e-3 * F.max()]
        assert len(peaks) > 100
        for i in peaks:
            d = np.abs(thetas - i * binw)
            assert d.min() < binw, (i, d.min() / binw)
            matched.add(int(d.argmin()))
    assert len(matched) > 100


def test_eigenmode_converges_to_continuum_cavity():
    """f_mnp = (c/2) sqrt((m/a)^2 + (n/b)^2 + (p/d)^2): the discrete frequency approaches it at O(dx^2)."""
    base = (6, 5, 7)
    m = (1, 1, 1)
    errs = []
    for r in (1, 2, 4):
        n = tuple(b * r for b in base)
        probes = [H.point_probe(2, (n[0] // 3, n[1] // 3, n[2] // 3))]
        sc = H.box_scene(n, detectors=probes)
        nsteps = 120 * r
        _, det = O.forward(sc, nsteps, H.mode_fields(n, m))
        theta = math.acos(H.fit_cos_theta(det))
        omega_dx = theta / sc.courant                     # omega * dx / c
        cont = math.pi * math.sqrt(sum((m[d] / n[d]) ** 2 for d in range(3)))
        errs.append(abs(omega_dx - cont) / cont)
    assert errs[0] > errs[1] > errs[2]
    for r in (errs[0] / errs[1], errs[1] / errs[2]):
        assert 3.6 < r < 4.4, errs


# ------------------------------------------------------------------------------------------------
# Exact invariants: discrete energy and Gauss law in a lossless PEC box
# ------------------------------------------------------------------------------------------------

def _random_state(n, seed):
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((6, nz, ny, nx))
    f[0, 0, :, :] = 0; f[0, :, 0, :] = 0
    f[1, 0, :, :] = 0; f[1, :, :, 0] = 0
    f[2, :, 0, :] = 0; f[2, :, :, 0] = 0
    return f


def test_discrete_energy_is_invariant():
    n = (9, 8, 7)
    nx, ny, nz = n
    rng = np.random.default_rng(5)
    eps_inv = rng.uniform(0.3, 1.0, (nz, ny, nx)).astype(np.float32)
    sc = H.box_scene(n, eps_inv=eps_inv)
    init = _random_state(n, 6)
    eps = 1.0 / eps_inv.astype(np.float64)

    def energy(nstep):
        f0, _ = O.forward(sc, nstep, init)
        f1, _ = O.forward(sc, nstep + 1, init)
        return np.sum(eps * (f0[0] ** 2 + f0[1] ** 2 + f0[2] ** 2)) + np.sum(f0[3:] * f1[3:])

    w0 = energy(0)
    for nstep in (1, 37, 1000, 10000):
        assert abs(energy(nstep) - w0) / abs(w0) < 1e-12


def test_gauss_law_is_invariant():
    n = (10, 9, 8)
    nx, ny, nz = n
    rng = np.random.default_rng(8)
    eps_inv = rng.uniform(0.2, 1.0, (nz, ny, nx)).astype(np.float32)
    sc = H.box_scene(n, eps_inv=eps_inv)
    init = _random_state(n, 9)

    def div_d(f):
        d = f[:3] / eps_inv.astype(np.float64)[None]
        # node (i, j, k), i, j, k >= 1: sum_c D_c[p] - D_c[p - e_c]
        return ((d[0][1:, 1:, 1:] - d[0][1:, 1:, :-1]) + (d[1][1:, 1:, 1:] - d[1][1:, :-1, 1:]) +
                (d[2][1:, 1:, 1:] - d[2][:-1, 1:, 1:]))

    f, _ = O.forward(sc, 200, init)
    g0 = div_d(init)
    g1 = div_d(f)
    assert np.max(np.abs(g1 - g0)) < 1e-12 * np.max(np.abs(g0))
    # and the field did change
    assert np.max(np.abs(f[:3] - init[:3])) > 0.1


# ------------------------------------------------------------------------------------------------
# Inverse step (Sec. 2.2): forward then inverse returns the initial state
# ------------------------------------------------------------------------------------------------

def test_roundtrip_pec_cavity():
    sc = S.cavity_32(200)
    init = S.random_fields(sc, 11).astype(np.float64)
    fwd, back = O.roundtrip(sc, 200, init)
    assert np.max(np.abs(fwd - init)) > 0.5
    assert np.max(np.abs(back - init)) < 1e-12 * np.max(np.abs(init))


def test_roundtrip_cpml_region_with_face_replay():
    n = (20, 18, 22)
    pml = (4, 3, 5, 4, 3, 4)
    nx, ny, nz = n
    rng = np.random.default_rng(12)
    eps_inv = rng.uniform(0.25, 1.0, (nz, ny, nx)).astype(np.float32)
    src = H.point_source(1, (9, 8, 10), wavelength=8.0)
    sc = H.box_scene(n, pml=pml, eps_inv=eps_inv, sources=[src])
    init = S.random_fields(sc, 13).astype(np.float64)
    fwd, back = O.roundtrip(sc, 300, init)
    m = H.r_masks(sc)
    assert np.max(np.abs(fwd[m] - init[m])) > 0.5
    assert np.max(np.abs(back[m] - init[m])) < 1e-12 * np.max(np.abs(init))
    # the face set is 2 tangential H per face cell; its size matches the six planes
    ri = [min(n[d] - pml[2 * d + 1], n[d] - 1) - pml[2 * d] + 1 for d in range(3)]
    expect = sum(2 * 2 * ri[(d + 1) % 3] * ri[(d + 2) % 3] for d in range(3))
    assert O.face_count(sc) == expect


# ------------------------------------------------------------------------------------------------
# Reverse-mode gradient: complex step, finite differences, and three storage strategies agree
# ------------------------------------------------------------------------------------------------

def _grad_scene_pec():
    n = (12, 12, 12)
    nx, ny, nz = n
    rng = np.random.default_rng(21)
    eps_inv = rng.uniform(0.3, 1.0, (nz, ny, nx)).astype(np.float32)
    src = H.point_source(2, (4, 5, 6), wavelength=8.0)
    dets = [H.point_probe(0, (8, 7, 6)), H.point_probe(4, (7, 8, 8)),
            S.Detector(S.DET_PLANE_E2_SUM, (2, 2, 9), (10, 10, 10)),
            S.Detector(S.DET_PLANE_FLUX, (2, 3, 2), (9, 4, 10), axis=1)]
    return H.box_scene(n, eps_inv=eps_inv, sources=[src], detectors=dets, design=((3, 3, 3), (9, 9, 9)))


def _grad_scene_cpml():
    n = (16, 16, 16)
    nx, ny, nz = n
    rng = np.random.default_rng(22)
    eps_inv = np.ones((nz, ny, nx), dtype=np.float32)
    eps_inv[5:11, 5:11, 5:11] = rng.uniform(0.2, 1.0, (6, 6, 6)).astype(np.float32)
    src = H.point_source(0, (6, 7, 4), wavelength=8.0)
    dets = [H.point_probe(1, (9, 9, 11)),
            S.Detector(S.DET_PLANE_E2_SUM, (4, 4, 11), (12, 12, 12)),
            S.Detector(S.DET_PLANE_FLUX, (4, 4, 10), (12, 12, 11), axis=2)]
    return H.box_scene(n, pml=(4,) * 6, eps_inv=eps_inv, sources=[src], detectors=dets,
                       design=((5, 5, 5), (11, 11, 11)))


def _gvec(sc, nsteps, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(O.detector_total(sc, nsteps))


def test_store_all_gradient_matches_complex_step_pec():
    sc = _grad_scene_pec()
    nsteps = 80
    g = _gvec(sc, nsteps, 1)
    _, dLda, _ = O.gradient(sc, nsteps, g, O.METHOD_STORE_ALL, full=True)
    vox = [(5, 5, 5), (3, 8, 4), (10, 2, 7), (6, 6, 9)]
    cs = O.complex_step(sc, nsteps, g, vox)
    a = sc.eps_inv.astype(np.float64)
    adj = np.array([-a[k, j, i] ** 2 * dLda[k, j, i] for (i, j, k) in vox])
    scale = np.max(np.abs(adj))
    assert scale > 0
    assert np.max(np.abs(adj - cs)) < 1e-12 * scale, (adj, cs)


def test_time_reversal_gradient_matches_complex_step_cpml():
    sc = _grad_scene_cpml()
    nsteps = 120
    g = _gvec(sc, nsteps, 2)
    grad, _, _ = O.gradient(sc, nsteps, g, O.METHOD_TIME_REVERSAL)
    vox = [(5, 5, 5), (8, 7, 6), (10, 10, 10), (6, 9, 8)]
    cs = O.complex_step(sc, nsteps, g, vox)
    lo = sc.design_lo
    tr = np.array([grad[k - lo[2], j - lo[1], i - lo[0]] for (i, j, k) in vox])
    scale = np.max(np.abs(grad))
    assert np.max(np.abs(tr - cs)) < 1e-11 * scale, (tr, cs)


def test_three_gradient_strategies_agree():
    for sc, nsteps in ((_grad_scene_pec(), 70), (_grad_scene_cpml(), 90)):
        g = _gvec(sc, nsteps, 3)
        g_all, _, det0 = O.gradient(sc, nsteps, g, O.METHOD_STORE_ALL)
        g_ck, _, det1 = O.gradient(sc, nsteps, g, O.METHOD_CHECKPOINT, interval=16)
        g_tr, _, det2 = O.gradient(sc, nsteps, g, O.METHOD_TIME_REVERSAL)
        scale = np.max(np.abs(g_all))
        assert scale > 0
        assert np.max(np.abs(g_ck - g_all)) < 1e-13 * scale
        assert np.max(np.abs(g_tr - g_all)) < 1e-12 * scale
        assert np.array_equal(det0, det1) and np.array_equal(det0, det2)


def test_gradient_matches_central_finite_difference():
    sc = _grad_scene_cpml()
    nsteps = 90
    g = _gvec(sc, nsteps, 4)
    grad, _, _ = O.gradient(sc, nsteps, g, O.METHOD_TIME_REVERSAL)
    base = sc.eps_inv.astype(np.float64)
    h = 1e-6
    lo = sc.design_lo
    scale = np.max(np.abs(grad))
    for (i, j, k) in [(7, 7, 7), (5, 10, 9)]:
        eps0 = 1.0 / base[k, j, i]
        vals = []
        for sgn in (+1, -1):
            e = base.copy()
            e[k, j, i] = 1.0 / (eps0 + sgn * h)
            sc2 = H.box_scene(sc.n, pml=sc.pml, eps_inv=e, sources=sc.sources, detectors=sc.detectors,
                              design=(sc.design_lo, sc.design_hi))
            _, det = O.forward(sc2, nsteps)
            vals.append(float(np.dot(g, det)))
        fd = (vals[0] - vals[1]) / (2 * h)
        adj = grad[k - lo[2], j - lo[1], i - lo[0]]
        assert abs(fd - adj) < 1e-7 * scale, (fd, adj)


def test_gradient_from_a_random_initial_state():
    """The gradient of a solve that starts from a given state (E^0, H^{-1/2} random on the PML-free
    region): the three strategies agree, and central finite differences of the forward from the same
    state match it. The state is an input the forward and the reverse sweep share, so a gradient that
    ignored it (started from zero fields) would fail both."""
    sc = _grad_scene_cpml()
    nsteps = 40
    init = S.random_fields(sc, 23, in_r_only=True).astype(np.float64)
    g = _gvec(sc, nsteps, 5)
    g_all, _, det0 = O.gradient(sc, nsteps, g, O.METHOD_STORE_ALL, init=init)
    g_ck, _, _ = O.gradient(sc, nsteps, g, O.METHOD_CHECKPOINT, interval=16, init=init)
    g_tr, _, det2 = O.gradient(sc, nsteps, g, O.METHOD_TIME_REVERSAL, init=init)
    g_zero, _, _ = O.gradient(sc, nsteps, g, O.METHOD_STORE_ALL)
    scale = np.max(np.abs(g_all))
    assert scale > 0 and np.max(np.abs(g_zero - g_all)) > 1e-3 * scale  # the state matters
    assert np.max(np.abs(g_ck - g_all)) < 1e-13 * scale
    assert np.max(np.abs(g_tr - g_all)) < 1e-12 * scale
    assert np.array_equal(det0, det2)
    assert np.array_equal(det0, O.forward(sc, nsteps, init=init)[1])
    base = sc.eps_inv.astype(np.float64)
    h = 1e-6
    lo = sc.design_lo
    for (i, j, k) in [(7, 7, 7), (10, 5, 9)]:
        eps0 = 1.0 / base[k, j, i]
        vals = []
        for sgn in (+1, -1):
            e = base.copy()
            e[k, j, i] = 1.0 / (eps0 + sgn * h)
            sc2 = H.box_scene(sc.n, pml=sc.pml, eps_inv=e, sources=sc.sources, detectors=sc.detectors,
                              design=(sc.design_lo, sc.design_hi))
            vals.append(float(np.dot(g, O.forward(sc2, nsteps, init=init)[1])))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g_all[k - lo[2], j - lo[1], i - lo[0]]) < 1e-7 * scale


# ------------------------------------------------------------------------------------------------
# Reciprocity, linearity and detector definitions
# ------------------------------------------------------------------------------------------------

def test_reciprocity_of_point_responses():
    n = (14, 12, 10)
    nx, ny, nz = n
    rng = np.random.default_rng(31)
    eps_inv = rng.uniform(0.3, 1.0, (nz, ny, nx)).astype(np.float32)
    A, B = (4, 5, 3), (9, 7, 6)
    eps_inv[A[2], A[1], A[0]] = 1.0
    eps_inv[B[2], B[1], B[0]] = 1.0
    for ca, cb in ((2, 2), (0, 1)):
        s1 = H.box_scene(n, eps_inv=eps_inv, sources=[H.point_source(ca, A, 8.0)], detectors=[H.point_probe(cb, B)])
        s2 = H.box_scene(n, eps_inv=eps_inv, sources=[H.point_source(cb, B, 8.0)], detectors=[H.point_probe(ca, A)])
        _, d1 = O.forward(s1, 300)
        _, d2 = O.forward(s2, 300)
        assert np.max(np.abs(d1)) > 1e-6
        assert np.max(np.abs(d1 - d2)) < 1e-12 * np.max(np.abs(d1))


def mirror(f, axis, n_axis, sign, half):
    """The field array f (nz, ny, nx) reflected through the grid's mid-plane along `axis` (0 = x):
    half-position components (index i at i + 1/2) map i -> N-1-i, integer-position ones i -> N-i
    (index 0 and the implicit index N are the PEC walls, both 0), times `sign`."""
    ax = 2 - axis
    g = np.zeros_like(f)
    idx = np.arange(n_axis)
    src = (n_axis - 1 - idx) if half else (n_axis - idx)
    ok = (src >= 0) & (src < n_axis) & (half | (idx > 0))
    take = [slice(None)] * 3
    put = [slice(None)] * 3
    take[ax] = src[ok]
    put[ax] = idx[ok]
    g[tuple(put)] = sign * f[tuple(take)]
    return g


@pytest.mark.parametrize("axis", [0, 1])
def test_mirror_symmetry_of_fields(axis):
    """A scene symmetric under reflection through the mid-plane x = N/2 (or y = N/2): permittivity
    varying only along the other axes, equal CPML on the two mirrored faces, an E_z point source on the
    mid-plane. The fields are then mirror images: E_z, E_t (the other tangential E) and H_n (H along the
    mirror normal) even, E_n and the tangential H odd (E is a polar vector, H an axial one)."""
    n = (24, 20, 22)
    nx, ny, nz = n
    rng = np.random.default_rng(41)
    prof = rng.uniform(0.25, 1.0, (nz, ny if axis == 0 else 1, nx if axis == 1 else 1)).astype(np.float32)
    eps_inv = np.ascontiguousarray(np.broadcast_to(prof, (nz, ny, nx)))
    c = [n[0] // 2, n[1] // 2, 9]
    c[1 - axis] = 7  # off-centre along the other axis, so that no second symmetry hides an error
    sc = H.box_scene(n, pml=(4, 4, 3, 3, 5, 2), eps_inv=eps_inv, sources=[H.point_source(2, tuple(c), 8.0)])
    f, _ = O.forward(sc, 160)
    N = n[axis]
    # per component: sign under the reflection, half-position along the mirror axis
    for comp in range(6):
        is_h = comp >= 3
        along = comp % 3 == axis
        half = along != is_h  # E_a is at a half position along a, H_a at an integer one
        sign = (-1.0 if along else 1.0) * (-1.0 if is_h else 1.0)
        g = mirror(f[comp], axis, N, sign, half)
        scale = np.max(np.abs(f[comp]))
        assert scale > 1e-8, comp
        assert np.max(np.abs(f[comp] - g)) <= 1e-12 * scale, (comp, np.max(np.abs(f[comp] - g)) / scale)


def test_superposition_of_sources():
    n = (12, 11, 10)
    sa = H.point_source(2, (3, 4, 5), 8.0)
    sb = H.point_source(0, (8, 6, 4), 10.0, amplitude=-0.7)
    det = [H.point_probe(1, (6, 6, 6)), S.Detector(S.DET_PLANE_FLUX, (1, 1, 7), (11, 10, 8), axis=2)]
    d_a = O.forward(H.box_scene(n, sources=[sa], detectors=det), 150)[1]
    d_b = O.forward(H.box_scene(n, sources=[sb], detectors=det), 150)[1]
    f_ab, d_ab = O.forward(H.box_scene(n, sources=[sa, sb], detectors=det[:1]), 150)
    assert np.max(np.abs(d_ab - (d_a[:150] + d_b[:150]))) < 1e-13 * np.max(np.abs(d_ab))


def test_detectors_match_point_series():
    n = (12, 12, 12)
    cell = (6, 5, 7)
    src = H.point_source(2, (4, 4, 4), 8.0)
    points = [H.point_probe(c, cell) for c in range(6)]
    e2 = S.Detector(S.DET_PLANE_E2_SUM, cell, (cell[0] + 1, cell[1] + 1, cell[2] + 1))
    fl = [S.Detector(S.DET_PLANE_FLUX, cell, (cell[0] + 1, cell[1] + 1, cell[2] + 1), axis=ax) for ax in range(3)]
    nsteps = 120
    _, det = O.forward(H.box_scene(n, sources=[src], detectors=points + [e2] + fl), nsteps)
    p = det[:6 * nsteps].reshape(6, nsteps)
    e2v = det[6 * nsteps]
    assert abs(e2v - np.sum(p[:3] ** 2)) < 1e-14 * abs(e2v)
    for ax in range(3):
        f = det[6 * nsteps + 1 + ax * nsteps: 6 * nsteps + 1 + (ax + 1) * nsteps]
        a1, a2 = (ax + 1) % 3, (ax + 2) % 3
        ref = p[a1] * p[3 + a2] - p[a2] * p[3 + a1]
        assert np.max(np.abs(f - ref)) < 1e-14 * np.max(np.abs(ref))


def test_flux_sign_follows_propagation_direction():
    """A dipole at the centre of an absorbing box radiates outward: the time-integrated flux with
    normal +x is positive on the +x side and negative on the -x side."""
    n = (30, 30, 30)
    src = H.point_source(2, (15, 15, 15), 10.0)
    r = 7
    dets = [S.Detector(S.DET_PLANE_FLUX, (15 + r, 8, 8), (16 + r, 22, 22), axis=0),
            S.Detector(S.DET_PLANE_FLUX, (15 - r, 8, 8), (16 - r, 22, 22), axis=0)]
    nsteps = 160
    sc = H.box_scene(n, pml=(6,) * 6, sources=[src], detectors=dets)
    _, det = O.forward(sc, nsteps)
    plus, minus = det[:nsteps].sum(), det[nsteps:].sum()
    assert plus > 0 and minus < 0
    assert 0.7 < -minus / plus < 1.3


def test_source_timing_first_step():
    """With zero fields, the first step leaves E at a point source equal to A g(1/2) with
    g(s) = sin(2 pi (s - t0)/P) exp(-((s - t0)/tau)^2), P = lambda / S."""
    n = (8, 8, 8)
    src = H.point_source(2, (4, 4, 4), 12.0, amplitude=2.5)
    sc = H.box_scene(n, sources=[src], detectors=[H.point_probe(2, (4, 4, 4))])
    _, det = O.forward(sc, 1)
    P = 12.0 / sc.courant
    u = 0.5 - src.t0_steps
    expect = 2.5 * math.sin(2 * math.pi * u / P) * math.exp(-(u / src.tau_steps) ** 2)
    assert abs(det[0] - expect) <= 1e-15 * abs(expect)


# ------------------------------------------------------------------------------------------------
# CPML (Sec. 2.1): reflection from the absorbing layer, against a longer domain
# ------------------------------------------------------------------------------------------------

def _cpml_probe(nz, pml_hi_z, nsteps):
    n = (32, 32, nz)
    src = H.point_source(0, (16, 16, 14), 8.0)
    probe = H.point_probe(0, (16, 16, 21))
    sc = H.box_scene(n, pml=(8, 8, 8, 8, 8, pml_hi_z), sources=[src], detectors=[probe])
    return O.forward(sc, nsteps)[1]


# The reflection bar: the oracle's polynomial-graded CPML (m = 3, kappa_max = 1, alpha_max = 0,
# sigma_max = 0.8 (m + 1) S) measures -76 dB on this probe; a grading error that every face shares
# (so that mirror symmetry and GPU parity cannot see it) raises it above -65 dB.
CPML_BAR_DB = -65.0


def _cpml_reflection_db(nsteps=200):
    ref = _cpml_probe(32 + 96, 8, nsteps)          # far boundary: its echo arrives after the window
    short = _cpml_probe(32, 8, nsteps)             # CPML 3 cells beyond the probe
    return 20 * math.log10(np.max(np.abs(short - ref)) / np.max(np.abs(ref)))


def test_cpml_reflection_below_minus_65_db():
    nsteps = 200
    ref = _cpml_probe(32 + 96, 8, nsteps)
    pec = _cpml_probe(32, 0, nsteps)               # same domain closed by PEC: strong reflection
    r_pec = np.max(np.abs(pec - ref)) / np.max(np.abs(ref))
    assert r_pec > 0.1
    db = _cpml_reflection_db(nsteps)
    assert db < CPML_BAR_DB, db


@pytest.mark.parametrize("plant", ["swap_integer_and_half_tables", "depth_from_the_wrong_plane"])
def test_cpml_bar_fails_planted_grading_errors(plant, tmp_path, monkeypatch):
    """The reflection bar bites: a copy of the oracle with a grading error planted on every face
    (the integer- and half-position tables exchanged, or the depth counted from one cell outside the
    interface) fails it, while both sides of the comparison use the same planted copy."""
    from oracle import build as OB
    src = open(OB.SRC).read()
    if plant == "swap_integer_and_half_tables":
        bad = src.replace("grade(s, d, double(i), a.b_int[i]", "grade(s, d, i + 0.5, a.b_int[i]")
        bad = bad.replace("grade(s, d, i + 0.5, a.b_half[i]", "grade(s, d, double(i), a.b_half[i]")
    else:
        bad = src.replace("d = (p0 - x) / p0;", "d = (p0 - 1 - x) / p0;")
        bad = bad.replace("d = (x - (N - p1)) / p1;", "d = (x + 1 - (N - p1)) / p1;")
    assert bad != src
    cpp = tmp_path / "planted.cpp"
    cpp.write_text(bad)
    lib = OB.compile_source(str(cpp), str(tmp_path / "planted.so"))
    monkeypatch.setattr(O, "_LIB", O.load(lib))
    db = _cpml_reflection_db()
    assert db > CPML_BAR_DB, (plant, db)
