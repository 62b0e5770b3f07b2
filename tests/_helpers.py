"""Scene builders and index sets shared by the tests (inputs and test-side bookkeeping only)."""
import math

import numpy as np

from paper_2412_12360_b300 import scenes as S


def box_scene(n, pml=(0,) * 6, eps_inv=None, sources=(), detectors=(), design=None, nsteps=100,
              courant=None, sigma_max=None, name="test"):
    nx, ny, nz = n
    Sn = S.courant_from_factor(0.99) if courant is None else courant
    if eps_inv is None:
        eps_inv = np.ones((nz, ny, nx), dtype=np.float32)
    if design is None:
        design = ((0, 0, 0), (0, 0, 0))
    sm = S.default_sigma_max(Sn) if sigma_max is None else sigma_max
    return S.Scene(name, tuple(n), Sn, tuple(pml), sm, 1.0, 0.0, 3, np.asarray(eps_inv), list(sources),
                   list(detectors), tuple(design[0]), tuple(design[1]), nsteps)


def point_source(comp, cell, wavelength=20.0, amplitude=1.0, courant=None):
    Sn = S.courant_from_factor(0.99) if courant is None else courant
    c = tuple(cell)
    return S.default_pulse(S.Source(comp, c, (c[0] + 1, c[1] + 1, c[2] + 1), None, amplitude, wavelength), Sn)


def point_probe(comp, cell):
    c = tuple(cell)
    return S.Detector(S.DET_POINT_SERIES, c, (c[0] + 1, c[1] + 1, c[2] + 1), component=comp)


def r_masks(scene):
    """Boolean masks (6, nz, ny, nx) of the components in the PML-free region R: along an axis with
    layers p0, p1 and N cells, integer positions p0 .. min(N - p1, N - 1) and half positions
    p0 .. N - p1 - 1; E tangential to a PEC wall at index 0 is excluded."""
    nx, ny, nz = scene.n
    n = (nx, ny, nz)
    rng_int, rng_half = [], []
    for d in range(3):
        p0, p1 = scene.pml[2 * d], scene.pml[2 * d + 1]
        idx = np.arange(n[d])
        rng_int.append((idx >= p0) & (idx <= min(n[d] - p1, n[d] - 1)))
        rng_half.append((idx >= p0) & (idx <= n[d] - p1 - 1))
    masks = np.zeros((6, nz, ny, nx), dtype=bool)
    for f in range(6):
        c = f % 3
        sel = []
        for d in range(3):
            own = (d == c)
            half = own if f < 3 else not own   # E_c is half along c; H_c is half along the others
            sel.append(rng_half[d] if half else rng_int[d])
        m = sel[2][:, None, None] & sel[1][None, :, None] & sel[0][None, None, :]
        if f < 3:
            c1, c2 = (c + 1) % 3, (c + 2) % 3
            idx = [np.arange(n[d]) for d in range(3)]
            pec = np.zeros((nz, ny, nx), dtype=bool)
            for d in (c1, c2):
                shape = [1, 1, 1]
                shape[2 - d] = n[d]
                pec |= (idx[d] == 0).reshape(shape)
            m &= ~pec
        masks[f] = m
    return masks


def mode_fields(n, m, seed_vec=(1.0, 2.0, 3.0)):
    """Divergence-free discrete PEC cavity mode (m_x, m_y, m_z) on the Yee grid, as initial E (H = 0).

    E_x(i+1/2, j, k) = A_x cos(k_x (i+1/2)) sin(k_y j) sin(k_z k), and cyclically, with k_c = m_c pi / N_c
    and A orthogonal to (sin(k_x/2), sin(k_y/2), sin(k_z/2)) so that the discrete divergence vanishes.
    """
    nx, ny, nz = n
    k = [m[d] * math.pi / n[d] for d in range(3)]
    s = np.array([math.sin(kk / 2) for kk in k])
    A = np.cross(s, np.asarray(seed_vec, dtype=np.float64))
    if np.linalg.norm(A) < 1e-6:
        A = np.cross(s, np.array([3.0, -1.0, 2.0]))
    A /= np.linalg.norm(A)
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    kk = np.arange(nz)[:, None, None]
    f = np.zeros((6, nz, ny, nx))
    f[0] = A[0] * np.cos(k[0] * (i + 0.5)) * np.sin(k[1] * j) * np.sin(k[2] * kk)
    f[1] = A[1] * np.sin(k[0] * i) * np.cos(k[1] * (j + 0.5)) * np.sin(k[2] * kk)
    f[2] = A[2] * np.sin(k[0] * i) * np.sin(k[1] * j) * np.cos(k[2] * (kk + 0.5))
    return f


def fit_cos_theta(e):
    """Least-squares c in e[n+1] + e[n-1] = 2 c e[n]."""
    e = np.asarray(e, dtype=np.float64)
    num = np.sum((e[2:] + e[:-2]) * e[1:-1])
    den = 2.0 * np.sum(e[1:-1] ** 2)
    return num / den


def discrete_theta(n, m, courant, a=1.0):
    """Yee dispersion for a PEC cavity mode: sin(theta/2) = S sqrt(a) sqrt(sum sin^2(m_c pi / (2 N_c)))."""
    ssum = sum(math.sin(m[d] * math.pi / (2 * n[d])) ** 2 for d in range(3))
    return 2.0 * math.asin(courant * math.sqrt(a) * math.sqrt(ssum))
