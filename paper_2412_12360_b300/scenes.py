"""Seeded synthetic scenes (inputs only) for the Yee FDTD hot path.

This module builds inputs: grid sizes, the per-cell inverse permittivity a = 1/eps, source boxes and
their spatial profiles, detector boxes and design boxes. It holds none of the method's arithmetic
(no field update, no CPML coefficient, no waveform sample), so both the CUDA path and the FP64
oracle can take their inputs from it.

Workloads are synthetic stand-ins shaped like the scenes of arXiv 2412.12360: the speed-test volume
of Sec. 3.1 (Table 2), the Si/SiO2 waveguide with a design box of Sec. 3.2, and a random-density
design region. The paper's device geometries and datasets are not used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Field component indices, x fastest in every array.
EX, EY, EZ, HX, HY, HZ = range(6)

# Detector kinds.
DET_POINT_SERIES = 0   # one field component at one cell, every step
DET_PLANE_E2_SUM = 1   # per cell of a box: sum over steps of Ex^2 + Ey^2 + Ez^2
DET_PLANE_FLUX = 2     # per step: sum over a box of (E x H) along an axis
DET_PLANE_E2_SUM_INTERP = 3  # as 1, with E interpolated to the cell centres
DET_PLANE_FLUX_INTERP = 4    # as 2, with E and H at the cell centres and E at time n + 1/2

SPEED_OF_LIGHT = 299792458.0


@dataclass
class Source:
    """Source on E component `component` over the cell box [lo, hi): a soft source (tfsf = 0) or the
    plane of a one-sided total-field / scattered-field source (tfsf = +-(axis + 1), the sign giving
    the direction of travel; the box is one cell thick along the axis)."""
    component: int
    lo: Tuple[int, int, int]
    hi: Tuple[int, int, int]
    profile: Optional[np.ndarray]   # float32 (hz, hy, hx) weights or None (1 everywhere)
    amplitude: float = 1.0
    wavelength_cells: float = 20.0
    tau_steps: float = 0.0          # 0: filled in as one period by `default_pulse`
    t0_steps: float = 0.0
    tfsf: int = 0
    eps_background: float = 1.0     # TFSF: permittivity of the incident-field line


@dataclass
class Detector:
    kind: int
    lo: Tuple[int, int, int]
    hi: Tuple[int, int, int]
    component: int = 0
    axis: int = 2


@dataclass
class Scene:
    name: str
    n: Tuple[int, int, int]                 # cells (nx, ny, nz)
    courant: float                          # S = c dt / dx
    pml: Tuple[int, int, int, int, int, int]
    sigma_max: float
    kappa_max: float
    alpha_max: float
    grading_m: int
    eps_inv: np.ndarray                     # float32 (nz, ny, nx)
    sources: List[Source]
    detectors: List[Detector]
    design_lo: Tuple[int, int, int]
    design_hi: Tuple[int, int, int]
    nsteps: int
    extra: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def r_cell_box(self):
        """Cells all six of whose components lie in the PML-free region (lo inclusive, hi exclusive)."""
        lo = tuple(self.pml[2 * d] for d in range(3))
        hi = tuple(self.n[d] - self.pml[2 * d + 1] for d in range(3))
        return lo, hi

    def design_shape(self):
        return tuple(self.design_hi[d] - self.design_lo[d] for d in (2, 1, 0))


def courant_from_factor(factor: float = 0.99) -> float:
    """Courant number S = c dt / dx for a factor of the 3D stability limit 1/sqrt(3).

    Sec. 3.1 and Table 2 give step counts that equal T c sqrt(3) / (0.99 dx), i.e. the paper's
    "courant factor 0.99" multiplies the 3D limit.
    """
    return factor / math.sqrt(3.0)


def steps_for(duration_s: float, dx_m: float, factor: float = 0.99) -> int:
    """Time steps for a simulated duration at grid spacing dx (Table 2 of Sec. 3.1)."""
    dt = courant_from_factor(factor) * dx_m / SPEED_OF_LIGHT
    return int(round(duration_s / dt))


def grid_for(size_m: Sequence[float], dx_m: float) -> Tuple[int, int, int]:
    """Cells per axis for a box of physical size `size_m` at spacing dx."""
    return tuple(int(round(s / dx_m)) for s in size_m)


def default_sigma_max(courant: float, grading_m: int = 3, eps_background: float = 1.0) -> float:
    """Normalised peak PML conductivity 0.8 (m + 1) S / sqrt(eps_bg): the usual polynomial-grading
    choice for the CPML of Sec. 2.1 (the paper gives no parameters)."""
    return 0.8 * (grading_m + 1) * courant / math.sqrt(eps_background)


def default_pulse(src: Source, courant: float) -> Source:
    """Envelope width of one period and a centre three widths in, in steps."""
    period = src.wavelength_cells / courant
    if src.tau_steps <= 0:
        src.tau_steps = period
    if src.t0_steps <= 0:
        src.t0_steps = 3.0 * src.tau_steps
    return src


def gaussian_sheet(shape_hw: Tuple[int, int], w0: float) -> np.ndarray:
    """exp(-r^2 / w0^2) over a (rows, cols) sheet, centred on the sheet (float32)."""
    h, w = shape_hw
    yy = np.arange(h, dtype=np.float64) - (h - 1) / 2.0
    xx = np.arange(w, dtype=np.float64) - (w - 1) / 2.0
    r2 = yy[:, None] ** 2 + xx[None, :] ** 2
    return np.exp(-r2 / (w0 * w0)).astype(np.float32)


def uniform_rho(shape, seed: int) -> np.ndarray:
    """rho ~ U[0, 1), float32, from a seeded torch CPU generator (shape (dz, dy, dx))."""
    import torch
    g = torch.Generator().manual_seed(int(seed))
    return torch.rand(tuple(shape), generator=g, dtype=torch.float32).numpy()


def inv(eps: np.ndarray) -> np.ndarray:
    """Per-cell inverse permittivity, rounded once to float32 (the value both sides use)."""
    return (1.0 / np.asarray(eps, dtype=np.float64)).astype(np.float32)


def _box(lo, hi):
    return tuple(int(v) for v in lo), tuple(int(v) for v in hi)


# ---------------------------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------------------------

def cavity_32(nsteps: int = 500) -> Scene:
    """32^3 PEC box, dx = lambda/20 at lambda = 1.55 um, vacuum with a centred 8^3 cube of eps 2.25,
    Ez point dipole with a Gaussian-modulated pulse (plain forward and round-trip workload)."""
    n = (32, 32, 32)
    S = courant_from_factor(0.99)
    eps = np.ones(n[::-1], dtype=np.float64)
    eps[12:20, 12:20, 12:20] = 2.25
    src = default_pulse(Source(EZ, (11, 13, 14), (12, 14, 15), None, 1.0, 20.0), S)
    dets = [Detector(DET_POINT_SERIES, (20, 18, 17), (21, 19, 18), component=EZ),
            Detector(DET_POINT_SERIES, (7, 22, 9), (8, 23, 10), component=HX),
            Detector(DET_PLANE_E2_SUM, (2, 2, 24), (30, 30, 25)),
            Detector(DET_PLANE_FLUX, (2, 2, 24), (30, 30, 25), axis=2)]
    return Scene("cavity_32", n, S, (0,) * 6, 0.0, 1.0, 0.0, 3, inv(eps), [src], dets,
                 (12, 12, 12), (20, 20, 20), nsteps)


def design_box_scene(n=(96, 96, 96), pml=10, design=40, nsteps=2000, seed=1234,
                     eps_lo=1.0, eps_hi=12.1, wavelength_cells=20.0, name=None, tfsf=False,
                     interp=False) -> Scene:
    """Cubic grid with a CPML on every face, an Ex Gaussian-beam sheet near z-lo (a soft source, or
    with tfsf=True a one-sided TFSF plane sending the beam towards +z), a centred design box with
    eps = eps_lo + (eps_hi - eps_lo) rho, rho ~ U[0,1), and a time-integrated |E|^2 plane near z-hi
    (objective: the sum of that plane; with interp=True the plane uses E interpolated to the cell
    centres)."""
    nx, ny, nz = n
    S = courant_from_factor(0.99)
    eps = np.ones((nz, ny, nx), dtype=np.float64)
    dlo = tuple((n[d] - design) // 2 for d in range(3))
    dhi = tuple(dlo[d] + design for d in range(3))
    rho = uniform_rho((design, design, design), seed)
    eps32 = (np.float32(eps_lo) + np.float32(eps_hi - eps_lo) * rho).astype(np.float32)
    eps[dlo[2]:dhi[2], dlo[1]:dhi[1], dlo[0]:dhi[0]] = eps32
    lo_r = (pml, pml)
    hi_r = (nx - pml, ny - pml)
    w0 = 0.25 * (nx - 2 * pml)
    zs = pml + 5
    zd = nz - pml - 8
    prof = gaussian_sheet((hi_r[1] - lo_r[1], hi_r[0] - lo_r[0]), w0)[None]
    src = default_pulse(Source(EX, (lo_r[0], lo_r[1], zs), (hi_r[0], hi_r[1], zs + 1), prof, 1.0,
                               wavelength_cells, tfsf=3 if tfsf else 0), S)
    if interp:  # the interpolation stencil reaches one cell beyond the box: keep it in the PML-free region
        det = Detector(DET_PLANE_E2_SUM_INTERP, (lo_r[0], lo_r[1], zd), (hi_r[0] - 1, hi_r[1] - 1, zd + 1))
    else:
        det = Detector(DET_PLANE_E2_SUM, (lo_r[0], lo_r[1], zd), (hi_r[0], hi_r[1], zd + 1))
    sc = Scene(name or "design_%d" % nx, n, S, (pml,) * 6, default_sigma_max(S), 1.0, 0.0, 3, inv(eps),
               [src], [det], dlo, dhi, nsteps)
    sc.extra.update(rho=rho, eps_lo=eps_lo, eps_hi=eps_hi, seed=seed)
    return sc


def design_96(nsteps: int = 2000) -> Scene:
    """96^3, 10-cell CPML, Gaussian-beam sheet, 40^3 design box eps = 1 + 11.1 rho (seed 1234),
    |E|^2 plane objective."""
    return design_box_scene((96, 96, 96), 10, 40, nsteps, 1234, 1.0, 12.1, 20.0, "design_96")


def waveguide_scene(n=(600, 600, 600), pml=12, design=200, nsteps=4000, seed=600, axis=0,
                    core=(25, 11), eps_clad=2.085, eps_core=12.25, wavelength_cells=77.5,
                    name=None) -> Scene:
    """Si waveguide (eps 12.25, core `core` cells) along `axis` in SiO2 (eps 2.085), a centred design
    box eps = 2.085 + 10.165 rho (`design` cells per axis, or (dx, dy, dz)), an E sheet over the core
    cross-section near the low end and a Poynting-flux plane near the high end (objective: the time
    sum of the flux)."""
    nx, ny, nz = n
    S = courant_from_factor(0.99)
    eps = np.full((nz, ny, nx), eps_clad, dtype=np.float32)
    t1, t2 = (axis + 1) % 3, (axis + 2) % 3
    c_lo = [0, 0, 0]
    c_hi = list(n)
    c_lo[t1] = (n[t1] - core[0]) // 2
    c_hi[t1] = c_lo[t1] + core[0]
    c_lo[t2] = (n[t2] - core[1]) // 2
    c_hi[t2] = c_lo[t2] + core[1]
    sl = tuple(slice(c_lo[d], c_hi[d]) for d in (2, 1, 0))
    eps[sl] = eps_core
    dsz = (design,) * 3 if np.isscalar(design) else tuple(int(v) for v in design)
    dlo = tuple((n[d] - dsz[d]) // 2 for d in range(3))
    dhi = tuple(dlo[d] + dsz[d] for d in range(3))
    rho = uniform_rho(dsz[::-1], seed)
    eps[dlo[2]:dhi[2], dlo[1]:dhi[1], dlo[0]:dhi[0]] = (
        np.float32(eps_clad) + np.float32(eps_core - eps_clad) * rho)
    # source sheet over the core cross-section, transverse component t1
    s_lo = list(c_lo)
    s_hi = list(c_hi)
    s_lo[axis] = pml + 10
    s_hi[axis] = pml + 11
    w0 = 0.5 * max(core)
    # Gaussian profile over the (t1, t2) cross-section, laid out as the box (hz, hy, hx)
    coords = [np.arange(s_lo[d], s_hi[d], dtype=np.float64) - (c_lo[d] + c_hi[d] - 1) / 2.0
              for d in range(3)]
    zz, yy, xx = np.meshgrid(coords[2], coords[1], coords[0], indexing="ij")
    rr = [xx, yy, zz]
    r2 = rr[t1] ** 2 + rr[t2] ** 2
    prof = np.exp(-r2 / (w0 * w0)).astype(np.float32)
    src = default_pulse(Source(t1, tuple(s_lo), tuple(s_hi), prof, 1.0, wavelength_cells), S)
    f_lo = [pml, pml, pml]
    f_hi = [n[0] - pml, n[1] - pml, n[2] - pml]
    f_lo[axis] = n[axis] - pml - 11
    f_hi[axis] = f_lo[axis] + 1
    det = Detector(DET_PLANE_FLUX, tuple(f_lo), tuple(f_hi), axis=axis)
    sc = Scene(name or "waveguide_%dx%dx%d" % n, n, S, (pml,) * 6,
               default_sigma_max(S, 3, eps_clad), 1.0, 0.0, 3, inv(eps.astype(np.float64)), [src], [det],
               dlo, dhi, nsteps)
    sc.extra.update(rho=rho, eps_lo=eps_clad, eps_hi=eps_core, seed=seed)
    return sc


def waveguide_600(nsteps: int = 4000) -> Scene:
    """600^3 (216 M cells), dx = 20 nm, 12-cell CPML, Si waveguide along x, 200^3 design box."""
    return waveguide_scene((600, 600, 600), 12, 200, nsteps, 600, 0, name="waveguide_600")


def waveguide_600_slab(nz: int = 64, nsteps: int = 4000) -> Scene:
    """A z-slab of waveguide_600: its full 600 x 600 cross-section (12-cell CPML, Si core along x, the
    sheet source at x = 22 and the flux plane at x = 577) over nz planes with a 12-cell CPML at both
    z ends, and the design box cut to 200 x 200 x (nz - 24). A bounded sample of the large solve for
    timing the CPU oracle, whose FP64 state for the full grid is about 70 GB."""
    return waveguide_scene((600, 600, nz), 12, (200, 200, nz - 24), nsteps, 600, 0,
                           name="waveguide_600_slab%d" % nz)


def waveguide_batch_member(b: int, nsteps: int = 3000, n=(240, 240, 960), design=120) -> Scene:
    """One of 16 designs of a 240x240x960 waveguide (along z), 120^3 design box, seed 500 + b."""
    return waveguide_scene(n, 12, design, nsteps, 500 + b, 2, name="waveguide_batch_%d" % b)


SERVED_GRIDS = [(64, 64, 64), (96, 96, 96), (128, 128, 256), (200, 200, 200)]


def served_request(req_id: int, rng: np.random.Generator, grids=None) -> Scene:
    """A served fwd+grad request: grid drawn from `grids` (default {64^3, 96^3, 128x128x256, 200^3}),
    1000-3000 steps, 10-cell CPML, design box of half the extent, rho seed 10000 + id."""
    grids = SERVED_GRIDS if grids is None else grids
    n = grids[int(rng.integers(len(grids)))]
    nsteps = int(rng.integers(1000, 3001))
    design = min(n) // 2
    sc = design_box_scene(n, 10, design, nsteps, 10000 + req_id, 1.0, 12.1, 20.0, "served_%d" % req_id)
    return sc


def random_fields(scene: Scene, seed: int, in_r_only: bool = False) -> np.ndarray:
    """Seeded random initial fields (6, nz, ny, nx) float32, zero on E components held by a PEC wall
    (tangential E at index 0). With in_r_only, zero outside the PML-free cell box."""
    nx, ny, nz = scene.n
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((6, nz, ny, nx)).astype(np.float32)
    f[EX, 0, :, :] = 0; f[EX, :, 0, :] = 0
    f[EY, 0, :, :] = 0; f[EY, :, :, 0] = 0
    f[EZ, :, 0, :] = 0; f[EZ, :, :, 0] = 0
    if in_r_only:
        (lx, ly, lz), (hx, hy, hz) = scene.r_cell_box()
        mask = np.zeros((nz, ny, nx), dtype=bool)
        mask[lz:hz, ly:hy, lx:hx] = True
        f *= mask[None]
    return f
