"""The launch plan fdtd_create chooses, computed on the host (no GPU): the reverse-step kind of a grid
and the frame of the split adjoint step (tile columns and rows that need the x/y CPML loop around a
rectangle of plain tiles). The frame must cover exactly the tiles whose march reaches a layer, so that
the plain kernel, which holds no CPML code, never runs a tile that needs it."""
import ctypes as C
import dataclasses

import numpy as np

from paper_2412_12360_b300 import fdtd as F
from paper_2412_12360_b300 import scenes as S

TX, TY = 32, 16  # column tile of the fused kernels (x cells, y rows)


def needs_cpml(offset, width, n, p_lo, p_hi):
    """A tile column (or row) starting at `offset` needs the x/y CPML loop when the tile, its one-cell
    low halo or the +1 neighbours of its cells reach a layer of that axis."""
    return offset - 1 < p_lo or offset + width >= n - p_hi - 1


_BASE = S.design_box_scene((40, 36, 44), 6, 12, 10, 71)


def grid(n, p):
    """A scene with grid n and layers p on every face (only the grid and the layers are read)."""
    return dataclasses.replace(_BASE, n=tuple(n), pml=(p,) * 6)


def test_reverse_kind_and_frame_of_the_workloads():
    assert F.reverse_kind(grid((600, 600, 600), 12)) == 1              # the 600^3 waveguide
    assert F.adjoint_frame(grid((600, 600, 600), 12)) == (1, (1, 1, 1, 2))
    assert F.reverse_kind(grid((96, 96, 96), 10)) == 0                 # design_96
    assert F.reverse_kind(grid((240, 240, 960), 12)) == 1              # 55 M cells, 35 % CPML tiles
    assert F.reverse_kind(grid((200, 200, 200), 10)) == 0              # 56 % CPML tiles
    assert F.reverse_kind(grid((256, 256, 256), 10)) == 1
    assert F.reverse_kind(grid((128, 128, 256), 10)) == 0              # 4 M cells
    assert F.adjoint_frame(_BASE)[0] == 0   # two tile columns, both at a layer: one launch


def test_frame_covers_exactly_the_cpml_tiles():
    rng = np.random.default_rng(11)
    checked = split = 0
    for _ in range(400):
        n = tuple(int(v) for v in rng.integers(20, 700, size=3))
        pml = tuple(int(v) for v in rng.integers(0, 16, size=6))
        if any(pml[2 * d] + pml[2 * d + 1] + 4 > n[d] for d in range(3)):
            continue
        sc = dataclasses.replace(_BASE, n=n, pml=pml)
        ok, (xl, xh, yl, yh) = F.adjoint_frame(sc)
        ntx, nty = -(-n[0] // TX), -(-n[1] // TY)
        cols = [needs_cpml(b * TX, TX, n[0], pml[0], pml[1]) for b in range(ntx)]
        rows = [needs_cpml(b * TY, TY, n[1], pml[2], pml[3]) for b in range(nty)]
        if ok:
            split += 1
            assert xl + xh < ntx and yl + yh < nty
            assert all(cols[:xl]) and all(cols[ntx - xh:]) and not any(cols[xl:ntx - xh])
            assert all(rows[:yl]) and all(rows[nty - yh:]) and not any(rows[yl:nty - yh])
        else:  # no plain rectangle: every column or every row needs the CPML loop
            assert all(cols) or all(rows)
        checked += 1
    assert checked > 200 and split > 100


def test_launch_plan_queries_reject_bad_input():
    L = F.lib()
    g, p = F.make_grid((4, 4, 4)), F.make_pml(_BASE)
    f = (C.c_int32 * 4)()
    assert L.fdtd_reverse_kind(None, C.byref(p)) == F.FDTD_ERR_INVALID_ARG
    assert L.fdtd_adjoint_frame(C.byref(g), C.byref(p), f) == F.FDTD_ERR_INVALID_ARG  # layers wider than the grid
    assert L.fdtd_adjoint_frame(C.byref(g), C.byref(p), None) == F.FDTD_ERR_INVALID_ARG
