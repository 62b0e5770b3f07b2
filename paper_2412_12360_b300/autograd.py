"""torch.autograd.Function over the FDTD solve and its time-reversal gradient (arXiv 2412.12360 Sec. 2.2).

    det = FDTDSolve.apply(rho, solvers, eps_lo, eps_hi, nsteps, mode)

rho is a CUDA float tensor [B, dz, dy, dx] of design densities in [0, 1] (eps = eps_lo + (eps_hi -
eps_lo) rho on each solver's design box); det is [B, n_det] float64, the concatenated detector
outputs of each design. Any torch loss of det can be back-propagated: the backward pass hands
dL/d(det) to the library's reverse sweep and returns dL/drho. All field arithmetic, the density map
and the dL/drho scaling run in the CUDA library; this module only moves pointers and orders the
solvers' streams against torch's current stream (events both ways), so that solvers created on
their own streams, or calls made under torch.cuda.stream(...), read inputs that are complete and
hand back outputs that are.

mode "keep" records the boundary faces during the forward pass and reverses from them (one forward
and one reversed sweep per design). mode "recompute" runs a plain forward first and, in backward,
runs the recorded forward again immediately before the reverse sweep of each design and frees that
history afterwards, so only one face history at a time is held in device memory (used for batches
whose histories do not fit). An integer mode k is the mix of the two: designs 0..k-1 keep their
histories from the forward pass, the others recompute; the backward reverses the kept designs first
and frees each history, so the recomputed ones find the room (for batches where some, but not all,
histories fit beside the states).
"""
from __future__ import annotations

from typing import List, Sequence

import torch

from . import fdtd


def _det_buffer(solver, device):
    return torch.empty(solver.fdtd_detector_total(), dtype=torch.float64, device=device)


def _torch_stream(solver, device):
    """The torch view of the stream a solver enqueues on (None at creation: the legacy default stream)."""
    st = solver.stream
    if st is None:
        return torch.cuda.default_stream(device)
    if isinstance(st, torch.cuda.Stream):
        return st
    return torch.cuda.ExternalStream(int(st), device=device)


def _streams(solvers, device):
    out = {}
    for s in solvers:
        st = _torch_stream(s, device)
        out.setdefault(st.cuda_stream, st)
    return list(out.values())


def _wait_for_torch(streams, device):
    """Make every solver stream wait for the work queued so far on torch's current stream (the inputs
    the solvers read are produced there)."""
    cur = torch.cuda.current_stream(device)
    ev = torch.cuda.Event()
    ev.record(cur)
    for st in streams:
        if st.cuda_stream != cur.cuda_stream:
            st.wait_event(ev)


def _torch_waits(streams, device, tensors=()):
    """Make torch's current stream wait for the solver streams (their outputs are read there), and
    keep the caching allocator from reusing `tensors` before the solver streams are done with them."""
    cur = torch.cuda.current_stream(device)
    for st in streams:
        if st.cuda_stream == cur.cuda_stream:
            continue
        ev = torch.cuda.Event()
        ev.record(st)
        cur.wait_event(ev)
        for t in tensors:
            t.record_stream(st)


class FDTDSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho: torch.Tensor, solvers: Sequence["fdtd.Solver"], eps_lo: float, eps_hi: float,
                nsteps: int, mode: str = "keep"):
        if not rho.is_cuda or rho.dtype != torch.float32:
            raise TypeError("rho must be a CUDA float32 tensor [B, dz, dy, dx]")
        if rho.shape[0] != len(solvers):
            raise ValueError("one solver per design is needed")
        if isinstance(mode, bool) or not (mode in ("keep", "recompute") or (isinstance(mode, int) and mode >= 0)):
            raise ValueError("mode is 'keep', 'recompute' or the number of designs that keep their histories")
        nkeep = len(solvers) if mode == "keep" else (0 if mode == "recompute" else min(int(mode), len(solvers)))
        rho_c = rho.detach().contiguous()
        streams = _streams(solvers, rho.device)
        outs: List[torch.Tensor] = [_det_buffer(s, rho.device) for s in solvers]
        _wait_for_torch(streams, rho.device)
        for b, s in enumerate(solvers):
            s.fdtd_set_design_density(rho_c[b], eps_lo, eps_hi)
            s.fdtd_forward(nsteps, record_faces=b < nkeep)
            s.fdtd_read_detectors(outs[b])
        _torch_waits(streams, rho.device, [rho_c] + outs)
        ctx.solvers = list(solvers)
        ctx.eps = (float(eps_lo), float(eps_hi))
        ctx.nsteps = int(nsteps)
        ctx.mode = mode
        ctx.nkeep = nkeep
        ctx.save_for_backward(rho_c)
        return torch.stack(outs)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        (rho_c,) = ctx.saved_tensors
        grad = torch.empty_like(rho_c)
        gd = g.detach().to(torch.float64).contiguous()
        streams = _streams(ctx.solvers, rho_c.device)
        _wait_for_torch(streams, rho_c.device)
        for b, s in enumerate(ctx.solvers):  # the designs that kept their histories come first
            if b >= ctx.nkeep:
                s.fdtd_set_design_density(rho_c[b], *ctx.eps)
                s.fdtd_forward(ctx.nsteps, record_faces=True)
            s.fdtd_backward_density(gd[b], grad[b])
            if ctx.mode != "keep":
                s.fdtd_release_history()  # room for the designs still to recompute
        _torch_waits(streams, rho_c.device, [rho_c, gd, grad])
        return grad, None, None, None, None, None


def solve(rho: torch.Tensor, solvers: Sequence["fdtd.Solver"], eps_lo: float, eps_hi: float, nsteps: int,
          mode="keep") -> torch.Tensor:
    """Differentiable detector outputs [B, n_det] for densities rho [B, dz, dy, dx]."""
    return FDTDSolve.apply(rho, solvers, eps_lo, eps_hi, nsteps, mode)


def histories_that_fit(scenes, nsteps: int, budget_bytes: int) -> int:
    """How many designs (from the first) can keep their face histories beside every design's state;
    the rest recompute (the mode to pass to `solve`). -1 when not even the states and one history fit."""
    base = sum(fdtd.footprint_bytes(sc, nsteps, record_faces=False) for sc in scenes)
    hist = [fdtd.footprint_bytes(sc, nsteps, record_faces=True) - fdtd.footprint_bytes(sc, nsteps, record_faces=False)
            for sc in scenes]
    if base + max(hist, default=0) > budget_bytes:
        return -1
    k, used = 0, base
    while k < len(scenes) and used + hist[k] <= budget_bytes:
        used += hist[k]
        k += 1
    return k


def fits_in_memory(scenes, nsteps: int, budget_bytes: int) -> bool:
    """Whether every design's solver with its face history fits in `budget_bytes` at once."""
    return sum(fdtd.footprint_bytes(sc, nsteps, record_faces=True) for sc in scenes) <= budget_bytes
