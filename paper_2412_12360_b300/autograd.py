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

mode says how each design's reverse sweep gets its boundary-face history (Sec. 2.2):
  "keep": recorded whole during the forward pass (one forward and one reversed sweep per design);
  "recompute": a plain forward first and, in backward, the recorded forward again right before the
    design's reverse sweep (only one history at a time in device memory);
  an integer k: designs 0..k-1 keep, the others recompute;
  a list plan[b] per design: 0 keeps the whole history, L > 0 keeps segments of L steps (the faces
    of the last segment and the segment start states; the reverse sweep regenerates the earlier
    segments, T - L extra forward steps instead of T), -1 recomputes (see history_plan).
The backward reverses the designs that hold histories first and frees each design's reverse-sweep
state after its sweep, so the recomputed ones find the room.
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
        plan = _plan_of(mode, len(solvers))
        rho_c = rho.detach().contiguous()
        streams = _streams(solvers, rho.device)
        outs: List[torch.Tensor] = []
        _wait_for_torch(streams, rho.device)
        for b, s in enumerate(solvers):
            s.fdtd_set_design_density(rho_c[b], eps_lo, eps_hi)
            s.fdtd_set_segment_steps(max(plan[b], 0))
            s.fdtd_forward(nsteps, record_faces=plan[b] >= 0)
            outs.append(_det_buffer(s, rho.device))  # (its size is known once a forward has run)
            s.fdtd_read_detectors(outs[b])
        _torch_waits(streams, rho.device, [rho_c] + outs)
        ctx.solvers = list(solvers)
        ctx.eps = (float(eps_lo), float(eps_hi))
        ctx.nsteps = int(nsteps)
        ctx.plan = plan
        ctx.save_for_backward(rho_c)
        return torch.stack(outs)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        (rho_c,) = ctx.saved_tensors
        grad = torch.empty_like(rho_c)
        gd = g.detach().to(torch.float64).contiguous()
        streams = _streams(ctx.solvers, rho_c.device)
        _wait_for_torch(streams, rho_c.device)
        order = [b for b in range(len(ctx.solvers)) if ctx.plan[b] >= 0] + \
                [b for b in range(len(ctx.solvers)) if ctx.plan[b] < 0]   # histories held come first
        for b in order:
            s = ctx.solvers[b]
            if ctx.plan[b] < 0:
                s.fdtd_set_design_density(rho_c[b], *ctx.eps)
                s.fdtd_set_segment_steps(0)
                s.fdtd_forward(ctx.nsteps, record_faces=True)
            s.fdtd_backward_density(gd[b], grad[b])
            if len(ctx.solvers) > 1:
                s.fdtd_release_history()  # room for the designs still to come
        _torch_waits(streams, rho_c.device, [rho_c, gd, grad])
        return grad, None, None, None, None, None


def _plan_of(mode, n):
    """Per-design history plan (0 whole, L > 0 segments of L steps, -1 recompute) for a mode."""
    if isinstance(mode, bool):
        raise ValueError("bad mode")
    if mode == "keep":
        return [0] * n
    if mode == "recompute":
        return [-1] * n
    if isinstance(mode, int) and mode >= 0:
        return [0 if b < mode else -1 for b in range(n)]
    if isinstance(mode, (list, tuple)) and len(mode) == n and all(isinstance(v, int) and v >= -1 for v in mode):
        return list(mode)
    raise ValueError("mode is 'keep', 'recompute', the number of designs that keep their histories, or a "
                     "per-design plan (0 whole history, L > 0 segments of L steps, -1 recompute)")


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


def history_plan(scenes, nsteps: int, budget_bytes: int, max_segments: int = 16):
    """Per design (in order): 0 when its whole face history still fits beside every design's state and
    the histories planned so far, else the segment length L (segments of L steps; the fewest extra
    forward steps, T - L, among the lengths whose history fits), else -1 (recompute in backward).
    The backward frees each design's reverse-sweep state after its sweep, so one adjoint state at a
    time is counted. Returns (plan, extra forward steps)."""
    adj = [fdtd.adjoint_bytes(sc) for sc in scenes]
    base = sum(fdtd.footprint_bytes(sc, nsteps, record_faces=False) for sc in scenes) - sum(adj) + max(adj, default=0)
    used = base
    plan, extra = [], 0
    for sc in scenes:
        whole = fdtd.history_bytes(sc, nsteps, 0)
        if used + whole <= budget_bytes:
            plan.append(0)
            used += whole
            continue
        best = None
        for S in range(2, max_segments + 1):
            L = -(-nsteps // S)
            hb = fdtd.history_bytes(sc, nsteps, L)
            if used + hb <= budget_bytes:
                best = (L, hb)
                break
        if best is None:
            plan.append(-1)
            extra += nsteps
        else:
            plan.append(best[0])
            used += best[1]
            extra += nsteps - best[0]
    return plan, extra


def fits_in_memory(scenes, nsteps: int, budget_bytes: int) -> bool:
    """Whether every design's solver with its face history fits in `budget_bytes` at once."""
    return sum(fdtd.footprint_bytes(sc, nsteps, record_faces=True) for sc in scenes) <= budget_bytes
