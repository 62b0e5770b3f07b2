"""Inverse-design loop driving the forward and time-reversal gradient solves (arXiv 2412.12360
Sec. 3.2-3.3: designs optimised by gradient steps, quantised to two materials).

    loop = DesignLoop(solver, theta0, eps_lo, eps_hi, nsteps, objective, lr=0.02,
                      beta_of=lambda it: 0.0 if it < 10 else 8.0)
    losses = loop.run(iters)

Densities rho = P_beta(theta) of latent variables theta in [0, 1] (smoothed Heaviside projection,
which binarises rho as beta grows), eps = eps_lo + (eps_hi - eps_lo) rho on the solver's design box,
Adam on theta. Per iteration: projection, density map, forward with the face record, the user's
objective of the detector outputs, the reverse sweep for dL/drho, the Adam step. The projection, the
density map, both solves and the Adam step run in the CUDA library; `objective` is the user's loss
(torch on the device, like any loss put through the autograd Function).
"""
from __future__ import annotations

from typing import Callable, List, Tuple

import torch

from . import fdtd


class DesignLoop:
    def __init__(self, solver: "fdtd.Solver", theta0: torch.Tensor, eps_lo: float, eps_hi: float, nsteps: int,
                 objective: Callable[[torch.Tensor], Tuple[torch.Tensor, torch.Tensor]], lr: float = 0.02,
                 beta_of: Callable[[int], float] = lambda it: 0.0, proj_eta: float = 0.5, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8):
        if not theta0.is_cuda or theta0.dtype != torch.float32:
            raise TypeError("theta0 must be a CUDA float32 tensor of the design-box shape")
        self.s = solver
        self.theta = theta0.detach().clone().contiguous()
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.rho = torch.empty_like(self.theta)
        self.g_rho = torch.empty_like(self.theta)
        self.det = torch.empty(0, dtype=torch.float64, device=self.theta.device)
        self.eps_lo, self.eps_hi = float(eps_lo), float(eps_hi)
        self.nsteps = int(nsteps)
        self.objective = objective
        self.lr = float(lr)
        self.beta_of = beta_of
        self.eta = float(proj_eta)
        self.b1, self.b2, self.eps = float(beta1), float(beta2), float(eps)
        self.t = 0

    def step(self) -> torch.Tensor:
        """One design iteration; returns the loss (a device scalar) at the densities it started from."""
        s = self.s
        beta = float(self.beta_of(self.t))
        s.fdtd_design_project(self.theta, self.rho, beta, self.eta)
        s.fdtd_set_design_density(self.rho, self.eps_lo, self.eps_hi)
        s.fdtd_forward(self.nsteps, record_faces=True)
        n = s.fdtd_detector_total()
        if self.det.numel() != n:
            self.det = torch.empty(n, dtype=torch.float64, device=self.theta.device)
        st = s.stream if isinstance(s.stream, torch.cuda.Stream) else None
        with torch.cuda.stream(st):
            s.fdtd_read_detectors(self.det)
            loss, dL_ddet = self.objective(self.det)
            dL_ddet = dL_ddet.detach().to(torch.float64).contiguous()
        s.fdtd_backward_density(dL_ddet, self.g_rho)
        self.t += 1
        s.fdtd_design_adam_step(self.g_rho, self.theta, self.m, self.v, self.rho, self.t, self.lr, self.b1, self.b2,
                                self.eps, beta, self.eta)
        return loss.detach()

    def run(self, iters: int) -> List[float]:
        losses = [self.step() for _ in range(iters)]
        self.s.fdtd_synchronize()
        return [float(x) for x in losses]
