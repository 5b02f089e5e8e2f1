"""torch.autograd wrapper of the library's misfit gradient (ec_grad).

``ProbeMisfit.apply(r_diag, src, problem)`` returns J = sum_k ||C I^k - v^k||^2 of
a plain-form run whose resistance matrix is ``R_off + diag(r_diag)``; its backward
hands back dJ/dr_diag and dJ/dsrc, both computed by the library's adjoint
kernels.  Anything upstream (per-element resistivity -> r_diag, waveform knots ->
src samples) is ordinary torch autograd.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import eddy


@dataclass
class MisfitProblem:
    L: np.ndarray            # (N, N) inductance
    R_off: np.ndarray        # (N, N) resistance without its diagonal
    M: np.ndarray            # (N, S) coil mutuals
    C: np.ndarray            # (P, N) probe rows
    v: np.ndarray            # (P, T) target probe signals
    theta: float
    dt: float
    ckpt_every: int = 250
    device: int = 0


class ProbeMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r_diag: torch.Tensor, src: torch.Tensor, problem: MisfitProblem):
        R = problem.R_off + np.diag(r_diag.detach().cpu().numpy().astype(np.float64))
        T = problem.v.shape[1]
        tm = eddy.ThetaMethod("plain", problem.theta, problem.dt, device=problem.device)
        tm.setup(problem.L, R, None, problem.M, None, problem.C)
        J, gR, gs = tm.grad(T, src.detach().cpu().numpy().astype(np.float64), problem.v,
                            problem.ckpt_every)
        tm.close()
        ctx.save_for_backward(torch.from_numpy(gR), torch.from_numpy(gs))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        gR, gs = ctx.saved_tensors
        return gJ * gR, gJ * gs, None
