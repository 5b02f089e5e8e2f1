"""FP64 CPU oracle of the probe-misfit gradient of the plain theta-method.

TEST INFRASTRUCTURE ONLY (same rule as oracle/theta.py): only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may import this module.

The paper integrates (Sec. 3.3.1, Eq. time_integration, no electrodes, K = 1)

    Z I^{k+1} = A I^k - M (s^{k+1} - s^k),   Z = L + theta dt R,  A = L - (1 - theta) dt R,

and this module differentiates the misfit of the probe outputs

    J = sum_{k=1..T} || C I^k - v^k ||^2

by the discrete adjoint of that recurrence (the paper has no gradient; this is the
"differentiation" use of its method for eddy-current inversion).  With the
Lagrangian J - sum_k lambda^{k+1 T} (Z I^{k+1} - A I^k + M (s^{k+1} - s^k)):

    Z lambda^k = A lambda^{k+1} + 2 C^T (C I^k - v^k),   k = T .. 1,  lambda^{T+1} = 0,
    dJ/dR_ee   = - dt sum_{k=1..T} lambda^k_e (theta I^k_e + (1 - theta) I^{k-1}_e),
    dJ/ds^j    = mu^{j+1} - mu^j,   mu^k = M^T lambda^k (mu^0 = mu^{T+1} = 0).

Plain definitions; no checkpointing (all states are kept).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


@dataclass
class MisfitGrad:
    J: float
    dJ_dRdiag: np.ndarray    # (N,)
    dJ_dsrc: np.ndarray      # (S, T+1)
    probes: np.ndarray       # (P, T)


def misfit_and_gradient(L, R, M, C, theta: float, dt: float, src, v, I0=None) -> MisfitGrad:
    L = np.asarray(L, np.float64)
    R = np.asarray(R, np.float64)
    N = L.shape[0]
    M = np.asarray(M, np.float64).reshape(N, -1)
    C = np.asarray(C, np.float64).reshape(-1, N)
    src = np.asarray(src, np.float64).reshape(M.shape[1], -1)
    T = src.shape[1] - 1
    v = np.asarray(v, np.float64).reshape(C.shape[0], T)
    Z = L + theta * dt * R
    A = L - (1.0 - theta) * dt * R
    cz = sla.cho_factor(Z, lower=True)
    I = np.zeros((N, T + 1))
    I[:, 0] = 0.0 if I0 is None else I0
    for k in range(T):
        I[:, k + 1] = sla.cho_solve(cz, A @ I[:, k] - M @ (src[:, k + 1] - src[:, k]))
    probes = C @ I[:, 1:]
    res = probes - v
    J = float(np.sum(res * res))
    lam_next = np.zeros(N)
    gR = np.zeros(N)
    mu = np.zeros((M.shape[1], T + 2))
    for k in range(T, 0, -1):
        lam = sla.cho_solve(cz, A @ lam_next + 2.0 * (C.T @ res[:, k - 1]))
        gR -= dt * lam * (theta * I[:, k] + (1.0 - theta) * I[:, k - 1])
        mu[:, k] = M.T @ lam
        lam_next = lam
    dsrc = mu[:, 1:] - mu[:, :-1]
    return MisfitGrad(J, gR, dsrc, probes)


def misfit(L, R, M, C, theta, dt, src, v, I0=None) -> float:
    """J alone (forward recurrence only), for finite-difference checks."""
    return misfit_and_gradient(L, R, M, C, theta, dt, src, v, I0).J


def hat_basis(T: int, n_knots: int) -> np.ndarray:
    """(n_knots, T+1) piecewise-linear hat functions on uniform knots over steps 0..T."""
    t = np.arange(T + 1, dtype=np.float64)
    knots = np.linspace(0.0, float(T), n_knots)
    h = knots[1] - knots[0]
    return np.maximum(0.0, 1.0 - np.abs(t[None, :] - knots[:, None]) / h)
