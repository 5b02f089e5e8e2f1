"""FP64 CPU oracle of exact modal integration for piecewise-linear sources.

TEST INFRASTRUCTURE ONLY (same rule as oracle/theta.py).

Sec. 3.3 notes that once the system is decoupled into modes (Eq.
modal_decomposition_discrete), analytical solutions for polynomial inputs become
easy, and leaves them to future work.  With R_n = 1 and L_n = tau_n each mode obeys

    tau_n x_n' + x_n = e_n(t),   e(t) = U^T F(t),
    F(t) = -R_D i_D(t) - L_D di_D/dt - M_0 di_0/dt          (Eq. circuit_equations_v2)

and for sources sampled at t_k and linear in between, e_n over [t_k, t_k + dt] is
e0 + e1 s (s = (t - t_k)/dt) with

    e0 = U^T ( -R_D i_D^k - L_D (di_D / dt) - M_0 (di_0 / dt) ),   e1 = U^T ( -R_D di_D ).

The step is integrated exactly (h = dt / tau_n):

    x^{k+1} = e^{-h} x^k + (1 - e^{-h}) e0 + (1 - (1 - e^{-h}) / h) e1.
"""
from __future__ import annotations

import numpy as np

from . import theta as th


def exp_coefficients(tau, dt: float):
    """(a, c0, c1) of the exact step: a = e^{-h}, c0 = 1 - e^{-h}, c1 = 1 - (1 - e^{-h})/h.

    For h < 1, c1 (which cancels to h/2 as h -> 0) is summed from its Taylor series
    c1 = sum_{j>=1} (-1)^{j+1} h^j / (j+1)!  (20 terms: truncation below 1e-18 relative)."""
    h = dt / np.asarray(tau, np.float64)
    c0 = -np.expm1(-h)
    a = np.exp(-h)
    c1 = 1.0 - c0 / h
    small = h < 1.0
    if np.any(small):
        hs = h[small]
        term = hs / 2.0
        ser = term.copy()
        for j in range(2, 21):
            term = -term * hs / (j + 1)
            ser = ser + term
        c1 = np.where(small, 0.0, c1)
        c1[small] = ser
    return a, c0, c1


def modal_exponential(red: th.Reduced, modes: th.Modes, dt: float, src, iD, T: int, I0=None,
                      snap_stride: int = 0) -> th.Trajectory:
    src, iD, Ii0 = th._prepare(red, src, iD, T, I0)
    U = modes.U
    a, c0, c1 = exp_coefficients(modes.tau, dt)
    x = U.T @ (red.Ri @ Ii0)
    G = red.CK @ U
    P, N = G.shape[0], red.K.shape[0]
    m, S = red.PE.shape[1], red.M0.shape[1]
    nsnap = T // snap_stride if snap_stride else 0
    probes = np.zeros((P, T))
    snaps = np.zeros((N, nsnap))
    for k in range(T):
        F0 = np.zeros(red.Li.shape[0])
        F1 = np.zeros(red.Li.shape[0])
        if m:
            dD = iD[:, k + 1] - iD[:, k]
            F0 -= red.RD @ iD[:, k] + red.LD @ (dD / dt)
            F1 -= red.RD @ dD
        if S:
            F0 -= red.M0 @ ((src[:, k + 1] - src[:, k]) / dt)
        x = a * x + c0 * (U.T @ F0) + c1 * (U.T @ F1)
        probes[:, k] = G @ x + red.CPE @ iD[:, k + 1]
        if snap_stride and (k + 1) % snap_stride == 0:
            snaps[:, (k + 1) // snap_stride - 1] = red.K @ (U @ x) + red.PE @ iD[:, k + 1]
    I_final = red.K @ (U @ x) + red.PE @ iD[:, T]
    return th.Trajectory(probes, snaps, I_final)


def run_problem(p, I0=None, T: int | None = None):
    T = p.T if T is None else T
    red = th.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    modes = th.modal_setup(red.Li, red.Ri)
    return modal_exponential(red, modes, p.dt, p.src[:, : T + 1], p.iD[:, : T + 1], T, I0,
                             p.snap_stride)
