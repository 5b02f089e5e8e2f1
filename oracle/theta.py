"""FP64 CPU oracle of the theta-method for L dI/dt + R I = V(t) with electrode constraints.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The
product path (the CUDA library and its binding) never calls it.

Everything here is the plain, slow, readable definition of what the method
computes, written from arXiv 2407.11993 (Chiariello et al., "Modal
Decomposition in Numerical Computation of Eddy Current Transients"):

* Sec. 3.1, Eq. discrete_version_1a/b:  R I + L dI/dt + E^T phi = V_0 + V_D,  E I = i_D.
* Sec. 3.1, Eq. current_electrodes:    I = K I_i + E^T (E E^T)^{-1} i_D, K a basis of ker E.
* Sec. 3.1, Eq. discrete_version_2 and circuit_equations_v2: the projected system
  R_i I_i + L_i dI_i/dt = -R_D i_D - L_D di_D/dt - M_0 di_0/dt.
* Sec. 3.3.1, Eq. time_integration: the theta-step solved with a Cholesky factor.
* Sec. 3.2, Eq. generalized_eigenvalues_discrete / modal_decomposition_discrete and
  Sec. 3.3.2: the same theta-step in the basis of generalised eigenvectors.

Library primitives used as steps: numpy matmul, numpy.linalg.qr (basis of
ker E), numpy.linalg.cholesky, scipy.linalg.solve_triangular and
numpy.linalg.eigh (symmetric standard eigenproblem).  No blocking, fusion or
reordering beyond the equations.

Readings of the paper taken here (where it is silent, garbled or ambiguous):

1. The modal update of Sec. 3.3.2 prints the forcing without a Delta t factor and
   theta-weights sampled forcing values.  This oracle projects the Cholesky-form
   right-hand side of Eq. time_integration onto the modes instead, so the modal
   and Cholesky forms are the same theta-scheme in two bases.
2. L_D = L_ie (E E^T)^{-1} + M^D mixes an N_0-row and an N-row object; it is read
   as K^T L E^T (E E^T)^{-1} + K^T M^D.  Likewise the M_0 of Eq. time_integration
   is K^T M^0 (as V_{0,i} = K^T V_0).
3. K (unspecified in the paper) is the orthonormal basis of ker E given by a
   complete QR factorisation of E^T.  Outputs I and probe signals do not depend
   on that choice.
4. Eigenvectors are R_i-orthonormal (V^T R_i V = 1, so R_n = 1 and L_n = tau_n)
   and sorted by decreasing tau (Sec. 2.3, property 5).
5. Initial state I^0 = 0 unless given; sources are sampled at t_k = k dt,
   k = 0..T, and their increments delta x = x^{k+1} - x^k enter Eq. time_integration.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


@dataclass
class Reduced:
    """Quantities of Eq. discrete_version_2 / circuit_equations_v2 for one system."""
    K: np.ndarray      # (N, N0) orthonormal basis of ker E
    PE: np.ndarray     # (N, m)  E^T (E E^T)^{-1}   (particular field per unit i_D)
    Li: np.ndarray     # (N0, N0) K^T L K
    Ri: np.ndarray     # (N0, N0) K^T R K
    RD: np.ndarray     # (N0, m)  K^T R E^T (E E^T)^{-1}
    LD: np.ndarray     # (N0, m)  K^T L E^T (E E^T)^{-1} + K^T M^D
    M0: np.ndarray     # (N0, S)  K^T M^0
    CK: np.ndarray     # (P, N0)  C K
    CPE: np.ndarray    # (P, m)   C E^T (E E^T)^{-1}


def eliminate(L, R, E, M, MD, C) -> Reduced:
    """Constraint elimination, Sec. 3.1 (Eq. current_electrodes, discrete_version_2,
    circuit_equations_v2).  E has m = N_e - 1 rows (m = 0: no electrodes)."""
    L = np.asarray(L, np.float64)
    R = np.asarray(R, np.float64)
    N = L.shape[0]
    E = np.asarray(E, np.float64).reshape(-1, N)
    m = E.shape[0]
    if m == 0:
        K = np.eye(N)
        PE = np.zeros((N, 0))
    else:
        Q, _ = np.linalg.qr(E.T, mode="complete")
        K = Q[:, m:]
        PE = E.T @ np.linalg.inv(E @ E.T)
    M = np.asarray(M, np.float64).reshape(N, -1)
    MD = np.asarray(MD, np.float64).reshape(N, m) if m else np.zeros((N, 0))
    C = np.asarray(C, np.float64).reshape(-1, N)
    Li = K.T @ L @ K
    Ri = K.T @ R @ K
    RD = K.T @ R @ PE
    LD = K.T @ L @ PE + K.T @ MD
    return Reduced(K, PE, 0.5 * (Li + Li.T), 0.5 * (Ri + Ri.T), RD, LD, K.T @ M, C @ K, C @ PE)


@dataclass
class Trajectory:
    probes: np.ndarray    # (P, T): column k-1 holds y^k = C I^k, k = 1..T
    snaps: np.ndarray     # (N, T // stride): column j holds I^{(j+1) stride}
    I_final: np.ndarray   # (N,) I^T


def _source_terms(red: Reduced, src, iD, k, theta, dt):
    """Everything on the right of Eq. time_integration except -dt R_i I_i^k."""
    g = np.zeros(red.Li.shape[0])
    m = red.PE.shape[1]
    if m:
        dD = iD[:, k + 1] - iD[:, k]
        g -= dt * (red.RD @ iD[:, k])
        g -= (red.LD + dt * theta * red.RD) @ dD
    if red.M0.shape[1]:
        g -= red.M0 @ (src[:, k + 1] - src[:, k])
    return g


def _prepare(red: Reduced, src, iD, T, I0):
    N = red.K.shape[0]
    src = np.asarray(src, np.float64).reshape(red.M0.shape[1], T + 1)
    iD = np.asarray(iD, np.float64).reshape(red.PE.shape[1], T + 1)
    I0 = np.zeros(N) if I0 is None else np.asarray(I0, np.float64)
    Ii0 = red.K.T @ I0          # K^T PE = 0, so this is the internal part of I^0
    return src, iD, Ii0


def theta_plain(red: Reduced, theta: float, dt: float, src, iD, T: int,
                I0=None, snap_stride: int = 0) -> Trajectory:
    """Cholesky form of the theta-method, Sec. 3.3.1 (Eq. time_integration):
    Z = L_i + theta dt R_i = C C^T once; per step forward then backward substitution."""
    src, iD, Ii = _prepare(red, src, iD, T, I0)
    Z = red.Li + dt * theta * red.Ri
    Cz = np.linalg.cholesky(Z)
    P = red.CK.shape[0]
    N = red.K.shape[0]
    nsnap = T // snap_stride if snap_stride else 0
    probes = np.zeros((P, T))
    snaps = np.zeros((N, nsnap))
    for k in range(T):
        b = -dt * (red.Ri @ Ii) + _source_terms(red, src, iD, k, theta, dt)
        y = sla.solve_triangular(Cz, b, lower=True)
        dI = sla.solve_triangular(Cz.T, y, lower=False)
        Ii = Ii + dI
        probes[:, k] = red.CK @ Ii + red.CPE @ iD[:, k + 1]
        if snap_stride and (k + 1) % snap_stride == 0:
            snaps[:, (k + 1) // snap_stride - 1] = red.K @ Ii + red.PE @ iD[:, k + 1]
    I_final = red.K @ Ii + red.PE @ iD[:, T]
    return Trajectory(probes, snaps, I_final)


@dataclass
class Modes:
    tau: np.ndarray   # (N0,) decreasing
    U: np.ndarray     # (N0, N0) columns: R_i-orthonormal generalised eigenvectors


def modal_setup(Li, Ri) -> Modes:
    """Generalised eigenproblem L_i V = tau R_i V (Eq. generalized_eigenvalues_discrete),
    in the order of the standard reduction: R_i = C_R C_R^T, A = C_R^{-1} L_i C_R^{-T},
    A = Y diag(tau) Y^T, V = C_R^{-T} Y; sorted by decreasing tau."""
    CR = np.linalg.cholesky(Ri)
    W = sla.solve_triangular(CR, Li, lower=True)          # C_R^{-1} L_i
    A = sla.solve_triangular(CR, W.T, lower=True)         # C_R^{-1} (C_R^{-1} L_i)^T
    A = 0.5 * (A + A.T)
    w, Y = np.linalg.eigh(A)
    order = np.argsort(-w, kind="stable")
    w, Y = w[order], Y[:, order]
    U = sla.solve_triangular(CR.T, Y, lower=False)        # C_R^{-T} Y
    return Modes(w, U)


def modal_coefficients(tau, theta: float, dt: float):
    """Per-mode update x^{k+1} = a x^k + c beta^k of Sec. 3.3.2 with R_n = 1, L_n = tau_n:
    a = (tau - (1 - theta) dt) / (tau + theta dt),  c = 1 / (tau + theta dt)."""
    tau = np.asarray(tau, np.float64)
    return (tau - (1.0 - theta) * dt) / (tau + theta * dt), 1.0 / (tau + theta * dt)


def theta_modal(red: Reduced, modes: Modes, theta: float, dt: float, src, iD, T: int,
                I0=None, snap_stride: int = 0) -> Trajectory:
    """Modal form of the theta-method, Sec. 3.2 (Eq. modal_decomposition_discrete) and
    Sec. 3.3.2: I_i = U x, each mode advanced by its scalar theta-recurrence."""
    src, iD, Ii0 = _prepare(red, src, iD, T, I0)
    U = modes.U
    a, c = modal_coefficients(modes.tau, theta, dt)
    # x^0 = U^{-1} I_i^0 = U^T R_i I_i^0 (R_i-orthonormal modes)
    x = U.T @ (red.Ri @ Ii0)
    G = red.CK @ U
    P = G.shape[0]
    N = red.K.shape[0]
    nsnap = T // snap_stride if snap_stride else 0
    probes = np.zeros((P, T))
    snaps = np.zeros((N, nsnap))
    for k in range(T):
        beta = U.T @ _source_terms(red, src, iD, k, theta, dt)
        x = a * x + c * beta
        probes[:, k] = G @ x + red.CPE @ iD[:, k + 1]
        if snap_stride and (k + 1) % snap_stride == 0:
            snaps[:, (k + 1) // snap_stride - 1] = red.K @ (U @ x) + red.PE @ iD[:, k + 1]
    I_final = red.K @ (U @ x) + red.PE @ iD[:, T]
    return Trajectory(probes, snaps, I_final)


def magnetic_energy(L, I) -> float:
    """W = 1/2 I^T L I."""
    I = np.asarray(I, np.float64)
    return 0.5 * float(I @ (np.asarray(L) @ I))


def run_problem(p, form: str = "plain", I0=None, T: int | None = None):
    """Convenience: eliminate + integrate a ``workloads.synth.Problem``."""
    T = p.T if T is None else T
    red = eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    src = p.src[:, : T + 1]
    iD = p.iD[:, : T + 1]
    if form == "plain":
        return theta_plain(red, p.theta, p.dt, src, iD, T, I0, p.snap_stride)
    modes = modal_setup(red.Li, red.Ri)
    return theta_modal(red, modes, p.theta, p.dt, src, iD, T, I0, p.snap_stride)
