"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form,
a textbook special case, an invariant stated in the paper, or a different
library algorithm (QZ, complex LU).  A plausible slip in the oracle (dropped
term, wrong sign or Delta t factor, transposed operand) fails at least one.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import theta as orc
from workloads import synth

EPS = np.finfo(np.float64).eps


def _one_mode(l, r):
    return orc.eliminate(np.array([[l]]), np.array([[r]]), np.zeros((0, 1)),
                         np.zeros((1, 0)), np.zeros((1, 0)), np.ones((1, 1)))


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.5, 1.0])
@pytest.mark.parametrize("form", ["plain", "modal"])
def test_single_mode_amplification(theta, form):
    """N = 1, no source: I^k = I^0 a^k with the theta-method amplification factor
    a = (1 - (1-theta) dt/tau) / (1 + theta dt/tau), tau = L/R (Sec. 3.3)."""
    l, r, dt, T = 2.0e-4, 3.0e-3, 1.0e-2, 60
    tau = l / r
    red = _one_mode(l, r)
    src = np.zeros((0, T + 1))
    iD = np.zeros((0, T + 1))
    if form == "plain":
        tr = orc.theta_plain(red, theta, dt, src, iD, T, I0=np.array([1.0]))
    else:
        tr = orc.theta_modal(red, orc.modal_setup(red.Li, red.Ri), theta, dt, src, iD, T,
                             I0=np.array([1.0]))
    # textbook special cases of the factor
    if theta == 0.0:
        a = 1.0 - dt / tau                      # explicit Euler
    elif theta == 1.0:
        a = 1.0 / (1.0 + dt / tau)              # implicit Euler
    elif theta == 0.5:
        a = (2 * tau - dt) / (2 * tau + dt)     # Crank-Nicolson
    else:
        a = (1 - (1 - theta) * dt / tau) / (1 + theta * dt / tau)
    k = np.arange(1, T + 1)
    expect = a ** k
    err = np.abs(tr.probes[0] - expect)
    assert np.all(err <= 8 * k * EPS * np.maximum(np.abs(expect), 1e-300) + 1e-300)


@pytest.mark.parametrize("theta,order", [(0.5, 2), (1.0, 1), (0.0, 1)])
def test_single_mode_converges_to_exponential(theta, order):
    """Closed form for N = 1: I(t) = I0 exp(-t/tau); the theta-method error at a fixed
    time shrinks like dt^2 (theta = 1/2) or dt (otherwise)."""
    l, r = 1.0e-3, 1.0
    tau = l / r
    t_end = 2.0e-3
    errs = []
    for T in (200, 400, 800):
        dt = t_end / T
        red = _one_mode(l, r)
        tr = orc.theta_plain(red, theta, dt, np.zeros((0, T + 1)), np.zeros((0, T + 1)), T,
                             I0=np.array([1.0]))
        errs.append(abs(tr.probes[0, -1] - np.exp(-t_end / tau)))
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    for q in ratios:
        assert abs(np.log2(q) - order) < 0.1, (errs, ratios)


def _random_spd_pair(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, n))
    return A @ A.T / n + 0.1 * np.eye(n), B @ B.T / n + 0.2 * np.eye(n)


@pytest.mark.parametrize("theta", [0.5, 0.75, 1.0])
def test_energy_nonincreasing_zero_source(theta):
    """1/2 I^T L I does not increase under zero source for theta >= 1/2
    (|a_n| <= 1 and L-orthogonal modes, Sec. 3.2), even for dt >> tau."""
    p = synth.small(48, T=40, seed=3, electrodes=True, coil=False, snap_stride=1)
    red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    rng = np.random.default_rng(1)
    I0 = red.K @ rng.standard_normal(red.K.shape[1])
    tau = orc.modal_setup(red.Li, red.Ri).tau
    for dt in (0.1 * tau.min(), 10.0 * tau.max()):
        tr = orc.theta_plain(red, theta, dt, np.zeros((0, 41)), np.zeros((1, 41)), 40, I0, 1)
        W = [orc.magnetic_energy(p.L, I0)] + [orc.magnetic_energy(p.L, tr.snaps[:, k])
                                              for k in range(40)]
        assert np.all(np.diff(W) <= 1e-12 * W[0]), (dt, W[:5])


def test_energy_grows_for_unstable_explicit_step():
    """The energy pin has teeth: explicit Euler with dt > 2 tau_min blows up."""
    p = synth.small(48, T=40, seed=3, electrodes=False, coil=False, snap_stride=1)
    red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    tau = orc.modal_setup(red.Li, red.Ri).tau
    dt = 3.0 * tau.min()
    I0 = np.random.default_rng(2).standard_normal(48)
    tr = orc.theta_plain(red, 0.0, dt, np.zeros((0, 41)), np.zeros((0, 41)), 40, I0, 1)
    assert orc.magnetic_energy(p.L, tr.snaps[:, -1]) > 10 * orc.magnetic_energy(p.L, I0)


def test_constraints_hold_every_step():
    """E I^k = i_D^k at every step (Eq. discrete_version_1b, current_electrodes)."""
    p = synth.small(64, T=60, seed=5, electrodes=True, coil=True, snap_stride=1)
    p.iD[0] = np.sin(np.arange(61) * 0.37) * 2.0 + 1.0
    for form in ("plain", "modal"):
        tr = orc.run_problem(p, form)
        lhs = p.E @ tr.snaps
        scale = np.abs(p.E) @ np.abs(tr.snaps)
        assert np.all(np.abs(lhs - p.iD[:, 1:]) <= 64 * EPS * scale), form


def test_eliminated_basis_properties():
    """K spans ker E and is orthonormal; E^T (E E^T)^{-1} reproduces unit electrode current."""
    p = synth.small(40, T=1, seed=7)
    red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    assert red.K.shape == (40, 39)
    assert np.linalg.norm(p.E @ red.K) < 1e-14 * np.linalg.norm(p.E)
    assert np.linalg.norm(red.K.T @ red.K - np.eye(39)) < 1e-13
    assert np.allclose(p.E @ red.PE, np.eye(1), atol=1e-14)
    assert np.linalg.matrix_rank(p.E) == 1   # N_e - 1 = 1 (Proposition dim H_D)


def test_eigen_invariants_and_qz():
    """L_i V = tau R_i V: residuals, R- and L-orthogonality, tau > 0 decreasing
    (Sec. 3.2, Sec. 2.3 properties 3-6), and tau against the QZ algorithm."""
    p = synth.small(60, T=1, seed=11)
    red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    md = orc.modal_setup(red.Li, red.Ri)
    n0 = red.Li.shape[0]
    U, tau = md.U, md.tau
    assert np.all(tau > 0) and np.all(np.diff(tau) <= 0)
    res = red.Li @ U - (red.Ri @ U) * tau
    assert np.linalg.norm(res) <= 50 * n0 * EPS * np.linalg.norm(red.Li) * np.linalg.norm(U)
    assert np.linalg.norm(U.T @ red.Ri @ U - np.eye(n0)) <= 50 * n0 * EPS
    LU = U.T @ red.Li @ U
    assert np.linalg.norm(LU - np.diag(tau)) <= 50 * n0 * EPS * tau.max()
    # QZ (generalised Schur, a different algorithm) on the same pencil
    w = sla.eig(red.Li, red.Ri, right=False)
    wq = np.sort(w.real)[::-1]
    assert np.max(np.abs(w.imag)) < 1e-10 * tau.max()
    assert np.allclose(wq, tau, rtol=1e-9, atol=1e-12 * tau.max())


def test_two_by_two_closed_form():
    """For N0 = 2, tau solves det(L - tau R) = 0, a quadratic."""
    L = np.array([[3.0, 1.2], [1.2, 2.0]])
    R = np.array([[2.0, -0.5], [-0.5, 1.5]])
    a = R[0, 0] * R[1, 1] - R[0, 1] ** 2
    b = -(L[0, 0] * R[1, 1] + L[1, 1] * R[0, 0] - 2 * L[0, 1] * R[0, 1])
    c = L[0, 0] * L[1, 1] - L[0, 1] ** 2
    disc = np.sqrt(b * b - 4 * a * c)
    roots = np.array([(-b + disc) / (2 * a), (-b - disc) / (2 * a)])
    md = orc.modal_setup(L, R)
    assert np.allclose(md.tau, roots, rtol=1e-14)


def test_resistance_scaling_rescales_tau():
    """R -> k R: tau -> tau / k with the same eigenvectors (Sec. 3.2)."""
    p = synth.small(50, T=1, seed=13, electrodes=False)
    md1 = orc.modal_setup(p.L, p.R)
    k = 3.7
    md2 = orc.modal_setup(p.L, k * p.R)
    assert np.allclose(md2.tau, md1.tau / k, rtol=1e-11)
    # R_i-normalised vectors scale by 1/sqrt(k); compare up to sign
    cos = np.abs(np.sum(md1.U * md2.U, axis=0)) / (np.linalg.norm(md1.U, axis=0) * np.linalg.norm(md2.U, axis=0))
    assert np.all(cos > 1 - 1e-9)


def test_monotonicity_in_resistivity():
    """eta_1 <= eta_2 implies tau_n(eta_1) >= tau_n(eta_2) for every n (Sec. 2.3, property 8;
    holds in the discrete setting, Sec. 3.2)."""
    g = synth.geometry(64, seed=17)
    L = synth.inductance(g)
    R1 = synth.resistance(g)
    g2 = synth.geometry(64, seed=17)
    g2.rho = g2.rho.copy()
    g2.rho[10:30] *= 2.0          # a block of elements at twice the resistivity
    R2 = synth.resistance(g2)
    t1 = orc.modal_setup(L, R1).tau
    t2 = orc.modal_setup(L, R2).tau
    assert np.all(t2 <= t1 * (1 + 1e-12))
    assert np.any(t2 < t1 * (1 - 1e-6))


def test_plain_and_modal_agree():
    """The modal form is the same theta-scheme in the eigenvector basis (Sec. 3.2-3.3)."""
    p = synth.small(72, T=150, seed=19, electrodes=True, coil=True, snap_stride=10)
    a = orc.run_problem(p, "plain")
    b = orc.run_problem(p, "modal")
    assert np.linalg.norm(a.probes - b.probes) <= 1e-11 * np.linalg.norm(a.probes)
    assert np.linalg.norm(a.snaps - b.snaps) <= 1e-11 * np.linalg.norm(a.snaps)


@pytest.mark.parametrize("form", ["plain", "modal"])
@pytest.mark.parametrize("electrodes", [False, True])
def test_trapezoid_matches_warped_phasor(form, electrodes):
    """theta = 1/2 with sinusoidal coil and electrode currents: the discrete trajectory is
    Im(X z^k), z = exp(j w dt), where X solves the frequency-domain saddle-point system
    [(j w~ L + R)  E^T; E 0] [X; Phi] = [-j w~ (M sigma + M^D d); d] at the warped
    frequency w~ = (2/dt) tan(w dt / 2) (the FD view of Sec. 4.6, solved by complex LU)."""
    T = 80
    p = synth.small(40, T=T, seed=23, electrodes=electrodes, coil=True, snap_stride=1, dt=2e-6)
    n = p.n
    w = 2 * np.pi * 7.3e3
    z = np.exp(1j * w * p.dt)
    wt = (2.0 / p.dt) * np.tan(w * p.dt / 2.0)
    sigma = 1.0 * np.exp(0.4j)
    d = (0.8 * np.exp(-1.1j)) if electrodes else 0.0
    m = p.E.shape[0]
    A = np.zeros((n + m, n + m), dtype=complex)
    A[:n, :n] = 1j * wt * p.L + p.R
    rhs = np.zeros(n + m, dtype=complex)
    rhs[:n] = -1j * wt * (p.M[:, 0] * sigma)
    if m:
        A[:n, n:] = p.E.T
        A[n:, :n] = p.E
        rhs[:n] += -1j * wt * (p.MD[:, 0] * d)
        rhs[n:] = d
    X = np.linalg.solve(A, rhs)[:n]
    k = np.arange(T + 1)
    p.src = np.imag(sigma * z ** k)[None, :]
    if m:
        p.iD = np.imag(d * z ** k)[None, :]
    tr = orc.run_problem(p, form, I0=np.imag(X))
    expect = np.imag(X[:, None] * z ** k[None, 1:])
    assert np.linalg.norm(tr.snaps - expect) <= 1e-11 * np.linalg.norm(expect)
    assert np.allclose(tr.probes, p.C @ expect, rtol=0, atol=1e-11 * np.abs(p.C @ expect).max())


def test_superposition_of_sources():
    """Linearity: coil-only plus electrode-only runs sum to the combined run."""
    p = synth.small(36, T=50, seed=29, electrodes=True, coil=True, snap_stride=5)
    both = orc.run_problem(p, "plain")
    q = synth.small(36, T=50, seed=29, electrodes=True, coil=True, snap_stride=5)
    q.iD[:] = 0.0
    coil = orc.run_problem(q, "plain")
    r = synth.small(36, T=50, seed=29, electrodes=True, coil=True, snap_stride=5)
    r.src[:] = 0.0
    elec = orc.run_problem(r, "plain")
    assert np.allclose(both.probes, coil.probes + elec.probes, rtol=1e-12,
                       atol=1e-13 * np.abs(both.probes).max())


def test_workload_matrices_are_spd():
    """The synthetic L and R are symmetric positive definite (Sec. 3.1 assumption)."""
    p = synth.config1(T=2)
    assert np.array_equal(p.L, p.L.T) and np.array_equal(p.R, p.R.T)
    assert np.linalg.eigvalsh(p.L).min() > 0
    assert np.linalg.eigvalsh(p.R).min() > 0
    # graph-Laplacian part has zero row sums
    lap = p.R - np.diag(np.diag(p.R))
    assert np.allclose(lap.sum(axis=1) + (np.diag(p.R) - p.geom.rho * synth.G_FACTOR), 0.0,
                       atol=1e-18)


def test_truncated_modes_error_is_the_dropped_modes_energy():
    """Selective integration (Sec. 2.3: modes can be advanced 'in a selective manner'):
    keeping the k slowest modes of a zero-source run gives the R_i-orthogonal projection
    of the full trajectory, so ||I_full - I_k||_R^2 = sum over dropped modes of
    (a_n^s x_n^0)^2 exactly (modes are R-orthonormal, Sec. 3.2)."""
    p = synth.small(45, T=12, seed=31, electrodes=False, coil=False, snap_stride=1, dt=2e-4)
    red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    md = orc.modal_setup(red.Li, red.Ri)
    I0 = np.random.default_rng(4).standard_normal(45)
    full = orc.theta_modal(red, md, p.theta, p.dt, p.src, p.iD, 12, I0, 1)
    k = 20
    trunc = orc.theta_modal(red, orc.Modes(md.tau[:k], md.U[:, :k]), p.theta, p.dt, p.src, p.iD,
                            12, I0, 1)
    a, _ = orc.modal_coefficients(md.tau, p.theta, p.dt)
    x0 = md.U.T @ (p.R @ I0)
    for s in (1, 5, 12):
        d = full.snaps[:, s - 1] - trunc.snaps[:, s - 1]
        e2 = float(d @ p.R @ d)
        expect = float(np.sum((a[k:] ** s * x0[k:]) ** 2))
        assert abs(e2 - expect) <= 1e-10 * expect
