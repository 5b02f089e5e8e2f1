"""Pins of the exact (exponential) modal integrator for piecewise-linear sources."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import exponential as ex
from oracle import theta as orc
from workloads import synth


def test_single_mode_linear_ramp_closed_form():
    """tau x' + x = e0 + e1 t/dt on one step, x(0) = x0: closed form of the linear ODE,
    evaluated independently with a fine-grained matrix exponential of the augmented
    system [x; e(t)] (scipy.linalg.expm)."""
    tau, dt, x0, e0, e1 = 2.0e-3, 5.0e-4, 0.7, -1.3, 2.1
    a, c0, c1 = ex.exp_coefficients(np.array([tau]), dt)
    x1 = a[0] * x0 + c0[0] * e0 + c1[0] * e1
    # augmented linear system y' = A y with y = [x, e(t), 1], e' = e1/dt
    A = np.array([[-1 / tau, 1 / tau, 0.0], [0.0, 0.0, e1 / dt], [0.0, 0.0, 0.0]])
    y = sla.expm(A * dt) @ np.array([x0, e0, 1.0])
    assert abs(x1 - y[0]) <= 1e-14 * abs(y[0]) + 1e-16


@pytest.mark.parametrize("h", [1e-9, 1e-6, 1e-3, 0.05, 0.7, 0.999, 1.001, 5.0, 60.0])
def test_coefficients_against_50_digit_arithmetic(h):
    """a, c0, c1 against their definitions evaluated in 50-digit arithmetic (mpmath),
    across the switch between series and direct formula."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    H = mp.mpf(h)
    a_ref = mp.e ** (-H)
    c0_ref = 1 - a_ref
    c1_ref = 1 - c0_ref / H
    a, c0, c1 = ex.exp_coefficients(np.array([1.0]), h)
    for got, ref in ((a[0], a_ref), (c0[0], c0_ref), (c1[0], c1_ref)):
        assert abs(got - float(ref)) <= 4e-16 * abs(float(ref)) + 1e-300


def test_exact_for_piecewise_linear_sources_under_step_refinement():
    """The integrator is exact for sources linear between samples: halving dt with the
    interpolated samples gives the same states at the common times (to round-off)."""
    p = synth.small(40, T=20, seed=3, electrodes=True, coil=True, snap_stride=1, dt=4e-6)
    q = synth.small(40, T=40, seed=3, electrodes=True, coil=True, snap_stride=2, dt=2e-6)
    # q's samples: p's samples at even steps, midpoints (linear interpolation) at odd steps
    q.src = np.zeros((1, 41))
    q.src[:, ::2] = p.src
    q.src[:, 1::2] = 0.5 * (p.src[:, :-1] + p.src[:, 1:])
    q.iD = np.zeros((1, 41))
    q.iD[:, ::2] = p.iD
    q.iD[:, 1::2] = 0.5 * (p.iD[:, :-1] + p.iD[:, 1:])
    a = ex.run_problem(p)
    b = ex.run_problem(q)
    assert np.linalg.norm(a.snaps - b.snaps) <= 1e-11 * np.linalg.norm(a.snaps)


def test_agrees_with_theta_method_as_dt_shrinks():
    """Both integrate the same ODE: the theta = 1/2 trajectory approaches the exact one
    at second order in dt."""
    errs = []
    for T in (50, 100, 200):
        p = synth.small(30, T=T, seed=5, electrodes=True, coil=True, dt=2e-4 / T, f_hz=2e3)
        e = ex.run_problem(p).I_final
        t = orc.run_problem(p, "modal").I_final
        errs.append(np.linalg.norm(e - t) / np.linalg.norm(e))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


def test_zero_source_is_pure_exponential_decay():
    p = synth.small(25, T=30, seed=8, electrodes=False, coil=False, snap_stride=1, dt=1e-3)
    red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    md = orc.modal_setup(red.Li, red.Ri)
    I0 = np.random.default_rng(0).standard_normal(25)
    tr = ex.modal_exponential(red, md, p.dt, p.src, p.iD, 30, I0, 1)
    # exact: I(t) = U exp(-t/tau) U^T R I0
    x0 = md.U.T @ (p.R @ I0)
    for k in (1, 10, 30):
        Ik = md.U @ (np.exp(-k * p.dt / md.tau) * x0)
        assert np.allclose(tr.snaps[:, k - 1], Ik, rtol=1e-10, atol=1e-12 * np.abs(Ik).max())
