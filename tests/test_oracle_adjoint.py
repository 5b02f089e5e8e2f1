"""Pins of the oracle's misfit gradient: central finite differences of J.

J is quadratic in the source samples, so the central difference is exact up to
rounding there; in R it is accurate to O(h^2).  A wrong sign, a dropped theta
weight or an off-by-one in the adjoint recursion fails these.
"""
import numpy as np
import pytest

from oracle import adjoint as adj
from workloads import synth


def _case(n=40, T=30, seed=3, theta=0.5):
    p = synth.small(n, T=T, seed=seed, electrodes=False, coil=True, dt=2e-6, theta=theta)
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((p.C.shape[0], T)) * 1e-9
    return p, v


@pytest.mark.parametrize("theta", [0.5, 1.0, 0.7])
def test_gradient_wrt_resistance_diagonal_matches_central_fd(theta):
    p, v = _case(theta=theta)
    g = adj.misfit_and_gradient(p.L, p.R, p.M, p.C, p.theta, p.dt, p.src, v)
    for e in (0, 7, 23, 39):
        h = 1e-3 * p.R[e, e]
        Rp = p.R.copy(); Rp[e, e] += h
        Rm = p.R.copy(); Rm[e, e] -= h
        fd = (adj.misfit(p.L, Rp, p.M, p.C, p.theta, p.dt, p.src, v)
              - adj.misfit(p.L, Rm, p.M, p.C, p.theta, p.dt, p.src, v)) / (2 * h)
        assert abs(fd - g.dJ_dRdiag[e]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g.dJ_dRdiag).max())


def test_gradient_wrt_source_samples_matches_central_fd():
    p, v = _case()
    g = adj.misfit_and_gradient(p.L, p.R, p.M, p.C, p.theta, p.dt, p.src, v)
    for j in (0, 1, 10, 29, 30):
        h = 1e-3
        sp = p.src.copy(); sp[0, j] += h
        sm = p.src.copy(); sm[0, j] -= h
        fd = (adj.misfit(p.L, p.R, p.M, p.C, p.theta, p.dt, sp, v)
              - adj.misfit(p.L, p.R, p.M, p.C, p.theta, p.dt, sm, v)) / (2 * h)
        assert abs(fd - g.dJ_dsrc[0, j]) <= 1e-7 * np.abs(g.dJ_dsrc).max()


def test_knot_gradient_by_chain_rule():
    """Coil waveform as 8 hat-function knots: dJ/dc = Phi dJ/ds (linear map)."""
    p, v = _case(T=28)
    Phi = adj.hat_basis(28, 8)
    c = np.random.default_rng(1).standard_normal(8)
    src = (c @ Phi)[None, :]
    g = adj.misfit_and_gradient(p.L, p.R, p.M, p.C, p.theta, p.dt, src, v)
    gc = Phi @ g.dJ_dsrc[0]
    for j in (0, 3, 7):
        h = 1e-3
        cp = c.copy(); cp[j] += h
        cm = c.copy(); cm[j] -= h
        fd = (adj.misfit(p.L, p.R, p.M, p.C, p.theta, p.dt, (cp @ Phi)[None, :], v)
              - adj.misfit(p.L, p.R, p.M, p.C, p.theta, p.dt, (cm @ Phi)[None, :], v)) / (2 * h)
        assert abs(fd - gc[j]) <= 1e-7 * np.abs(gc).max()


def test_forward_matches_theta_plain():
    """The adjoint module's forward recurrence is the plain theta-method of oracle/theta."""
    from oracle import theta as orc
    p, v = _case()
    g = adj.misfit_and_gradient(p.L, p.R, p.M, p.C, p.theta, p.dt, p.src, v)
    ref = orc.run_problem(p, "plain")
    assert np.allclose(g.probes, ref.probes, rtol=1e-12, atol=1e-14 * np.abs(ref.probes).max())
