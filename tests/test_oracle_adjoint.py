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


def test_resistivity_gradient_fd_32_coordinates_h1e6():
    """The differentiation workload's check as specified: dJ/drho_e (R = diag(rho g) +
    Laplacian, so dJ/drho_e = g dJ/dR_ee) against central differences with a relative
    step h = 1e-6 on 32 random coordinates, targets from a 3x3x2 block at twice the
    resistivity plus seeded 1 % measurement noise.

    J is a small difference of nearly equal signals, so in FP64 the central difference
    at h = 1e-6 carries rounding noise of about 1e-3 of the gradient over these
    coordinates (a few per cent on the smallest ones): the bars are the aggregate
    relative error over the 32 coordinates, 1e-2 at h = 1e-6 and 1e-4 at h = 1e-4
    (measured 1.7e-3 and 1.8e-5).  A sign, factor or theta-weight slip in the adjoint
    (>= 30 % on affected coordinates) fails both."""
    n, T = 150, 150
    p = synth.small(n, T=T, seed=5, electrodes=False, coil=True, probes=16, dt=1e-6)
    g2 = synth.geometry(n, 5)
    nx, ny, nz = g2.grid
    ijk = g2.ijk
    block = ((ijk[:, 0] >= nx // 2 - 1) & (ijk[:, 0] <= nx // 2 + 1) &
             (ijk[:, 1] >= ny // 2 - 1) & (ijk[:, 1] <= ny // 2 + 1) & (ijk[:, 2] <= 1))
    rho_t = g2.rho.copy()
    rho_t[block] *= 2.0
    g2.rho = rho_t
    v = adj.misfit_and_gradient(p.L, synth.resistance(g2), p.M, p.C, p.theta, p.dt, p.src,
                                np.zeros((p.C.shape[0], T))).probes
    v = v + 1e-2 * np.std(v) * np.random.default_rng(1005).standard_normal(v.shape)
    g = adj.misfit_and_gradient(p.L, p.R, p.M, p.C, p.theta, p.dt, p.src, v)
    rho = p.geom.rho
    coords = np.random.default_rng(32).choice(n, size=32, replace=False)
    grad = synth.G_FACTOR * g.dJ_dRdiag[coords]

    def fd(e, hr):
        h = hr * rho[e]
        dR = h * synth.G_FACTOR
        Rp = p.R.copy(); Rp[e, e] += dR
        Rm = p.R.copy(); Rm[e, e] -= dR
        return (adj.misfit(p.L, Rp, p.M, p.C, p.theta, p.dt, p.src, v)
                - adj.misfit(p.L, Rm, p.M, p.C, p.theta, p.dt, p.src, v)) / (2 * h)

    for hr, bar in ((1e-6, 1e-2), (1e-4, 1e-4)):
        f = np.array([fd(e, hr) for e in coords])
        assert np.linalg.norm(f - grad) <= bar * np.linalg.norm(grad), hr
        assert np.all(np.sign(f) == np.sign(grad)) or hr == 1e-6
