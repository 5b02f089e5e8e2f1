"""GPU adjoint (ec_grad) against the oracle's gradient and finite differences."""
import numpy as np
import pytest

from oracle import adjoint as adj
from workloads import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def eddy():
    from paper_2407_11993_gb300 import build, eddy as e
    build.build()
    return e


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def inversion_case(n, T, seed=0, dt=1e-6, noise=1e-2):
    """Targets from a run with a 3x3x2 block of elements at twice the resistivity, plus
    seeded measurement noise (noise x the probe signals' standard deviation).

    The misfit residual C I - v is a difference of two nearly equal signals; with
    noise = 0 it is ~1e-5 of the signal and the 1e-13 relative parity of the
    probes becomes ~1e-8 in J.  Realistic noise keeps the residual well
    conditioned so the gradient comparison tests the adjoint, not cancellation."""
    p = synth.small(n, T=T, seed=seed, electrodes=False, coil=True, probes=16, dt=dt)
    g2 = synth.geometry(n, seed)
    nx, ny, nz = g2.grid
    ijk = g2.ijk
    block = ((ijk[:, 0] >= nx // 2 - 1) & (ijk[:, 0] <= nx // 2 + 1) &
             (ijk[:, 1] >= ny // 2 - 1) & (ijk[:, 1] <= ny // 2 + 1) & (ijk[:, 2] <= 1))
    g2.rho = g2.rho.copy()
    g2.rho[block] *= 2.0
    Rt = synth.resistance(g2)
    v = adj.misfit_and_gradient(p.L, Rt, p.M, p.C, p.theta, p.dt, p.src,
                                np.zeros((p.C.shape[0], T))).probes
    rng = np.random.default_rng(seed + 1000)
    v = v + noise * np.std(v) * rng.standard_normal(v.shape)
    return p, v


def gpu_grad(eddy, p, v, T, ckpt, R=None, src=None):
    tm = eddy.ThetaMethod("plain", p.theta, p.dt)
    tm.setup(p.L, p.R if R is None else R, None, p.M, None, p.C)
    return tm.grad(T, p.src if src is None else src, v, ckpt)


@pytest.mark.parametrize("n,T,ckpt", [(512, 300, 50), (777, 120, 7), (130, 64, 64)])
def test_gradient_matches_oracle(eddy, n, T, ckpt):
    p, v = inversion_case(n, T)
    ref = adj.misfit_and_gradient(p.L, p.R, p.M, p.C, p.theta, p.dt, p.src, v)
    J, gR, gs = gpu_grad(eddy, p, v, T, ckpt)
    assert abs(J - ref.J) <= TOL * ref.J
    assert rel(gR, ref.dJ_dRdiag) < TOL
    assert rel(gs, ref.dJ_dsrc) < TOL


def test_checkpoint_interval_does_not_change_the_result(eddy):
    p, v = inversion_case(300, 90)
    outs = [gpu_grad(eddy, p, v, 90, ck) for ck in (1, 13, 90)]
    for J, gR, gs in outs[1:]:
        assert J == outs[0][0]
        assert np.array_equal(gR, outs[0][1]) and np.array_equal(gs, outs[0][2])


def test_gradient_matches_central_fd_on_gpu(eddy):
    p, v = inversion_case(256, 80)
    J, gR, gs = gpu_grad(eddy, p, v, 80, 20)
    for e in (5, 100, 250):
        h = 1e-3 * p.R[e, e]
        Rp = p.R.copy(); Rp[e, e] += h
        Rm = p.R.copy(); Rm[e, e] -= h
        fd = (gpu_grad(eddy, p, v, 80, 20, R=Rp)[0] - gpu_grad(eddy, p, v, 80, 20, R=Rm)[0]) / (2 * h)
        assert abs(fd - gR[e]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gR).max())


def test_autograd_resistivity_and_knots(eddy):
    import torch
    from paper_2407_11993_gb300.autograd import MisfitProblem, ProbeMisfit
    n, T, nk = 200, 60, 8
    p, v = inversion_case(n, T)
    g = p.geom
    lap_diag = np.diag(p.R) - g.rho * synth.G_FACTOR
    R_off = p.R - np.diag(np.diag(p.R))
    Phi = torch.from_numpy(adj.hat_basis(T, nk))
    rho = torch.tensor(g.rho, dtype=torch.float64, requires_grad=True)
    knots = torch.tensor(np.linspace(0.0, 1.0, nk), dtype=torch.float64, requires_grad=True)
    r_diag = rho * synth.G_FACTOR + torch.from_numpy(lap_diag)
    src = (knots @ Phi)[None, :]
    prob = MisfitProblem(p.L, R_off, p.M, p.C, v, p.theta, p.dt, ckpt_every=16)
    J = ProbeMisfit.apply(r_diag, src, prob)
    J.backward()
    ref = adj.misfit_and_gradient(p.L, p.R - np.diag(np.diag(p.R)) + np.diag(r_diag.detach().numpy()),
                                  p.M, p.C, p.theta, p.dt, src.detach().numpy(), v)
    assert abs(J.item() - ref.J) <= TOL * ref.J
    assert rel(rho.grad.numpy(), ref.dJ_dRdiag * synth.G_FACTOR) < TOL
    assert rel(knots.grad.numpy(), adj.hat_basis(T, nk) @ ref.dJ_dsrc[0]) < TOL


def test_tiny_misfit_within_cancellation_bound(eddy):
    """Noise-free targets: J is limited by the cancellation in C I - v.  The bound is
    |dJ| <= 2 ||r|| ||dp|| with ||dp|| <= 1e-13 ||p|| (probe parity of the plain form)."""
    p, v = inversion_case(512, 200, noise=0.0)
    ref = adj.misfit_and_gradient(p.L, p.R, p.M, p.C, p.theta, p.dt, p.src, v)
    J, gR, gs = gpu_grad(eddy, p, v, 200, 40)
    r = np.linalg.norm(ref.probes - v)
    bound = 2.0 * r * 1e-13 * np.linalg.norm(ref.probes)
    assert abs(J - ref.J) <= bound
    assert rel(gR, ref.dJ_dRdiag) < 1e-13 * np.linalg.norm(ref.probes) / r + TOL


def test_config5_shape_n4096(eddy):
    """N = 4096 (32x16x8 plate), 16 probes, checkpoints every 250 steps (first 500 steps)."""
    p, v = inversion_case(4096, 500)
    ref = adj.misfit_and_gradient(p.L, p.R, p.M, p.C, p.theta, p.dt, p.src, v)
    J, gR, gs = gpu_grad(eddy, p, v, 500, 250)
    assert abs(J - ref.J) <= TOL * ref.J
    assert rel(gR, ref.dJ_dRdiag) < TOL
    assert rel(gs, ref.dJ_dsrc) < TOL


def test_resistivity_gradient_fd_32_coordinates_h1e6(eddy):
    """Central differences of the GPU's own misfit, relative step h = 1e-6 (and 1e-4) in
    rho on 32 random coordinates, against the GPU adjoint gradient (dJ/drho_e =
    g dJ/dR_ee).  Same bars as the oracle's check: aggregate relative error over the 32
    coordinates 1e-2 at h = 1e-6 (FP64 rounding of the small misfit difference) and 1e-4
    at h = 1e-4."""
    n, T = 1024, 300
    p, v = inversion_case(n, T, seed=3)
    J, gR, _ = gpu_grad(eddy, p, v, T, 100)
    rho = p.geom.rho
    coords = np.random.default_rng(32).choice(n, size=32, replace=False)
    grad = synth.G_FACTOR * gR[coords]

    def misfit(R):
        tm = eddy.ThetaMethod("plain", p.theta, p.dt)
        tm.setup(p.L, R, None, p.M, None, p.C)
        probes, _ = tm.run(T, p.src, None, 0)
        tm.close()
        return float(np.sum((probes - v) ** 2))

    for hr, bar in ((1e-6, 1e-2), (1e-4, 1e-4)):
        f = []
        for e in coords:
            h = hr * rho[e]
            Rp = p.R.copy(); Rp[e, e] += h * synth.G_FACTOR
            Rm = p.R.copy(); Rm[e, e] -= h * synth.G_FACTOR
            f.append((misfit(Rp) - misfit(Rm)) / (2 * h))
        f = np.array(f)
        assert np.linalg.norm(f - grad) <= bar * np.linalg.norm(grad), hr
