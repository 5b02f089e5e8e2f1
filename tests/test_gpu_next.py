"""GPU parity of the 'next' features: selective (truncated) modal integration,
multi-sine excitation with phasor extraction, and dt reuse of one modal setup."""
import numpy as np
import pytest

from oracle import phasor as ph
from oracle import theta as orc
from parity import rel_snaps, rel_traces
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


@pytest.mark.parametrize("keep", [1, 37, 200])
def test_truncated_modes_match_oracle(eddy, keep):
    p = synth.small(300, T=60, seed=6, electrodes=False, coil=True, snap_stride=20)
    red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    md = orc.modal_setup(red.Li, red.Ri)
    ref = orc.theta_modal(red, orc.Modes(md.tau[:keep], md.U[:, :keep]), p.theta, p.dt, p.src,
                          p.iD, p.T, None, p.snap_stride)
    tm = eddy.ThetaMethod("modal", p.theta, p.dt)
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    tm.set_mode_count(keep)
    probes, snaps = tm.run(p.T, p.src, None, p.snap_stride)
    assert rel_traces(probes, ref.probes) < TOL
    assert rel_snaps(snaps, ref.snaps) < TOL


def test_phasor_kernel_matches_oracle(eddy):
    rng = np.random.default_rng(0)
    y = rng.standard_normal((5, 3001))
    f = np.array(synth.MULTISINE_HZ)
    got = eddy.phasors(y, 0.25, 3.3e-5, f)
    ref = ph.phasors(y, 0.25, 3.3e-5, f)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)) * 10


def test_multisine_run_and_phasors(eddy):
    """Plate driven by the 30-tone multi-sine (Sec. 4.3) sampled at 30 kS/s (Sec. 4.6):
    GPU probes and their phasors against the oracle's."""
    p = synth.config1(T=900)
    p.dt = 1.0 / 30000.0
    p.src = synth.multisine(900, p.dt)[None, :]
    ref = orc.run_problem(p, "plain")
    tm = eddy.ThetaMethod("modal", p.theta, p.dt)
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    probes, _ = tm.run(p.T, p.src, None, 0)
    assert rel_traces(probes, ref.probes) < TOL
    f = np.array([100.0, 1000.0, 10000.0])
    Xg = eddy.phasors(probes[:, 300:], 301 * p.dt, p.dt, f)
    Xo = ph.phasors(ref.probes[:, 300:], 301 * p.dt, p.dt, f)
    assert np.max(np.abs(Xg - Xo)) <= 1e-9 * np.max(np.abs(Xo))


def test_steady_state_phasor_equals_frequency_domain_solve(eddy):
    """theta = 1/2, single tone, started on its discrete steady state: the probe phasor
    equals -i C X with X from the complex system (j w~ L + R) X = -j w~ M at the warped
    frequency w~ = (2/dt) tan(w dt / 2) (the frequency-domain method of Sec. 4.6)."""
    T, dt = 2000, 5e-6
    f = 1.0 / (200 * dt)                   # 200 samples per period, 10 periods
    p = synth.small(150, T=T, seed=9, electrodes=False, coil=True, dt=dt)
    w = 2 * np.pi * f
    wt = (2.0 / dt) * np.tan(w * dt / 2.0)
    X = np.linalg.solve(1j * wt * p.L + p.R, -1j * wt * p.M[:, 0])
    k = np.arange(T + 1)
    p.src = np.sin(w * dt * k)[None, :]
    tm = eddy.ThetaMethod("modal", 0.5, dt)
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    tm.set_current(np.imag(X))
    probes, _ = tm.run(T, p.src, None, 0)
    Xp = eddy.phasors(probes, dt, dt, [f])[0]
    assert np.allclose(Xp, -1j * (p.C @ X) * np.exp(0j), rtol=1e-8, atol=1e-8 * np.abs(p.C @ X).max())


def test_one_modal_setup_many_steps(eddy):
    """dt reuse (Sec. 5): one eigensolve, three step sizes, each matching the oracle."""
    p = synth.small(400, T=40, seed=10, electrodes=True, coil=True, snap_stride=10)
    tm = eddy.ThetaMethod("modal", p.theta, p.dt)
    tm.setup(p.L, p.R, p.E, p.M, p.MD, p.C)
    for dt in (1e-6, 4e-6, 2.5e-7):
        q = synth.small(400, T=40, seed=10, electrodes=True, coil=True, snap_stride=10, dt=dt)
        tm.set_current(np.zeros(400))
        tm.set_step(0.5, dt)
        probes, snaps = tm.run(q.T, q.src, q.iD, q.snap_stride)
        ref = orc.run_problem(q, "plain")
        assert rel_traces(probes, ref.probes) < TOL and rel_snaps(snaps, ref.snaps) < TOL
