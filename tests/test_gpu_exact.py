"""Exact per-mode integration (EC_INTEG_EXACT) on the GPU against its FP64 oracle."""
import numpy as np
import pytest

from oracle import exponential as ex
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


def run_exact(eddy, p):
    tm = eddy.ThetaMethod("modal", p.theta, p.dt, integrator="exact")
    m = p.E.shape[0]
    tm.setup(p.L, p.R, p.E if m else None, p.M if p.M.shape[1] else None, p.MD if m else None, p.C)
    return tm, tm.run(p.T, p.src if p.M.shape[1] else None, p.iD if m else None, p.snap_stride)


def test_config1_exact(eddy):
    p = synth.config1(T=500)
    ref = ex.run_problem(p)
    _, (probes, _) = run_exact(eddy, p)
    assert rel_traces(probes, ref.probes) < TOL


@pytest.mark.parametrize("n,T", [(65, 40), (300, 80), (700, 2500)])
def test_electrodes_and_coil_exact(eddy, n, T):
    p = synth.small(n, T=T, seed=n, electrodes=True, coil=True, snap_stride=20, dt=1e-6)
    ref = ex.run_problem(p)
    _, (probes, snaps) = run_exact(eddy, p)
    assert rel_traces(probes, ref.probes) < TOL
    assert rel_snaps(snaps, ref.snaps) < TOL


def test_exact_set_step(eddy):
    p = synth.small(200, T=50, seed=2, electrodes=True, coil=True, snap_stride=10, dt=1e-6)
    q = synth.small(200, T=50, seed=2, electrodes=True, coil=True, snap_stride=10, dt=7e-6)
    tm, _ = run_exact(eddy, p)
    tm.set_current(np.zeros(200))
    tm.set_step(0.5, q.dt)
    probes, snaps = tm.run(q.T, q.src, q.iD, q.snap_stride)
    ref = ex.run_problem(q)
    assert rel_traces(probes, ref.probes) < TOL and rel_snaps(snaps, ref.snaps) < TOL
