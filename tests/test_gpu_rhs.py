"""Independent right-hand sides (batched coil excitations) against per-coil oracle runs."""
import numpy as np
import pytest

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


def per_coil_oracle(p, r):
    red = orc.eliminate(p.L, p.R, p.E, p.M[:, r:r + 1], p.MD, p.C)
    return orc.theta_plain(red, p.theta, p.dt, p.src[r:r + 1], p.iD, p.T, None, p.snap_stride)


@pytest.mark.parametrize("form", ["plain", "modal"])
def test_independent_coils_with_probe_grid(eddy, form):
    p = synth.coil_scan(200, T=30, n_side=2, probes=3)
    p.src = p.src * np.array([1.0, -0.5, 2.0, 0.25])[:, None]
    p.snap_stride = 10
    tm = eddy.ThetaMethod(form, p.theta, p.dt, rhs="independent")
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    probes, snaps = tm.run(p.T, p.src, None, p.snap_stride)
    assert probes.shape == (4, p.C.shape[0], p.T) and snaps.shape == (4, 200, 3)
    for r in range(4):
        ref = per_coil_oracle(p, r)
        assert rel_traces(probes[r], ref.probes) < TOL, r
        assert rel_snaps(snaps[r], ref.snaps) < TOL, r


@pytest.mark.parametrize("form", ["plain", "modal"])
@pytest.mark.parametrize("side", [3, 9])
def test_paired_self_pickup(eddy, form, side):
    """Config 3 read-out: trajectory r is read by its own coil (C = M^T); 81 coils is
    past the 64 probe rows of the summed mode (paired read-out has no such limit)."""
    p = synth.coil_scan(256, T=25, n_side=side)
    S = side * side
    tm = eddy.ThetaMethod(form, p.theta, p.dt, rhs="paired")
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    probes, _ = tm.run(p.T, p.src, None, 0)
    assert probes.shape == (S, 1, p.T)
    for r in sorted({0, S // 2, S - 1}):
        ref = per_coil_oracle(p, r)
        assert rel_traces(probes[r, 0], ref.probes[r]) < TOL, r


def test_independent_modal_long_run(eddy):
    p = synth.coil_scan(300, T=2600, n_side=2, probes=2, dt=2e-7)
    tm = eddy.ThetaMethod("modal", p.theta, p.dt, rhs="independent")
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    probes, _ = tm.run(p.T, p.src, None, 0)
    for r in (0, 3):
        ref = per_coil_oracle(p, r)
        assert rel_traces(probes[r], ref.probes) < TOL


def test_rhs_modes_reject_electrodes(eddy):
    p = synth.small(100, T=2, seed=1, electrodes=True, coil=True)
    tm = eddy.ThetaMethod("modal", p.theta, p.dt, rhs="independent")
    with pytest.raises(eddy.EcError) as e:
        tm.setup(p.L, p.R, p.E, p.M, p.MD, p.C)
    assert e.value.code == 10
