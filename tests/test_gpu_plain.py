"""Plain (Cholesky) form on the GPU against the FP64 oracle (Sec. 3.3.1).

Tolerance: 1e-10 relative in the 2-norm per output (the FP64 bar); the
oracle's own plain and modal forms agree to ~1e-15 on these inputs, so any
larger gap is a kernel error, not conditioning.
"""
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
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


SOLVERS = ["inverse", "substitution"]


def run_gpu(eddy, p, form="plain", T=None, I0=None, solver="inverse"):
    T = p.T if T is None else T
    tm = eddy.ThetaMethod(form, p.theta, p.dt, solver=solver)
    tm.setup(p.L, p.R, p.E if p.E.shape[0] else None, p.M if p.M.shape[1] else None,
             p.MD if p.E.shape[0] else None, p.C)
    if I0 is not None:
        tm.set_current(I0)
    probes, snaps = tm.run(T, p.src[:, :T + 1] if p.M.shape[1] else None,
                           p.iD[:, :T + 1] if p.E.shape[0] else None, p.snap_stride)
    return tm, probes, snaps


@pytest.mark.parametrize("solver", SOLVERS)
def test_config1_coil_n512(eddy, solver):
    p = synth.config1()
    ref = orc.run_problem(p, "plain")
    _, probes, _ = run_gpu(eddy, p, solver=solver)
    assert probes.shape == ref.probes.shape
    assert rel_traces(probes, ref.probes) < TOL


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 200, 517, 1100])
def test_ragged_sizes_with_electrode_and_coil(eddy, n, solver):
    electrodes = n >= 4
    p = synth.small(n, T=40, seed=n, electrodes=electrodes, coil=True, snap_stride=7)
    ref = orc.run_problem(p, "plain")
    _, probes, snaps = run_gpu(eddy, p, solver=solver)
    assert rel_traces(probes, ref.probes) < TOL
    assert rel_snaps(snaps, ref.snaps) < TOL


def test_two_electrode_rows(eddy):
    p = synth.small(150, T=30, seed=4, electrodes=True, coil=True, snap_stride=5)
    rng = np.random.default_rng(0)
    E2 = np.zeros((2, 150))
    E2[0] = p.E[0]
    face = p.geom.ijk[:, 0] == p.geom.grid[0] - 1
    E2[1, face] = np.cos(p.geom.phi[face])
    p.E = E2
    p.MD = np.concatenate([p.MD, 0.5 * p.MD], axis=1)
    p.iD = np.stack([p.iD[0], 0.3 * np.sin(np.arange(31) * 0.2)])
    ref = orc.run_problem(p, "plain")
    _, probes, snaps = run_gpu(eddy, p)
    assert rel_traces(probes, ref.probes) < TOL
    assert rel_snaps(snaps, ref.snaps) < TOL
    # constraint E I = i_D holds on the GPU snapshots
    assert np.allclose(p.E @ snaps, p.iD[:, 5::5], atol=1e-12)


def test_initial_current_and_zero_source_decay(eddy):
    p = synth.small(96, T=25, seed=8, electrodes=False, coil=False, snap_stride=1)
    I0 = np.random.default_rng(3).standard_normal(96)
    ref = orc.run_problem(p, "plain", I0=I0)
    _, probes, snaps = run_gpu(eddy, p, I0=I0)
    assert rel_snaps(snaps, ref.snaps) < TOL
    W = [orc.magnetic_energy(p.L, snaps[:, k]) for k in range(25)]
    assert np.all(np.diff(W) <= 1e-12 * W[0])


@pytest.mark.parametrize("solver", SOLVERS)
def test_resume_is_bitwise(eddy, solver):
    p = synth.small(130, T=60, seed=9, electrodes=True, coil=True)
    tm, full, _ = run_gpu(eddy, p, solver=solver)
    state_full = tm.get_state()
    tm2 = eddy.ThetaMethod("plain", p.theta, p.dt, solver=solver)
    tm2.setup(p.L, p.R, p.E, p.M, p.MD, p.C)
    a, _ = tm2.run(25, p.src[:, :26], p.iD[:, :26])
    st = tm2.get_state()
    tm3 = eddy.ThetaMethod("plain", p.theta, p.dt, solver=solver)
    tm3.setup(p.L, p.R, p.E, p.M, p.MD, p.C)
    tm3.set_state(st)
    b, _ = tm3.run(35, p.src[:, 25:], p.iD[:, 25:])
    assert np.array_equal(np.concatenate([a, b], axis=1), full)
    assert np.array_equal(tm3.get_state(), state_full)


def test_not_spd_is_reported(eddy):
    p = synth.small(80, T=2, seed=1, electrodes=False, coil=True)
    L = p.L.copy()
    L[37, 37] = -1.0
    tm = eddy.ThetaMethod("plain", 0.5, p.dt)
    with pytest.raises(eddy.EcError) as e:
        tm.setup(L, p.R, None, p.M, None, p.C)
    assert e.value.code == 3
    assert 0 <= e.value.info <= 37


def test_bounded_wait_times_out(eddy):
    assert eddy.selftest_wait_timeout(2000) == 7   # EC_ERR_TIMEOUT


@pytest.fixture(scope="module")
def config2_ref():
    p = synth.config2(T=40, snap_stride=20)
    return p, orc.run_problem(p, "plain")


@pytest.mark.parametrize("solver", SOLVERS)
def test_config2_electrodes_n8192_first_steps(eddy, config2_ref, solver):
    """N = 8192 with the electrode step, 16 pickups: first 40 steps + snapshots."""
    p, ref = config2_ref
    _, probes, snaps = run_gpu(eddy, p, solver=solver)
    assert rel_traces(probes, ref.probes) < TOL
    assert rel_snaps(snaps, ref.snaps) < TOL


def test_solvers_agree_and_set_step_refactors(eddy):
    """Both solve paths give the same trajectory; set_step re-forms and re-factors Z."""
    p = synth.small(300, T=30, seed=21, electrodes=True, coil=True, snap_stride=10)
    q = synth.small(300, T=30, seed=21, electrodes=True, coil=True, snap_stride=10, dt=4e-6,
                    theta=1.0)
    ref = orc.run_problem(q, "plain")
    outs = []
    for solver in SOLVERS:
        tm = eddy.ThetaMethod("plain", p.theta, p.dt, solver=solver)
        tm.setup(p.L, p.R, p.E, p.M, p.MD, p.C)
        tm.set_step(q.theta, q.dt)
        probes, snaps = tm.run(q.T, q.src, q.iD, q.snap_stride)
        assert rel_traces(probes, ref.probes) < TOL and rel_snaps(snaps, ref.snaps) < TOL
        outs.append(probes)
    assert rel_traces(outs[0], outs[1]) < TOL


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("n", [700, 1029])
def test_solve_z_matches_dense_solve(eddy, solver, n):
    """x = Z^{-1} b with Z = L + theta dt R (no electrodes: the internal basis is the identity)."""
    p = synth.small(n, T=1, seed=31, electrodes=False, coil=True)
    tm = eddy.ThetaMethod("plain", p.theta, p.dt, solver=solver)
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    b = np.random.default_rng(5).standard_normal(n)
    x = tm.solve_z(b)
    Z = p.L + p.dt * p.theta * p.R
    x_ref = np.linalg.solve(Z, b)
    assert rel(x, x_ref) < TOL


def test_inverse_factor_export(eddy):
    p = synth.small(300, T=1, seed=32, electrodes=False, coil=True)
    tm = eddy.ThetaMethod("plain", p.theta, p.dt)
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    Wt = tm.inverse_factor()          # row-major view of the column-major C^{-1}
    W = Wt.T
    assert np.allclose(np.triu(W, 1), 0.0)
    Z = p.L + p.dt * p.theta * p.R
    assert rel(W.T @ W, np.linalg.inv(Z)) < 1e-10


def test_tile_launch_shapes_are_bitwise_identical(eddy):
    """Every launch shape of the packed-tile products (and the autotuned one) sums each
    output in the same order: solves and trajectories agree to the last bit.  n = 6300
    spans 99 tile rows with a ragged 28-row tail, so units hold two tiles each."""
    p = synth.small(6300, T=4, seed=33, electrodes=False, coil=True)
    b = np.random.default_rng(6).standard_normal(p.L.shape[0])
    Z = p.L + p.dt * p.theta * p.R
    x_ref = np.linalg.solve(Z, b)
    xs, probes = [], []
    for v in range(4):
        tm = eddy.ThetaMethod("plain", p.theta, p.dt, tile_variant=v)
        tm.setup(p.L, p.R, None, p.M, None, p.C)
        xs.append(tm.solve_z(b))
        probes.append(tm.run(p.T, p.src, None, 0)[0])
        tm.close()
    assert rel(xs[0], x_ref) < TOL
    for v in range(1, 4):
        assert np.array_equal(xs[v], xs[0])
        assert np.array_equal(probes[v], probes[0])


@pytest.mark.parametrize("form", ["plain", "modal"])
def test_release_inputs_after_setup(eddy, form):
    """release_inputs frees the dense copies of L, R (and Z) that stepping does not read:
    the run is unchanged; the plain form then refuses a new dt (EC_ERR_STATE), the modal
    form still takes one (its per-mode coefficients only) and still sets a current."""
    p = synth.small(300, T=30, seed=51, electrodes=True, coil=True, snap_stride=10)
    ref = orc.run_problem(p, "plain")
    tm = eddy.ThetaMethod(form, p.theta, p.dt, release_inputs=True)
    tm.setup(p.L, p.R, p.E, p.M, p.MD, p.C)
    probes, snaps = tm.run(p.T, p.src, p.iD, p.snap_stride)
    assert rel_traces(probes, ref.probes) < TOL and rel_snaps(snaps, ref.snaps) < TOL
    if form == "plain":
        with pytest.raises(eddy.EcError) as e:
            tm.set_step(p.theta, 2 * p.dt)
        assert e.value.code == 8
    else:
        q = synth.small(300, T=30, seed=51, electrodes=True, coil=True, snap_stride=10,
                        dt=2 * p.dt)
        tm.set_step(q.theta, q.dt)
        tm.set_state(np.zeros(tm.state_size()))
        probes, snaps = tm.run(q.T, q.src, q.iD, q.snap_stride)
        refq = orc.run_problem(q, "plain")
        assert rel_traces(probes, refq.probes) < TOL and rel_snaps(snaps, refq.snaps) < TOL
    tm.close()
