"""Failure paths of ec_setup, each made on the host (no GPU fault is injected).

* A rank-deficient electrode operator E (two identical rows) is reported as
  EC_ERR_RANK (Sec. 3.1: E must have full row rank, rank E = N_e - 1).
* A NaN or infinite entry in any input is refused with EC_ERR_ARG before any
  factorisation, and ec_last_info names the input.
* Device allocation failures, made by the library's allocator hook, surface as
  EC_ERR_OOM from whichever allocation ran out, and the context stays usable: after
  disarming the hook a new ec_setup on the same context runs and matches the oracle.
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


@pytest.mark.parametrize("form", ["plain", "modal"])
def test_rank_deficient_electrodes(eddy, form):
    p = synth.small(120, T=5, seed=5, electrodes=True, coil=True)
    E2 = np.concatenate([p.E, p.E], axis=0)              # two identical rows
    MD2 = np.concatenate([p.MD, p.MD], axis=1)
    tm = eddy.ThetaMethod(form, p.theta, p.dt)
    with pytest.raises(eddy.EcError) as e:
        tm.setup(p.L, p.R, E2, p.M, MD2, p.C)
    assert e.value.code == 4                             # EC_ERR_RANK
    # the context is usable for a new setup with a valid operator
    tm.setup(p.L, p.R, p.E, p.M, p.MD, p.C)
    probes, _ = tm.run(p.T, p.src, p.iD)
    ref = orc.run_problem(p, "plain")
    assert rel_traces(probes, ref.probes) < TOL
    tm.close()


@pytest.mark.parametrize("which,idx", [("L", 0), ("R", 1), ("E", 2), ("M", 3), ("MD", 4),
                                       ("C", 5)])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_input_refused(eddy, which, idx, bad):
    p = synth.small(90, T=5, seed=6, electrodes=True, coil=True)
    arrays = dict(L=p.L.copy(), R=p.R.copy(), E=p.E.copy(), M=p.M.copy(), MD=p.MD.copy(),
                  C=p.C.copy())
    a = arrays[which]
    a[a.shape[0] - 1, a.shape[1] // 2] = bad             # in the lower triangle for L, R
    tm = eddy.ThetaMethod("modal", p.theta, p.dt)
    with pytest.raises(eddy.EcError) as e:
        tm.setup(arrays["L"], arrays["R"], arrays["E"], arrays["M"], arrays["MD"], arrays["C"])
    assert e.value.code == 1 and e.value.info == idx     # EC_ERR_ARG, which input
    tm.close()


@pytest.mark.parametrize("form", ["plain", "modal"])
def test_out_of_memory_at_every_allocation(eddy, form):
    """Fail the k-th device allocation of a setup for every k; each failure is
    EC_ERR_OOM, and the same context then sets up and runs correctly."""
    p = synth.small(150, T=20, seed=7, electrodes=True, coil=True, snap_stride=5)
    ref = orc.run_problem(p, "plain")
    tm = eddy.ThetaMethod(form, p.theta, p.dt)
    failures = 0
    try:
        for k in range(0, 400):
            eddy.selftest_fail_alloc(k)
            try:
                tm.setup(p.L, p.R, p.E, p.M, p.MD, p.C)
            except eddy.EcError as e:
                assert e.code == 5, (k, e.code)          # EC_ERR_OOM
                failures += 1
                continue
            break                                        # k allocations were enough
        else:
            pytest.fail("setup never completed with the hook armed")
    finally:
        eddy.selftest_fail_alloc(-1)
    assert failures > 10                                 # many allocation sites exercised
    tm.setup(p.L, p.R, p.E, p.M, p.MD, p.C)
    probes, snaps = tm.run(p.T, p.src, p.iD, p.snap_stride)
    assert rel_traces(probes, ref.probes) < TOL
    assert rel_snaps(snaps, ref.snaps) < TOL
    tm.close()
