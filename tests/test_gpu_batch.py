"""Batched instances (ec_batch_run): uneven plain-form problems advanced together in one
graph-captured, persistent pass must reproduce each instance's own ec_run bit for bit,
and the FP64 oracle to the FP64 tolerance."""
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


# (n, electrodes, coil, seed): ragged sizes from a single partial tile to several
# tile rows, with and without the electrode constraint
CASES = [(97, False, True, 1), (700, True, True, 2), (1029, False, True, 3), (1500, True, False, 4),
         (2100, True, True, 5)]


def problems(T, stride):
    out = []
    for n, el, coil, seed in CASES:
        p = synth.small(n, T=T, seed=seed, electrodes=el, coil=coil, snap_stride=stride)
        out.append(p)
    return out


def make(eddy, p):
    tm = eddy.ThetaMethod("plain", p.theta, p.dt)
    has_e = p.E.shape[0] > 0
    tm.setup(p.L, p.R, p.E if has_e else None, p.M if p.M.shape[1] else None,
             p.MD if has_e else None, p.C)
    return tm


def test_batch_equals_individual_runs_bitwise_and_oracle(eddy):
    T, T2, stride = 40, 15, 10
    ps = problems(T + T2, stride)      # sources cover both batches below
    single = []
    for p in ps:
        tm = make(eddy, p)
        single.append(tm.run(T, p.src[:, :T + 1] if p.M.shape[1] else None,
                             p.iD[:, :T + 1] if p.E.shape[0] else None, stride))
        tm.close()
    models = [make(eddy, p) for p in ps]
    batched = eddy.batch_run(models, T, [p.src[:, :T + 1] for p in ps],
                             [p.iD[:, :T + 1] for p in ps], stride)
    for (pa, sa), (pb, sb) in zip(single, batched):
        assert np.array_equal(pa, pb)
        assert np.array_equal(sa, sb)
    for p, (pb, sb) in zip(ps, batched):
        ref = orc.run_problem(p, form="plain", T=T)
        assert rel_traces(pb, ref.probes) < TOL
        assert rel_snaps(sb, ref.snaps) < TOL
    # the batch leaves every instance at its own I^T: a second batch continues exactly
    more = eddy.batch_run(models, T2, [p.src[:, T:T + T2 + 1] for p in ps],
                          [p.iD[:, T:T + T2 + 1] for p in ps], 0)
    for p, m, (pb, _) in zip(ps, models, more):
        tm = make(eddy, p)
        full, _ = tm.run(T + T2, p.src[:, :T + T2 + 1] if p.M.shape[1] else None,
                         p.iD[:, :T + T2 + 1] if p.E.shape[0] else None, 0)
        assert np.array_equal(full[:, T:], pb)
        tm.close()
    for m in models:
        m.close()


def test_batch_rejects_modal_and_duplicates(eddy):
    p = synth.small(300, T=5, seed=9, electrodes=False, coil=True)
    a = make(eddy, p)
    mod = eddy.ThetaMethod("modal", p.theta, p.dt)
    mod.setup(p.L, p.R, None, p.M, None, p.C)
    with pytest.raises(eddy.EcError):
        eddy.batch_run([a, mod], 5, [p.src, p.src], None)
    with pytest.raises(eddy.EcError):
        eddy.batch_run([a, a], 5, [p.src, p.src], None)
    a.close()
    mod.close()


def test_batch_of_twenty_uneven_instances(eddy):
    """20 instances with N drawn uniformly from [200, 3000] (fixed seed, half of them with
    the electrode constraint): every instance bitwise equal to its own ec_run, and equal
    to the oracle per trace."""
    rng = np.random.default_rng(2024)
    sizes = [int(x) for x in rng.integers(200, 3001, size=20)]
    T, stride = 24, 8
    ps = [synth.small(n, T=T, seed=100 + i, electrodes=(i % 2 == 0), coil=True, snap_stride=stride)
          for i, n in enumerate(sizes)]
    single = []
    for p in ps:
        tm = make(eddy, p)
        single.append(tm.run(T, p.src, p.iD if p.E.shape[0] else None, stride))
        tm.close()
    models = [make(eddy, p) for p in ps]
    batched = eddy.batch_run(models, T, [p.src for p in ps], [p.iD for p in ps], stride)
    for (pa, sa), (pb, sb) in zip(single, batched):
        assert np.array_equal(pa, pb) and np.array_equal(sa, sb)
    for i in (0, 7, 19):
        ref = orc.run_problem(ps[i], form="plain", T=T)
        assert rel_traces(batched[i][0], ref.probes) < TOL
        assert rel_snaps(batched[i][1], ref.snaps) < TOL
    for m in models:
        m.close()
