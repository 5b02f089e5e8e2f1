"""Plain form with an FP32 inverse factor and FP64 iterative refinement (EC_PREC_FP32)
against the FP64 oracle.  Stated errors (relative 2-norm over the probe trace):
no refinement < 1e-4 (FP32 rounding of the factor and the products), one sweep
< 1e-8, two sweeps < 1e-10 (the FP64 bar).  Measured values are printed."""
import numpy as np
import pytest

from oracle import theta as orc
from workloads import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eddy():
    from paper_2407_11993_gb300 import build, eddy as e
    build.build()
    return e


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def case():
    p = synth.small(2100, T=60, seed=21, electrodes=False, coil=True, snap_stride=20)
    return p, orc.run_problem(p, form="plain")


@pytest.mark.parametrize("refine,bound", [(0, 1e-4), (1, 1e-8), (2, 1e-10)])
def test_fp32_refinement_levels(eddy, case, refine, bound):
    p, ref = case
    tm = eddy.ThetaMethod("plain", p.theta, p.dt, precision="fp32", refine_steps=refine)
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    probes, snaps = tm.run(p.T, p.src, None, p.snap_stride)
    e_p, e_s = rel(probes, ref.probes), rel(snaps, ref.snaps)
    print(f"fp32 refine={refine}: probes {e_p:.3e} snapshots {e_s:.3e}")
    assert e_p < bound and e_s < bound


def test_fp32_solve_z(eddy):
    p = synth.small(1500, T=1, seed=22, electrodes=False, coil=True)
    b = np.random.default_rng(8).standard_normal(1500)
    Z = p.L + p.dt * p.theta * p.R
    x_ref = np.linalg.solve(Z, b)
    errs = []
    for refine in (0, 3):
        tm = eddy.ThetaMethod("plain", p.theta, p.dt, precision="fp32", refine_steps=refine)
        tm.setup(p.L, p.R, None, p.M, None, p.C)
        errs.append(rel(tm.solve_z(b), x_ref))
        tm.close()
    print("fp32 solve_z errors (0, 3 sweeps):", errs)
    assert errs[0] < 1e-4 and errs[1] < 1e-12


def test_fp32_unsupported_combinations(eddy):
    p = synth.small(300, T=3, seed=23, electrodes=True, coil=True)
    tm = eddy.ThetaMethod("plain", p.theta, p.dt, precision="fp32")
    with pytest.raises(eddy.EcError):
        tm.setup(p.L, p.R, p.E, p.M, p.MD, p.C)
    # the reduced-precision inverse factor serves the inverse solver only
    with pytest.raises(eddy.EcError):
        eddy.ThetaMethod("plain", p.theta, p.dt, precision="fp32", solver="substitution")


@pytest.mark.parametrize("n,el", [(65, True), (2100, False), (1029, True)])
def test_fp32_pair_factor(eddy, n, el):
    """EC_PREC_FP32X2: the inverse factor as FP32 hi/lo pairs and compensated FP32
    products (about 2^-46 per product entry).  Stated error: 1e-10 per probe trace and
    per snapshot against the FP64 oracle (measured values printed); electrodes allowed."""
    from parity import rel_snaps, rel_traces
    p = synth.small(n, T=60, seed=n, electrodes=el, coil=True, snap_stride=20)
    ref = orc.run_problem(p, form="plain")
    tm = eddy.ThetaMethod("plain", p.theta, p.dt, precision="fp32x2")
    tm.setup(p.L, p.R, p.E if el else None, p.M, p.MD if el else None, p.C)
    probes, snaps = tm.run(p.T, p.src, p.iD if el else None, p.snap_stride)
    tm.close()
    e_p, e_s = rel_traces(probes, ref.probes), rel_snaps(snaps, ref.snaps)
    print(f"fp32x2 n={n}: probes {e_p:.3e} snapshots {e_s:.3e}")
    assert e_p < 1e-10 and e_s < 1e-10


def test_fp32_pair_solve_z(eddy):
    p = synth.small(1500, T=1, seed=22, electrodes=False, coil=True)
    b = np.random.default_rng(8).standard_normal(1500)
    Z = p.L + p.dt * p.theta * p.R
    tm = eddy.ThetaMethod("plain", p.theta, p.dt, precision="fp32x2")
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    err = rel(tm.solve_z(b), np.linalg.solve(Z, b))
    tm.close()
    print(f"fp32x2 solve_z error {err:.3e}")
    assert err < 1e-12
