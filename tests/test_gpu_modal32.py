"""The modal form's FP32 and FP32-pair variants (EC_PREC_FP32, EC_PREC_FP32X2).

Only the products with the mode matrix U change (projections U^T [R_D | L_D | M_0],
U^T (C K)^T and the snapshot reconstruction U x); the eigensolve and the per-mode
recurrence stay FP64.  Both variants are compared with the FP64 oracle on the same
seeded inputs.

* FP32X2 carries about 48 significant bits per U entry and compensated FP32
  arithmetic: it must meet the FP64 path's bar, 1e-10 per probe trace and per
  snapshot.
* FP32 rounds every operand to 24 bits and sums in FP32 within K segments: its error is
  stated against the size of the parts that cancel in the output (eddy currents against
  the injected particular field, as for the BF16 variants) with bound 1e-4.

Sizes cover a ragged n0 (not a multiple of the 4-row loads), 1 to 9 snapshots per run
(one and two column groups of the products), truncated modes (K < n0) and the
independent right-hand-side mode.
"""
import numpy as np
import pytest

from oracle import theta as orc
from parity import rel_snaps, rel_traces
from workloads import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eddy():
    from paper_2407_11993_gb300 import build, eddy as e
    build.build()
    return e


def cancel_rel(got, ref, part):
    """||got - ref|| / (||ref - part|| + ||part||), per column of a (rows, cols) array."""
    got, ref, part = (np.atleast_2d(np.asarray(x, dtype=np.float64)) for x in (got, ref, part))
    num = np.linalg.norm(got - ref, axis=0)
    den = np.linalg.norm(ref - part, axis=0) + np.linalg.norm(part, axis=0)
    den = np.where(den > 0, den, 1.0)
    return float((num / den).max())


@pytest.mark.parametrize("n,T,stride,electrodes", [(301, 45, 5, True), (514, 40, 40, False),
                                                   (1027, 36, 4, True)])
def test_modal_fp32x2_matches_oracle(eddy, n, T, stride, electrodes):
    p = synth.small(n, T, seed=n, electrodes=electrodes, coil=True, probes=4, snap_stride=stride)
    ref = orc.run_problem(p, "plain")
    tm = eddy.ThetaMethod("modal", p.theta, p.dt, precision="fp32x2")
    tm.setup(p.L, p.R, p.E if electrodes else None, p.M, p.MD if electrodes else None, p.C)
    probes, snaps = tm.run(p.T, p.src, p.iD if electrodes else None, stride)
    tm.close()
    ep, es = rel_traces(probes, ref.probes), rel_snaps(snaps, ref.snaps)
    print(f"fp32x2 modal n={n} T={T} stride={stride}: per-trace {ep:.2e}, per-snapshot {es:.2e}")
    assert ep < 1e-10 and es < 1e-10


@pytest.mark.parametrize("n,T,stride,electrodes", [(301, 45, 5, True), (1027, 36, 4, True),
                                                   (514, 40, 40, False)])
def test_modal_fp32_matches_oracle_at_stated_bound(eddy, n, T, stride, electrodes):
    p = synth.small(n, T, seed=n, electrodes=electrodes, coil=True, probes=4, snap_stride=stride)
    ref = orc.run_problem(p, "plain")
    red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    tm = eddy.ThetaMethod("modal", p.theta, p.dt, precision="fp32")
    tm.setup(p.L, p.R, p.E if electrodes else None, p.M, p.MD if electrodes else None, p.C)
    probes, snaps = tm.run(p.T, p.src, p.iD if electrodes else None, stride)
    tm.close()
    if electrodes:
        part_p = (red.CPE @ p.iD[:, 1:]).T
        part_s = red.PE @ p.iD[:, stride::stride]
    else:
        part_p = np.zeros_like(ref.probes.T)
        part_s = np.zeros_like(ref.snaps)
    ep = cancel_rel(probes.T, ref.probes.T, part_p)
    es = cancel_rel(snaps, ref.snaps, part_s)
    print(f"fp32 modal n={n}: probe {ep:.2e}, snapshot {es:.2e} (against the cancelling parts); "
          f"plain per-trace {rel_traces(probes, ref.probes):.2e}")
    assert ep < 1e-4 and es < 1e-4


def test_modal_fp32x2_truncated_modes(eddy):
    """K < n0 in the reconstruction: the nkeep slowest modes only, against the oracle's
    truncated modal run."""
    p = synth.small(402, 30, seed=5, electrodes=False, coil=True, probes=4, snap_stride=3)
    red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    md = orc.modal_setup(red.Li, red.Ri)
    keep = 37
    ref = orc.theta_modal(red, orc.Modes(md.tau[:keep], md.U[:, :keep]), p.theta, p.dt, p.src,
                          p.iD, p.T, None, p.snap_stride)
    tm = eddy.ThetaMethod("modal", p.theta, p.dt, precision="fp32x2")
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    tm.set_mode_count(keep)
    probes, snaps = tm.run(p.T, p.src, None, p.snap_stride)
    tm.close()
    ep, es = rel_traces(probes, ref.probes), rel_snaps(snaps, ref.snaps)
    print(f"fp32x2 keep={keep}: per-trace {ep:.2e}, per-snapshot {es:.2e}")
    assert ep < 1e-10 and es < 1e-10


def test_modal_fp32x2_independent_coils(eddy):
    """Nine coils as independent trajectories: 9 x nsnap right-hand columns (two column
    groups of the product) and nine projected source columns."""
    p = synth.coil_scan(300, T=20, n_side=3, probes=3)
    tm = eddy.ThetaMethod("modal", p.theta, p.dt, precision="fp32x2", rhs="independent")
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    probes, snaps = tm.run(p.T, p.src, None, 10)
    tm.close()
    t64 = eddy.ThetaMethod("modal", p.theta, p.dt, rhs="independent")
    t64.setup(p.L, p.R, None, p.M, None, p.C)
    p64, s64 = t64.run(p.T, p.src, None, 10)
    t64.close()
    ep, es = rel_traces(probes, p64), rel_snaps(snaps, s64)
    print(f"fp32x2 independent coils: per-trace {ep:.2e}, per-snapshot {es:.2e} vs FP64 GPU")
    assert ep < 1e-10 and es < 1e-10


def test_set_precision_reuses_the_modes(eddy):
    """One eigensolve, several arithmetics: switching to FP32X2 matches a context set up
    in FP32X2 bit for bit, and switching back to FP64 reproduces the FP64 run bit for
    bit (the modes are untouched).  Inputs released after the setup."""
    p = synth.small(333, 24, seed=9, electrodes=True, coil=True, probes=4, snap_stride=6)
    args = (p.L, p.R, p.E, p.M, p.MD, p.C)

    def run(tm):
        tm.set_state(np.zeros(tm.state_size()))
        return tm.run(p.T, p.src, p.iD, p.snap_stride)

    tm = eddy.ThetaMethod("modal", p.theta, p.dt, release_inputs=True)
    tm.setup(*args)
    p64, s64 = run(tm)
    tm.set_precision("fp32x2")
    px, sx = run(tm)
    tm.set_precision("fp64")
    p64b, s64b = run(tm)
    tm.close()
    direct = eddy.ThetaMethod("modal", p.theta, p.dt, precision="fp32x2")
    direct.setup(*args)
    pd, sd = run(direct)
    direct.close()
    assert np.array_equal(p64, p64b) and np.array_equal(s64, s64b)
    assert np.array_equal(px, pd) and np.array_equal(sx, sd)
    assert rel_traces(px, p64) < 1e-10 and rel_snaps(sx, s64) < 1e-10


@pytest.mark.parametrize("keep,stride", [(None, 3), (1500, 1), (4099, 30)])
def test_fp64_reconstruction_from_kept_slices(eddy, keep, stride):
    """From N0 = 4096 on, FP64 snapshot reconstructions multiply U's kept tensor-core
    slices (narrow MMAs for up to 32 columns).  Against the FP64-core path of the same
    setup arithmetic (no kept slices) on 1 to 30 snapshot columns and truncated modes, at the
    FP64 bar (the two setups round differently)."""
    p = synth.small(4100, 30, seed=3, electrodes=False, coil=True, probes=4, snap_stride=stride)
    outs = {}
    for g in ("tensor", "fp64"):
        tm = eddy.ThetaMethod("modal", p.theta, p.dt, setup_gemm=g)
        tm.setup(p.L, p.R, None, p.M, None, p.C)
        if keep:
            tm.set_mode_count(keep)
        outs[g] = tm.run(p.T, p.src, None, stride)
        tm.close()
    (pt, st_), (pf, sf) = outs["tensor"], outs["fp64"]
    ep, es = rel_traces(pt, pf), rel_snaps(st_, sf)
    print(f"kept slices keep={keep} stride={stride}: per-trace {ep:.2e}, per-snapshot {es:.2e}")
    assert ep < 1e-10 and es < 1e-10
