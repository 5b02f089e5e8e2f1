"""tcgen05 BF16 GEMM (FP32 accumulation) and the modal form's BF16 precision variant.

The GEMM is checked against an FP64 product of the same BF16-rounded inputs: the
only remaining error is FP32 accumulation, bounded by ~K 2^-24 |A||B|.  The
BF16 variant's outputs are compared with the FP64 oracle and must stay within the
BF16 rounding level of the projected quantities (stated bound 2e-2, measured
values printed).
"""
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


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 200, 1000), (1, 1, 1), (257, 129, 8191),
                                   (1000, 3, 5000), (4096, 256, 4096)])
def test_bf16_gemm_matches_fp64_product_of_rounded_inputs(eddy, M, N, K):
    import torch
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn((M, K), generator=g, dtype=torch.float64).cuda()
    B = torch.randn((K, N), generator=g, dtype=torch.float64).cuda()
    C = eddy.gemm_bf16(A, B)
    torch.cuda.synchronize()
    Ar = A.to(torch.bfloat16).double()
    Br = B.to(torch.bfloat16).double()
    ref = (Ar @ Br).cpu().numpy()
    got = C.cpu().numpy()
    bound = 4.0 * K * 2.0 ** -24 * (Ar.abs() @ Br.abs()).cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound + 1e-30), np.max(np.abs(got - ref) / (bound + 1e-30))


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision,bound", [("bf16", 2e-2), ("bf16x3", 1e-5)])
def test_modal_bf16_config1(eddy, precision, bound):
    p = synth.config1()
    ref = orc.run_problem(p, "plain")
    tm = eddy.ThetaMethod("modal", p.theta, p.dt, precision=precision)
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    probes, _ = tm.run(p.T, p.src, None, 0)
    err = rel(probes, ref.probes)
    print(f"modal {precision} N=512 probe rel err {err:.3e}")
    assert err < bound


@pytest.mark.parametrize("precision,bound", [("bf16", 2e-1), ("bf16x3", 1e-3)])
def test_modal_bf16_config2_snapshots(eddy, precision, bound):
    """Electrode step at N = 8192.  Early in the transient the eddy currents K U x
    nearly cancel the injected particular field E^T (E E^T)^{-1} i_D, so the BF16
    error is stated against the size of the two cancelling parts, not the small sum.
    (The FP64 variant is the one to use when that cancellation matters.)"""
    p = synth.config2(T=40, snap_stride=20)
    ref = orc.run_problem(p, "plain")
    red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
    tm = eddy.ThetaMethod("modal", p.theta, p.dt, precision=precision)
    tm.setup(p.L, p.R, p.E, None, p.MD, p.C)
    probes, snaps = tm.run(p.T, None, p.iD, p.snap_stride)
    part_s = red.PE @ p.iD[:, 20::20]
    part_p = red.CPE @ p.iD[:, 1:]
    scale_s = np.linalg.norm(ref.snaps - part_s) + np.linalg.norm(part_s)
    scale_p = np.linalg.norm(ref.probes - part_p) + np.linalg.norm(part_p)
    e_s = np.linalg.norm(snaps - ref.snaps) / scale_s
    e_p = np.linalg.norm(probes - ref.probes) / scale_p
    print(f"modal {precision} N=8192: probe err {e_p:.3e}, snapshot err {e_s:.3e} (relative to the "
          f"cancelling parts); plain relative {rel(probes, ref.probes):.3e} / {rel(snaps, ref.snaps):.3e}")
    assert e_p < bound and e_s < bound
