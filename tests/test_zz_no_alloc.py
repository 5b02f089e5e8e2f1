"""The allocation-free solve entry point against the context-based one.

ec_solve_inverse_noalloc serves callers that cannot allocate device memory (their
GPU memory belongs to another allocator, or a real-time loop cannot take
cudaMalloc's latency and implicit synchronisation).  It must reproduce what a
context computes with ec_solve_z, x = Z^{-1} b, from the exported inverse factor,
on consecutive calls that reuse the library's fixed scratch array.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("n", [700, 8192])
def test_noalloc_matches_context_solve_twice(eddy, n):
    import torch
    p = synth.small(n, T=1, seed=41, electrodes=False, coil=True)
    tm = eddy.ThetaMethod("plain", p.theta, p.dt)
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    W = tm.inverse_factor(mem=eddy.EC_MEM_DEVICE)          # device, column-major C^{-1}
    rng = np.random.default_rng(n)
    for call in range(2):                                   # two calls in a row share the scratch
        b = rng.standard_normal(n)
        x_ref = tm.solve_z(b)                               # existing entry point (context)
        bd = torch.from_numpy(b).cuda()
        xd = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        eddy.solve_inverse_noalloc(W, bd, xd, stream=stream)
        torch.cuda.synchronize()
        x = xd.cpu().numpy()
        assert np.all(np.isfinite(x)), call
        assert rel(x, x_ref) < TOL, call


def test_noalloc_rejects_sizes_above_the_limit(eddy):
    import torch
    n = eddy.NOALLOC_MAX_N + 1
    W = torch.zeros((1,), dtype=torch.float64, device="cuda")
    b = torch.zeros((1,), dtype=torch.float64, device="cuda")
    with pytest.raises(eddy.EcError) as e:
        eddy.solve_inverse_noalloc(W, b, b, n=n)
    assert e.value.code == 2        # EC_ERR_SHAPE, checked before anything runs
