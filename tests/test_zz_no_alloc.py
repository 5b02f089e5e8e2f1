"""The allocation-free solve entry point against a dense solve and the context-based one.

ec_solve_inverse_noalloc serves callers that cannot allocate device memory (their
GPU memory belongs to another allocator, or a real-time loop cannot take
cudaMalloc's latency and implicit synchronisation).  It must give x = Z^{-1} b from
the exported inverse factor -- checked against numpy's dense solve of
Z = L + theta dt R and against what a context computes with ec_solve_z -- on
consecutive calls that reuse the library's fixed scratch array.  This file is
collected last on purpose.
"""
from ctypes import c_void_p

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


def _setup(eddy, n, seed=41):
    p = synth.small(n, T=1, seed=seed, electrodes=False, coil=True)
    tm = eddy.ThetaMethod("plain", p.theta, p.dt)
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    Z = p.L + p.theta * p.dt * p.R          # no electrodes: Z = L_i + theta dt R_i, K = I
    return p, tm, Z


@pytest.mark.parametrize("n", [1, 63, 64, 65, 700, 8192])
def test_noalloc_matches_dense_solve_twice(eddy, n):
    import torch
    p, tm, Z = _setup(eddy, n)
    W = tm.inverse_factor(mem=eddy.EC_MEM_DEVICE)          # device, column-major C^{-1}
    rng = np.random.default_rng(n)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                                   # two calls in a row share the scratch
        b = rng.standard_normal(n)
        x_dense = np.linalg.solve(Z, b)
        x_ctx = tm.solve_z(b)                               # existing entry point (context)
        bd = torch.from_numpy(b).cuda()
        xd = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        eddy.solve_inverse_noalloc(W, bd, xd, stream=stream)
        torch.cuda.synchronize()
        x = xd.cpu().numpy()
        assert np.all(np.isfinite(x)), call
        assert rel(x, x_dense) < TOL, call
        assert rel(x, x_ctx) < TOL, call
    tm.close()


def test_noalloc_in_place_and_padded_leading_dimension(eddy):
    """b and x may alias; Winv may carry a leading dimension larger than n (raw ABI)."""
    import torch
    n, ldw = 517, 600
    p, tm, Z = _setup(eddy, n, seed=7)
    W = tm.inverse_factor(mem=eddy.EC_MEM_DEVICE)           # (n, n), memory column-major
    Wp = torch.full((n, ldw), float("nan"), dtype=torch.float64, device="cuda")
    Wp[:, :n] = W                                            # column j at offset j * ldw
    Wp[:, n:] = 0.0
    rng = np.random.default_rng(3)
    stream = torch.cuda.current_stream().cuda_stream
    b = rng.standard_normal(n)
    x_dense = np.linalg.solve(Z, b)
    xb = torch.from_numpy(b.copy()).cuda()
    eddy.solve_inverse_noalloc(W, xb, xb, stream=stream)     # in place
    torch.cuda.synchronize()
    assert rel(xb.cpu().numpy(), x_dense) < TOL
    xd = torch.empty(n, dtype=torch.float64, device="cuda")
    bd = torch.from_numpy(b).cuda()
    code = eddy.lib().ec_solve_inverse_noalloc(n, c_void_p(Wp.data_ptr()), ldw,
                                               c_void_p(bd.data_ptr()), c_void_p(xd.data_ptr()),
                                               c_void_p(stream))
    assert code == 0
    torch.cuda.synchronize()
    assert rel(xd.cpu().numpy(), x_dense) < TOL
    tm.close()


def test_noalloc_rejects_sizes_above_the_limit(eddy):
    import torch
    n = eddy.NOALLOC_MAX_N + 1
    W = torch.zeros((1,), dtype=torch.float64, device="cuda")
    b = torch.zeros((1,), dtype=torch.float64, device="cuda")
    # raw ABI: the library refuses before touching any pointer
    code = eddy.lib().ec_solve_inverse_noalloc(n, c_void_p(W.data_ptr()), n,
                                               c_void_p(b.data_ptr()), c_void_p(b.data_ptr()),
                                               None)
    assert code == 2        # EC_ERR_SHAPE, checked before anything runs
    # the binding refuses tensors too short for n before calling the library
    with pytest.raises(ValueError):
        eddy.solve_inverse_noalloc(W, b, b, n=n)
