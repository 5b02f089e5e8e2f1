"""FP64-accurate tensor-core product (ec_gemm_f64_emulated) against exact products.

The reference is the product of the same FP64 inputs in extended precision (numpy
longdouble, 64-bit significand) or, for integer-valued inputs, the exact integer
product.  Bars:
  * integer-valued inputs with exactly representable sums: bit-for-bit equal;
  * well-scaled random inputs: |C - C_exact| <= K 2^-53 |A||B| entrywise (the FP64
    GEMM bound), and no worse than 8x the error of numpy's own FP64 product;
  * rows / columns of widely varying magnitude: |C - C_exact| <= 2^-50 sqrt(K)
    max_k|a_ik| max_k|b_kj| (the scheme's per-row / per-column scale).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def eddy():
    from paper_2407_11993_gb300 import build, eddy as e
    build.build()
    return e


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(eddy, A, B, C0=None, alpha=1.0, beta=0.0, ta=False, tb=False, lower=False):
    import torch
    Cd = None if C0 is None else _cuda(C0)
    out = eddy.gemm_f64_emulated(_cuda(A), _cuda(B), Cd, alpha=alpha, beta=beta, ta=ta, tb=tb,
                                 lower=lower)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _exact(A, B, ta=False, tb=False):
    a = (A.T if ta else A).astype(np.longdouble)
    b = (B.T if tb else B).astype(np.longdouble)
    return a @ b


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (127, 65, 33), (128, 64, 192), (129, 63, 193),
                                   (300, 200, 385), (64, 1000, 1500),
                                   # narrow products (MMA width 16 / 32)
                                   (4096, 4, 1000), (257, 16, 200), (300, 17, 385), (700, 32, 64),
                                   (129, 33, 97)])
def test_integer_inputs_are_exact(eddy, M, N, K):
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.integers(-1000, 1001, size=(M, K)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(K, N)).astype(np.float64)
    C = _run(eddy, A, B)
    assert np.array_equal(C, A @ B)          # all sums below 2^53: exact in FP64 too


@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
@pytest.mark.parametrize("M,N,K", [(127, 65, 33), (300, 200, 385), (513, 130, 1000),
                                   (2000, 5, 3000), (300, 20, 385)])
def test_random_within_fp64_bound(eddy, M, N, K, ta, tb):
    rng = np.random.default_rng(M + 3 * N + 5 * K + 11 * ta + 13 * tb)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((N, K) if tb else (K, N))
    C = _run(eddy, A, B, ta=ta, tb=tb)
    ex = _exact(A, B, ta, tb)
    absab = np.abs(A.T if ta else A) @ np.abs(B.T if tb else B)
    err = np.abs(C - ex).astype(np.float64)
    assert np.all(err <= K * U * absab)
    err64 = np.abs((A.T if ta else A) @ (B.T if tb else B) - ex).astype(np.float64)
    assert err.max() <= 8 * max(err64.max(), U * absab.max())


def test_alpha_beta_and_lower_triangle(eddy):
    rng = np.random.default_rng(5)
    n, K = 300, 200
    P = rng.standard_normal((n, K))
    C0 = rng.standard_normal((n, n))
    C = _run(eddy, P, P, C0=C0, alpha=-1.0, beta=1.0, tb=True, lower=True)
    ex = C0.astype(np.longdouble) - _exact(P, P, False, True)
    low = np.tril(np.ones((n, n), dtype=bool))
    absab = np.abs(C0) + np.abs(P) @ np.abs(P).T
    assert np.all(np.abs(C - ex)[low] <= (K + 2) * U * absab[low])
    assert np.array_equal(C[~low], C0[~low])           # upper triangle untouched
    C2 = _run(eddy, P, P[:64].T.copy(), C0=C0[:, :64].copy(), alpha=0.5, beta=-2.0)
    ex2 = -2.0 * C0[:, :64].astype(np.longdouble) + 0.5 * _exact(P, P[:64].T.copy())
    ab2 = 2 * np.abs(C0[:, :64]) + 0.5 * np.abs(P) @ np.abs(P[:64].T)
    assert np.all(np.abs(C2 - ex2) <= (K + 2) * U * ab2)


@pytest.mark.parametrize("kept", [False, True])
def test_subnormal_rows_and_columns(eddy, kept):
    """Rows of A (and a column of B) whose largest entry is subnormal keep every bit of
    their fixed-point image (mantissa shift 11 against the row exponent -1021): their
    products meet the per-row / per-column bound like any other.  Against a large column
    the subnormal rows give normal results, which a flushed row would leave at zero; the
    results that fall in the subnormal range carry their final rounding (a few units of
    2^-1074), hence the absolute slack."""
    import torch
    rng = np.random.default_rng(41)
    M, N, K = 300, 20, 257
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    sub = [3, 150, 299]
    A[sub] *= 1e-310                            # subnormal rows
    B[:, 7] *= 1e-310                           # a subnormal column
    B[:, 3] *= 1e12                             # a large column
    C = eddy.gemm_f64_emulated(_cuda(A), _cuda(B), kept_slices=kept).cpu().numpy()
    torch.cuda.synchronize()
    ex = _exact(A, B)
    rowmax = np.abs(A).max(axis=1)[:, None]
    colmax = np.abs(B).max(axis=0)[None, :]
    err = np.abs(C - ex).astype(np.float64)
    assert np.all(err <= 2.0 ** -50 * np.sqrt(K) * rowmax * colmax + 1e-320)
    for i in sub:
        assert abs(C[i, 3]) > 2.0 ** -1022


def test_wide_dynamic_range(eddy):
    """Entries spread over 12 decades inside rows and columns: the error is relative to
    each row's and column's largest entry (the split's scale)."""
    rng = np.random.default_rng(9)
    M, N, K = 200, 150, 700
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-6, 6, (M, K))
    B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-3, 3, (K, N))
    C = _run(eddy, A, B)
    ex = _exact(A, B)
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :]
    assert np.all(np.abs(C - ex) <= 2.0 ** -50 * np.sqrt(K) * scale)


def test_zero_rows_and_columns(eddy):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((130, 70))
    B = rng.standard_normal((70, 90))
    A[5] = 0.0
    B[:, 7] = 0.0
    C = _run(eddy, A, B)
    assert np.all(C[5] == 0.0) and np.all(C[:, 7] == 0.0)
    assert np.all(np.abs(C - _exact(A, B)) <= 70 * U * (np.abs(A) @ np.abs(B)))


@pytest.mark.parametrize("M,N,K", [(20000, 4, 1000), (19500, 30, 700), (4100, 1, 4099),
                                   (300, 32, 385), (129, 17, 193), (33000, 8, 250),
                                   (700, 40, 300), (20000, 70, 33)])
def test_kept_slices_stream_k(eddy, M, N, K):
    """The modal snapshot path (A's slices kept as swizzled 64 KB blocks, one stream-K
    launch per group of up to 32 columns): with more row tiles than SMs some tiles are cut
    between two CTAs and added to the zeroed C by both (two addends: order-independent).  Integer inputs are exact; the result is the
    same as the per-call path bit for bit on random inputs only up to FP64 rounding, so
    random inputs are checked against the FP64 bound."""
    rng = np.random.default_rng(M + N + K)
    A = rng.integers(-1000, 1001, size=(M, K)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(K, N)).astype(np.float64)
    C = eddy.gemm_f64_emulated(_cuda(A), _cuda(B), kept_slices=True).cpu().numpy()
    assert np.array_equal(C, _exact(A, B))
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C1 = eddy.gemm_f64_emulated(_cuda(A), _cuda(B), kept_slices=True).cpu().numpy()
    C2 = eddy.gemm_f64_emulated(_cuda(A), _cuda(B), kept_slices=True).cpu().numpy()
    assert np.array_equal(C1, C2)                       # run to run
    bound = 4.0 * K * 2.0 ** -53 * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(C1 - A @ B) <= bound + 1e-300)
