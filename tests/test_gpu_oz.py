"""The FP64-accurate sliced product on the tensor cores (tsvd_dense_mm_f64tc),
through the C ABI, against exact and FP64 references.

* Integer data whose products and sums are exact in FP64: the result must equal
  numpy's bit for bit (this exercises the digit split, the exponent handling,
  the exact FP32 group sums, the 64-bit accumulation and the final scaling).
* Random data: the error bound stated in the header, against an exact
  reference (error-free products, math.fsum), and the usual 2 K eps |A||X|
  bound against numpy at larger sizes spanning many tiles, ragged tails, both
  tile-distribution modes, split K and the 64-bit flush.
* Inf/NaN propagate to their row (column); zero rows give zeros; two calls give
  the same bits.
"""

import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _t(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _tc(tsvd, torch, A, X, trans):
    return tsvd.dense_mm(_t(torch, A), _t(torch, X), trans=trans, tensor_cores=True).cpu().numpy()


def _veltkamp(a):
    c = a * 134217729.0  # 2^27 + 1
    hi = c - (c - a)
    return hi, a - hi


def _exact(A, X):
    """Correctly rounded A X: error-free products (Veltkamp split) summed by fsum."""
    a1, a2 = _veltkamp(A)
    x1, x2 = _veltkamp(X)
    M, K = A.shape
    N = X.shape[1]
    out = np.empty((M, N))
    for i in range(M):
        for j in range(N):
            terms = np.concatenate([a1[i] * x1[:, j], a1[i] * x2[:, j], a2[i] * x1[:, j], a2[i] * x2[:, j]])
            out[i, j] = math.fsum(terms)
    return out


def _pow2_above(v):
    """2^e with e the smallest integer such that |v| < 2^e (1 for v == 0)."""
    return np.where(v > 0, np.ldexp(1.0, np.frexp(v)[1]), 1.0)


def _bound(A, X, ref):
    """The header's error bound of the sliced product."""
    K = A.shape[1]
    ea = _pow2_above(np.abs(A).max(axis=1, keepdims=True))
    eb = _pow2_above(np.abs(X).max(axis=0, keepdims=True))
    return (2.0 ** -56 * (ea * np.abs(X).sum(axis=0, keepdims=True) + np.abs(A).sum(axis=1, keepdims=True) * eb)
            + 6.2 * K * ea * eb * 2.0 ** -56 + 2.0 ** -52 * (np.abs(A) @ np.abs(X)))


@pytest.mark.parametrize("trans", [0, 1])
@pytest.mark.parametrize("m,n,w", [(300, 200, 64), (1000, 77, 33), (129, 513, 100), (40_000, 64, 64)])
def test_integer_data_is_exact(tsvd, torch_cuda, trans, m, n, w):
    rng = np.random.default_rng(m + n + w + trans)
    A = rng.integers(-1000, 1001, size=(m, n)).astype(np.float64)
    X = rng.integers(-1000, 1001, size=((m if trans else n), w)).astype(np.float64)
    # rows of op(A) and columns of X at different binary scales: still exact
    if trans:
        A *= np.ldexp(1.0, rng.integers(-40, 40, size=(1, n)))
    else:
        A *= np.ldexp(1.0, rng.integers(-40, 40, size=(m, 1)))
    X *= np.ldexp(1.0, rng.integers(-30, 30, size=(1, w)))
    ref = (A.T @ X) if trans else (A @ X)
    Y = _tc(tsvd, torch_cuda, A, X, trans)
    assert np.array_equal(Y, ref)


@pytest.mark.parametrize("trans", [0, 1])
def test_random_data_within_stated_bound(tsvd, torch_cuda, trans):
    rng = np.random.default_rng(7 + trans)
    m, n, w = 700, 180, 24
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-5, 5, size=(m, 1)))
    X = rng.standard_normal(((m if trans else n), w))
    Y = _tc(tsvd, torch_cuda, A, X, trans)
    opA = A.T if trans else A
    ref = _exact(opA, X)
    err = np.abs(Y - ref)
    bound = _bound(opA, X, ref)
    print(f"trans={trans}: max error / bound {np.max(err / bound):.2e}")
    assert np.all(err <= bound)


@pytest.mark.parametrize("trans,m,n,w", [
    (0, 20_000, 600, 64),     # tiles > one wave: most tiles whole in one CTA (direct), the rest cut
    (0, 5_000, 1_100, 128),   # two 64-wide column tiles, split K blocks and the fix-up
    (1, 100_000, 576, 64),    # A^T X with K = 100,000 split over the CTAs (the projection shape)
    (1, 100_000, 64, 64),     # the Gram shape
    (1, 1_300_000, 64, 16),   # K blocks per CTA above one 64-bit accumulation: the flush path
    (0, 3_001, 45, 7),        # ragged everything, N < 32
])
def test_large_shapes_within_fp64_bound(tsvd, torch_cuda, trans, m, n, w):
    torch = torch_cuda
    g = torch.Generator(device="cuda").manual_seed(m + n + w)
    A = torch.randn(m, n, dtype=torch.float64, device="cuda", generator=g)
    X = torch.randn((m if trans else n), w, dtype=torch.float64, device="cuda", generator=g)
    Y = tsvd.dense_mm(A, X, trans=bool(trans), tensor_cores=True)
    Y2 = tsvd.dense_mm(A, X, trans=bool(trans), tensor_cores=True)
    assert torch.equal(Y, Y2)  # deterministic
    opA = A.T if trans else A
    ref = opA @ X
    K = opA.shape[1]
    bound = 2 * K * EPS * (opA.abs() @ X.abs())
    err = (Y - ref).abs()
    assert bool((err <= bound).all()), float((err / bound).max())
    # and much closer than the bound in practice
    print(f"trans={trans} {m}x{n}x{w}: max |err| / (K eps |A||X|) = {float((err / (bound / 2)).max()):.2e}")


def test_nonfinite_and_zero_rows(tsvd, torch_cuda):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((300, 100))
    X = rng.standard_normal((100, 40))
    A[5, 17] = np.nan
    A[9, 3] = np.inf
    A[11] = 0.0
    X[:, 7] = 0.0
    Y = _tc(tsvd, torch_cuda, A, X, 0)
    assert np.all(np.isnan(Y[5])) and np.all(np.isnan(Y[9]))
    assert np.all(Y[11] == 0.0) and np.all(Y[:, 7][np.isfinite(Y[:, 7])] == 0.0)
    ok = np.ones(300, bool)
    ok[[5, 9]] = False
    ref = A[ok] @ X
    assert np.all(np.abs(Y[ok] - ref) <= 2 * 100 * EPS * (np.abs(A[ok]) @ np.abs(X)))


def test_degenerate_shapes(tsvd, torch_cuda):
    torch = torch_cuda
    A = torch.randn(50, 0, dtype=torch.float64, device="cuda")
    X = torch.randn(0, 5, dtype=torch.float64, device="cuda")
    Y = tsvd.dense_mm(A, X, tensor_cores=True)
    assert tuple(Y.shape) == (50, 5) and bool((Y == 0).all())
    A = torch.randn(50, 30, dtype=torch.float64, device="cuda")
    Y = tsvd.dense_mm(A, torch.randn(30, 0, dtype=torch.float64, device="cuda"), tensor_cores=True)
    assert tuple(Y.shape) == (50, 0)
