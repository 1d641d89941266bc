"""The fused update + Gram pass of FP32 blocks (CGS-CQR2, Alg. 5 S2-S3 and S7-S8;
CholeskyQR2, Alg. 4, first step's Q L^{-T} with the second step's Gram matrix),
through the C ABI.

* The updated block has the same bits as the unfused FP32 product
  (tsvd_dense_mm_f32, the kernel the unfused path runs).
* The Gram matrix is within the FP32 bound of the exact Gram matrix of the block
  the call returned: per entry (r + 2) u |Y'|^T |Y'| with r the rows one CTA sums
  in FP32 (at most q rows) and u = 2^-24; both halves carry the same bits.
* Ragged sizes: rows not a multiple of the 64-row tile, widths 1 .. 128 around the
  64-column panels, one-column and wide inner dimensions.
* FP32 CGS-CQR2 (tsvd_cgs_cqr2_f32) against the FP64 oracle on the same
  FP32-valued inputs, with FP32 tolerances scaled by the block's condition number.
"""

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _f32(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _f64(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _np(t):
    return t.detach().cpu().numpy()


def _gram_bound(Yn, q):
    Ya = np.abs(Yn.astype(np.float64))
    return (q + 2) * U32 * (Ya.T @ Ya) + 1e-300


@pytest.mark.parametrize("q,s,b", [(64, 1, 1), (1000, 17, 33), (10007, 300, 64), (10007, 300, 65),
                                   (40000, 576, 128), (777, 128, 100)])
def test_update_matches_unfused_product_bits(tsvd, torch_cuda, q, s, b):
    torch = torch_cuda
    rng = np.random.default_rng(q + s + b)
    X = rng.standard_normal((q, s)).astype(np.float32)
    M = rng.standard_normal((s, b))
    Xt, Mt = _f32(torch, X), _f64(torch, M)
    Y1, W = tsvd.update_gram_f32(Xt, Mt, alpha=1.0, beta=0.0)
    # the unfused FP32 product of the same operands (M rounded to FP32, as the fused pass does)
    Y0 = tsvd.dense_mm(Xt, Mt.float())
    torch.cuda.synchronize()
    assert torch.equal(Y1, Y0)
    Yn, Wn = _np(Y1), _np(W)
    Y64 = Yn.astype(np.float64)
    assert np.all(np.abs(Wn - Y64.T @ Y64) <= _gram_bound(Yn, q))
    assert np.array_equal(Wn, Wn.T)


@pytest.mark.parametrize("q,s,b", [(5003, 320, 64), (20000, 256, 128), (130, 5, 7)])
def test_update_with_beta_and_its_gram(tsvd, torch_cuda, q, s, b):
    """Y' = Y - P H (the CGS update) and its Gram matrix, against FP64 arithmetic."""
    torch = torch_cuda
    rng = np.random.default_rng(7 * q + b)
    P = np.linalg.qr(rng.standard_normal((q, s)))[0].astype(np.float32)
    Y = (rng.standard_normal((q, b)) + P.astype(np.float64) @ rng.standard_normal((s, b))).astype(np.float32)
    H = P.astype(np.float64).T @ Y.astype(np.float64)
    Yt, W = tsvd.update_gram_f32(_f32(torch, P), _f64(torch, H), _f32(torch, Y), alpha=-1.0, beta=1.0)
    Yn, Wn = _np(Yt), _np(W)
    ref = Y.astype(np.float64) - P.astype(np.float64) @ H.astype(np.float32).astype(np.float64)
    bound = (s + 2) * U32 * (np.abs(Y.astype(np.float64))
                             + np.abs(P.astype(np.float64)) @ np.abs(H.astype(np.float32).astype(np.float64)))
    assert np.all(np.abs(Yn - ref) <= bound + U32 * np.abs(ref))
    Y64 = Yn.astype(np.float64)
    assert np.all(np.abs(Wn - Y64.T @ Y64) <= _gram_bound(Yn, q))
    # deterministic: a second call gives the same bits
    Yt2, W2 = tsvd.update_gram_f32(_f32(torch, P), _f64(torch, H), _f32(torch, Y), alpha=-1.0, beta=1.0)
    assert torch.equal(Yt, Yt2) and torch.equal(W, W2)


@pytest.mark.parametrize("q,b", [(9001, 64), (4096, 128), (300, 20)])
def test_in_place_triangular_update_and_gram(tsvd, torch_cuda, q, b):
    """CholeskyQR2's Y L^{-T} done in place, fused with the next step's Gram matrix."""
    torch = torch_cuda
    rng = np.random.default_rng(q)
    Y = rng.standard_normal((q, b)).astype(np.float32)
    Mfull = rng.standard_normal((b, b))
    Mup = np.triu(Mfull)
    Yt = _f32(torch, Y)
    Y0 = tsvd.dense_mm(Yt, _f64(torch, Mup).float())
    # entries below the diagonal of M must not be read
    Yo, W = tsvd.update_gram_f32(Yt, _f64(torch, Mfull), alpha=1.0, beta=0.0, upper=True, in_place=True)
    assert Yo.data_ptr() == Yt.data_ptr()
    assert torch.equal(Yo, Y0)
    Yn, Wn = _np(Yo), _np(W)
    Y64 = Yn.astype(np.float64)
    assert np.all(np.abs(Wn - Y64.T @ Y64) <= _gram_bound(Yn, q))


def test_update_gram_rejects_bad_shapes(tsvd, torch_cuda):
    torch = torch_cuda
    X = torch.zeros((100, 129), dtype=torch.float32, device="cuda")
    M = torch.zeros((129, 129), dtype=torch.float64, device="cuda")
    with pytest.raises(tsvd.TsvdError):
        tsvd.update_gram_f32(X, M)            # b > 128
    with pytest.raises(ValueError):
        tsvd.update_gram_f32(X[:, :10], M[:10, :5], in_place=True)


def _cond_block(rng, q, b, cond):
    U = np.linalg.qr(rng.standard_normal((q, b)))[0]
    V = np.linalg.qr(rng.standard_normal((b, b)))[0]
    return (U * np.logspace(0, -np.log10(cond), b)) @ V.T


@pytest.mark.parametrize("q,s,b,cond", [(5003, 320, 64, 10.0), (20000, 576, 64, 1e3), (3001, 0, 128, 1e2),
                                        (1000, 16, 16, 1.0), (3000, 7, 5, 1e2)])
def test_cgs_cqr2_f32_matches_oracle(tsvd, torch_cuda, q, s, b, cond):
    torch = torch_cuda
    rng = np.random.default_rng(q + s)
    P64 = np.linalg.qr(rng.standard_normal((q, max(s, 1))))[0][:, :s]
    P = P64.astype(np.float32)
    Y = (_cond_block(rng, q, b, cond) + P64 @ rng.standard_normal((s, b)) * 5).astype(np.float32)
    Pt = _f32(torch, P) if s > 0 else torch.zeros((q, 0), dtype=torch.float32, device="cuda")
    Q, H, R, bd = tsvd.cgs_cqr2(_f32(torch, Y), Pt)
    assert bd == 0
    Qn, Hn, Rn = _np(Q).astype(np.float64), _np(H), _np(R)
    # the oracle on the same FP32-valued inputs (P is orthonormal only to FP32 rounding,
    # which both sides see alike)
    Qo, Ho, Ro = oracle.cgs_cqr2(Y.astype(np.float64), P.astype(np.float64))
    tol = 200 * U32 * cond
    np.testing.assert_allclose(Rn, Ro, rtol=0, atol=tol * np.abs(Ro).max())
    if s > 0:
        np.testing.assert_allclose(Hn, Ho, rtol=0, atol=tol * np.abs(Ho).max())
        assert np.abs(P.astype(np.float64).T @ Qn).max() < 50 * U32 * np.sqrt(q)
    np.testing.assert_allclose(Qn, Qo, rtol=0, atol=tol)
    assert np.abs(Qn.T @ Qn - np.eye(b)).max() < 50 * U32 * np.sqrt(q)
