"""Why the fused FP32 pass of CGS-CQR2 (Alg. 5) fuses each update with the Gram
matrix of its result but not with the second projection: a numpy emulation of the
mixed form's arithmetic (FP32 blocks and products, FP64 Gram matrices, Cholesky
factors and projection coefficients).

* As built: the second projection P^T Y'' is taken from the normalised block
  Y'' = fl(Y' L^{-T}), so it also removes the rounding committed when Y'' is formed.
* The rejected variant: G = P^T Y' from the same pass that forms Y' = Y - P H, then
  H2 = G L^{-T}.  It misses that rounding, which is of order eps32 cond(Y'), so the
  final block is orthogonal to P only to a level that grows with cond(Y').

Design check, not a pin of the oracle: both sequences are written here."""

import numpy as np
import pytest


def _f32(x):
    return np.asarray(x, dtype=np.float32)


def _linv_t(W):
    return np.linalg.inv(np.linalg.cholesky(W)).T


def _cgs_cqr2_fp32(P, Y, fused_projection):
    P64 = P.astype(np.float64)
    H = P64.T @ Y.astype(np.float64)
    Y1 = _f32(Y - _f32(P @ _f32(H)))                       # S2 (FP32 update)
    W = Y1.astype(np.float64).T @ Y1.astype(np.float64)    # S3
    M = _linv_t(W)                                         # S4
    if fused_projection:
        H2 = (P64.T @ Y1.astype(np.float64)) @ M
    Y2 = _f32(Y1 @ _f32(M))                                # S5
    if not fused_projection:
        H2 = P64.T @ Y2.astype(np.float64)                 # S6
    Z = _f32(Y2 - _f32(P @ _f32(H2)))                      # S7
    W2 = Z.astype(np.float64).T @ Z.astype(np.float64)     # S8
    Q = _f32(Z @ _f32(_linv_t(W2))).astype(np.float64)     # S9, S10
    return np.abs(P64.T @ Q).max(), np.abs(Q.T @ Q - np.eye(Q.shape[1])).max()


def _case(rng, q, s, b, kappa):
    P = _f32(np.linalg.qr(rng.standard_normal((q, s)))[0])
    P64 = P.astype(np.float64)
    N = np.linalg.qr(rng.standard_normal((q, b)))[0]
    N = np.linalg.qr(N - P64 @ (P64.T @ N))[0]
    V = np.linalg.qr(rng.standard_normal((b, b)))[0]
    # mostly in span(P); the part outside it has condition number kappa
    Y = _f32(100.0 * P64 @ rng.standard_normal((s, b)) + (N * np.logspace(0, -np.log10(kappa), b)) @ V.T)
    return P, Y


@pytest.mark.parametrize("seed", [3, 11])
def test_second_projection_must_see_the_normalised_block(seed):
    rng = np.random.default_rng(seed)
    res = {}
    for kappa in (1e2, 1e4):
        P, Y = _case(rng, 20_000, 64, 16, kappa)
        res[kappa] = (_cgs_cqr2_fp32(P, Y, False), _cgs_cqr2_fp32(P, Y, True))
    for kappa, ((orth_a, unit_a), (orth_b, unit_b)) in res.items():
        # Alg. 5's order: orthogonal to P at FP32 rounding level whatever cond(Y')
        assert orth_a < 1e-8, (kappa, orth_a)
        # both produce orthonormal columns; the difference is the coupling to P
        assert unit_a < 1e-6 and unit_b < 1e-6
    # the fused projection loses orthogonality to P, the more the worse cond(Y')
    (_, _), (orth_b2, _) = res[1e2]
    (orth_a4, _), (orth_b4, _) = res[1e4]
    assert orth_b4 > 100 * orth_a4
    assert orth_b4 > 10 * orth_b2
