"""Pins of the oracle's truncated-SVD gradient (oracle/tsvd_backward.py) against
things other than itself: central finite differences of losses evaluated with
LAPACK's full SVD, the closed form dsum(sigma)/dA = U V^T, the rank-k special case
(where the complement terms reduce to the familiar (I - UU^T) U_bar S^-1 V^T form),
and agreement of its two complement solvers."""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import svd_backward


def _top_k(A, k):
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    U, V = U[:, :k], Vt[:k].T
    # sign convention of the library: largest-|.| entry of each v_j positive
    sg = np.sign(V[np.argmax(np.abs(V), axis=0), np.arange(k)])
    return s[:k], U * sg, V * sg


def _loss_parts(s, U, V, c, x, wu, y, wv):
    """L = sum c_i s_i + sum wu_i (u_i^T x)^2 + sum wv_i (v_i^T y)^2 (sign-invariant)."""
    ux, vy = U.T @ x, V.T @ y
    L = c @ s + wu @ ux ** 2 + wv @ vy ** 2
    return L, c.copy(), 2 * np.outer(x, wu * ux), 2 * np.outer(y, wv * vy)


@pytest.mark.parametrize("m,n", [(40, 30), (30, 40)])
def test_gradient_matches_central_differences_of_the_full_svd(m, n):
    rng = np.random.default_rng(0)
    k = 4
    A = rng.standard_normal((m, n))
    c, wu, wv = rng.standard_normal(k), rng.standard_normal(k), rng.standard_normal(k)
    x, y = rng.standard_normal(m), rng.standard_normal(n)
    s, U, V = _top_k(A, k)
    _, sb, Ub, Vb = _loss_parts(s, U, V, c, x, wu, y, wv)
    G, _ = svd_backward(A, s, U, V, sb, Ub, Vb)
    h = 1e-6
    for (i, j) in [(0, 0), (3, 7), (m - 1, n - 1), (12, 5), (20, 20)]:
        E = np.zeros((m, n))
        E[i, j] = h
        Lp = _loss_parts(*_top_k(A + E, k), c, x, wu, y, wv)[0]
        Lm = _loss_parts(*_top_k(A - E, k), c, x, wu, y, wv)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - G[i, j]) <= 1e-6 * max(1.0, abs(fd)), (i, j, fd, G[i, j])


def test_sum_of_singular_values_gives_u_vt():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((50, 35))
    s, U, V = _top_k(A, 6)
    G, _ = svd_backward(A, s, U, V, sigma_bar=np.ones(6))
    assert np.abs(G - U @ V.T).max() < 1e-13


def test_rank_k_matrix_reduces_to_the_thin_svd_formula():
    rng = np.random.default_rng(2)
    m, n, k = 30, 20, 4
    U0, _ = np.linalg.qr(rng.standard_normal((m, k)))
    V0, _ = np.linalg.qr(rng.standard_normal((n, k)))
    s0 = np.array([4.0, 3.0, 2.0, 1.5])
    A = (U0 * s0) @ V0.T
    s, U, V = _top_k(A, k)
    Ub, Vb = rng.standard_normal((m, k)), rng.standard_normal((n, k))
    G, _ = svd_backward(A, s, U, V, None, Ub, Vb)
    J, K = U.T @ Ub, V.T @ Vb
    F = np.zeros((k, k))
    off = ~np.eye(k, dtype=bool)
    F[off] = 1.0 / (s[None, :] ** 2 - s[:, None] ** 2)[off]
    C = (F * (J - J.T)) * s[None, :] + s[:, None] * (F * (K - K.T))
    thin = U @ C @ V.T + (Ub - U @ J) / s[None, :] @ V.T + U @ ((Vb - V @ K) / s[None, :]).T
    assert np.abs(G - thin).max() < 1e-12


def test_cg_solver_equals_dense_solver_on_sparse_input():
    rng = np.random.default_rng(3)
    A = sp.random(300, 200, density=0.05, random_state=3, format="csr") + sp.eye(300, 200, format="csr")
    k = 5
    s, U, V = _top_k(A.toarray(), k)
    Ub, Vb = rng.standard_normal((300, k)), rng.standard_normal((200, k))
    Gd, _ = svd_backward(A, s, U, V, np.ones(k), Ub, Vb, solver="dense")
    Gc, iters = svd_backward(A, s, U, V, np.ones(k), Ub, Vb, solver="cg")
    assert Gd.shape == (A.nnz,) and len(iters) == 2 * k
    assert np.abs(Gd - Gc).max() <= 1e-9 * np.abs(Gd).max()
    Gfull, _ = svd_backward(A, s, U, V, np.ones(k), Ub, Vb, pattern=False)
    rows = np.repeat(np.arange(300), np.diff(A.indptr))
    assert np.abs(Gfull[rows, A.indices] - Gd).max() < 1e-13 * np.abs(Gd).max()
