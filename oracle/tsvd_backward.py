"""FP64 CPU oracle of the gradient of a loss on the k leading singular triplets
with respect to A (the differentiation pattern built on top of the paper's
methods; the paper itself has no backward pass).

TEST INFRASTRUCTURE ONLY (see the package header): nothing in the product path
may import or call it.

Given A (m x n), its k leading triplets (sigma, U, V) and the adjoints
sigma_bar = dL/dsigma, U_bar = dL/dU, V_bar = dL/dV of a scalar loss L, the
derivative of the truncated SVD (the k leading triplets only; the other
singular values of A need not be zero) gives

    dL/dA = U C V^T + Y S V^T + U (A^T Y)^T + U S Z^T + (A Z) V^T

with S = diag(sigma), J = U^T U_bar, K = V^T V_bar,
F_ij = 1 / (sigma_j^2 - sigma_i^2) for i != j (0 on the diagonal),
C = (F o (J - J^T)) S + diag(sigma_bar) + S (F o (K - K^T)),
and the columns of Y and Z solving, on the orthogonal complements of span(U)
and span(V),
    (sigma_i^2 I - A A^T) y_i = (I - U U^T) u_bar_i,
    (sigma_i^2 I - A^T A) z_i = (I - V V^T) v_bar_i.
Those operators map each complement into itself and are positive definite there
when sigma_k > sigma_{k+1}, so the solves are well posed.  The derivation: the
exact relations A v_i = sigma_i u_i, A^T u_i = sigma_i v_i differentiate to
(sigma_i^2 I - A A^T) du_i = sigma_i dA v_i + A dA^T u_i - 2 sigma_i dsigma_i u_i;
projecting on the complement and taking the adjoint gives the Y terms (the Z
terms likewise from the second relation); inside span(U), span(V) the classical
formula of the thin SVD applies.  When A has rank exactly k the complement
operators are sigma_i^2 I and the terms reduce to the familiar
(I - U U^T) U_bar S^-1 V^T + U S^-1 V_bar^T (I - V V^T).

In factored form dL/dA = Lf Rf^T with Lf = [U C + Y S + A Z, U] and
Rf = [V, A^T Y + Z S] (rank 2k), so a sparse A needs only its pattern's entries.
"""

from __future__ import annotations

from typing import Optional

import numpy as np
import scipy.sparse as sp


def _dense_complement_solve(G: np.ndarray, shift: float, Q: np.ndarray, r: np.ndarray) -> np.ndarray:
    """y in the complement of span(Q) with (shift I - G) y = r (r in that complement):
    written out on an orthonormal basis N of the complement, y = N (N^T (shift I - G) N)^-1 N^T r."""
    full, _ = np.linalg.qr(np.concatenate([Q, np.eye(Q.shape[0])], axis=1))
    N = full[:, Q.shape[1]:Q.shape[0]]
    M = shift * np.eye(N.shape[1]) - N.T @ G @ N
    return N @ np.linalg.solve(M, N.T @ r)


def _cg_complement_solve(apply_G, shift: float, Q: np.ndarray, r: np.ndarray, tol: float, maxiter: int):
    """The same solve by conjugate gradients on x -> P (shift x - G x), P = I - Q Q^T
    (symmetric positive definite on the complement), from x = 0."""
    P = lambda x: x - Q @ (Q.T @ x)  # noqa: E731
    b = P(r)
    x = np.zeros_like(b)
    res = b.copy()
    p = res.copy()
    rr = float(res @ res)
    bn = np.sqrt(float(b @ b))
    it = 0
    while np.sqrt(rr) > tol * bn and it < maxiter:
        Ap = P(shift * p - apply_G(p))
        alpha = rr / float(p @ Ap)
        x += alpha * p
        res -= alpha * Ap
        rr_new = float(res @ res)
        p = res + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return P(x), it


def svd_backward(A, sigma, U, V, sigma_bar=None, U_bar=None, V_bar=None, pattern: bool = True,
                 solver: str = "dense", cg_tol: float = 1e-14, cg_maxiter: int = 20000):
    """dL/dA for a loss of the k leading triplets (formula in the module header).

    A: dense ndarray or scipy sparse, m x n.  sigma (k), U (m x k), V (n x k): the
    leading triplets of A.  sigma_bar (k), U_bar (m x k), V_bar (n x k): adjoints
    (None = 0).  ``solver``: "dense" (the complement solves written out with dense
    linear algebra; small cases) or "cg".  Returns the gradient: for sparse A and
    ``pattern`` its values on A's nonzeros in CSR order, else the dense m x n
    matrix.  Also returns the CG iteration counts (empty for "dense").
    """
    sparse = sp.issparse(A)
    A = sp.csr_matrix(A, dtype=np.float64) if sparse else np.asarray(A, dtype=np.float64)
    m, n = A.shape
    s = np.asarray(sigma, dtype=np.float64)
    k = s.size
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    sb = np.zeros(k) if sigma_bar is None else np.asarray(sigma_bar, dtype=np.float64)
    Ub = np.zeros((m, k)) if U_bar is None else np.asarray(U_bar, dtype=np.float64)
    Vb = np.zeros((n, k)) if V_bar is None else np.asarray(V_bar, dtype=np.float64)
    J = U.T @ Ub
    K = V.T @ Vb
    s2 = s * s
    D = s2[None, :] - s2[:, None]                      # D_ij = s_j^2 - s_i^2
    off = ~np.eye(k, dtype=bool)
    F = np.zeros((k, k))
    F[off] = 1.0 / D[off]
    C = (F * (J - J.T)) * s[None, :] + np.diag(sb) + s[:, None] * (F * (K - K.T))
    rU = Ub - U @ J                                     # (I - U U^T) U_bar
    rV = Vb - V @ K                                     # (I - V V^T) V_bar
    Y = np.zeros((m, k))
    Z = np.zeros((n, k))
    iters = []
    if solver == "dense":
        Ad = A.toarray() if sparse else A
        AAt, AtA = Ad @ Ad.T, Ad.T @ Ad
        for i in range(k):
            if np.any(rU[:, i]):
                Y[:, i] = _dense_complement_solve(AAt, s2[i], U, rU[:, i])
            if np.any(rV[:, i]):
                Z[:, i] = _dense_complement_solve(AtA, s2[i], V, rV[:, i])
    elif solver == "cg":
        for i in range(k):
            if np.any(rU[:, i]):
                Y[:, i], it = _cg_complement_solve(lambda x: A @ (A.T @ x), s2[i], U, rU[:, i], cg_tol, cg_maxiter)
                iters.append(it)
            if np.any(rV[:, i]):
                Z[:, i], it = _cg_complement_solve(lambda x: A.T @ (A @ x), s2[i], V, rV[:, i], cg_tol, cg_maxiter)
                iters.append(it)
    else:
        raise ValueError("solver must be 'dense' or 'cg'")
    Lf = np.concatenate([U @ C + Y * s[None, :] + A @ Z, U], axis=1)
    Rf = np.concatenate([V, A.T @ Y + Z * s[None, :]], axis=1)
    if sparse and pattern:
        rows = np.repeat(np.arange(m), np.diff(A.indptr))
        grad = np.einsum("ij,ij->i", Lf[rows], Rf[A.indices])
    else:
        grad = Lf @ Rf.T
    return grad, iters
