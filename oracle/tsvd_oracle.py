"""Plain FP64 oracle of RandSVD (Alg. 1), LancSVD (Alg. 2), CGS-QR (Alg. 3),
CholeskyQR2 (Alg. 4) and CGS-CQR2 (Alg. 5) of Tomas, Quintana-Orti and Anzt,
"Fast Truncated SVD of Sparse and Dense Matrices on Graphics Processors".

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): never imported by the
product path, and sharing no code with the CUDA library.

Each step follows the algorithm listing of the paper in its own order; a library
primitive (numpy matrix product, scipy CSR product, LAPACK SVD as in the paper's
Table 1, triangular solve as the paper's TRSM) stands for a single step.  Where
the paper is silent, garbled or inconsistent, the reading taken is named at the
point of use (labels G1..G25, listed with reasons in the design notes):

* G7  CholeskyQR2 returns R = Lbar^T L^T (the product order that satisfies
      Q_out R = Q_in; the listing prints the factors swapped).
* G8  CGS-CQR2 returns H = H + Hbar L^T, the exact accumulation of the two
      projection passes (the listing prints H + Hbar, equal to O(eps)).
* G9  the second Cholesky of CholeskyQR2 factors the second Gram matrix.
* G11 start blocks are i.i.d. N(0,1) (Philox4x32-10 + Box-Muller).
* G17 Cholesky breakdown: a pivot d <= b*eps*max_i W_ii (or non-finite) sends
      the block to column-wise classical Gram-Schmidt with one
      re-orthogonalisation pass (the fallback named in Sec. 3.2).
* G18 the LancSVD restart block is re-orthonormalised with CholeskyQR2.
* G19 singular values sorted descending; every small-SVD right vector and
      every output right vector has its largest-magnitude entry positive.
* G21 LancSVD convergence: rho_j = ||R_r vbar_j[last b rows]||_2 <= tol*sigma_1
      for all j < k, confirmed by the explicit residual.
* G1  residual: max over j of the two one-sided residuals ||A v_j - sigma_j u_j||_2
      and ||A^T u_j - sigma_j v_j||_2, divided by sigma_1 (the second is ~0 by
      construction for both methods, so this equals the first in exact arithmetic).
* G25 thick restart (the improved restart left to future work in Sec. 5), when
      ``keep`` > 0: the leading Ritz pairs are kept, B starts with their singular
      values and the coupling block of the residual block, and the recurrence
      continues from that block.
"""

from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.sparse as sp
from scipy.linalg import solve_triangular

EPS = float(np.finfo(np.float64).eps)

# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
# as 1, 2, 3", SC'11): 10 rounds of the 4x32 Philox round function with the
# published multipliers and Weyl key increments.
# ---------------------------------------------------------------------------
_PHILOX_M = (0xD2511F53, 0xCD9E8D57)
_PHILOX_W = (0x9E3779B9, 0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(counters: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 of every row of ``counters`` (N x 4 uint32) under ``key`` (2 words)."""
    x = [np.asarray(counters[:, i], dtype=np.uint64) for i in range(4)]
    k0, k1 = np.uint64(int(key[0]) & 0xFFFFFFFF), np.uint64(int(key[1]) & 0xFFFFFFFF)
    m0, m1 = np.uint64(_PHILOX_M[0]), np.uint64(_PHILOX_M[1])
    for rnd in range(10):
        if rnd:
            k0 = (k0 + np.uint64(_PHILOX_W[0])) & _MASK32
            k1 = (k1 + np.uint64(_PHILOX_W[1])) & _MASK32
        p0 = x[0] * m0  # < 2^64: exact in uint64
        p1 = x[2] * m1
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
    return np.stack(x, axis=1).astype(np.uint32)


def gaussian_block(rows: int, cols: int, seed: int, stream: int) -> np.ndarray:
    """Row-major ``rows x cols`` block of N(0,1) samples (reading G11).

    Element e = i*cols + j belongs to pair t = e >> 1.  Pair t draws Philox4x32-10
    at counter (t mod 2^32, t >> 32, stream, 0) with key (seed mod 2^32, seed >> 32);
    words (w0, w1) and (w2, w3) give the 53-bit uniforms
    u = ((w_a >> 5) * 2^26 + (w_b >> 6) + 1) * 2^-53 in (0, 1], and Box-Muller
    (Box and Muller 1958) turns (u1, u2) into
    z0 = sqrt(-2 ln u1) cos(2 pi u2) for even e and z1 = sqrt(-2 ln u1) sin(2 pi u2) for odd e.
    """
    n_el = rows * cols
    if n_el == 0:
        return np.zeros((rows, cols))
    n_pairs = (n_el + 1) // 2
    t = np.arange(n_pairs, dtype=np.uint64)
    ctr = np.zeros((n_pairs, 4), dtype=np.uint32)
    ctr[:, 0] = (t & _MASK32).astype(np.uint32)
    ctr[:, 1] = (t >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(stream & 0xFFFFFFFF)
    w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)).astype(np.uint64)
    two53 = 2.0 ** -53
    u1 = (((w[:, 0] >> np.uint64(5)) << np.uint64(26)) + (w[:, 1] >> np.uint64(6)) + np.uint64(1)).astype(np.float64) * two53
    u2 = (((w[:, 2] >> np.uint64(5)) << np.uint64(26)) + (w[:, 3] >> np.uint64(6)) + np.uint64(1)).astype(np.float64) * two53
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * n_pairs)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:n_el].reshape(rows, cols)


# Philox stream ids: one per random draw of the method.
STREAM_RSVD_START = 1      # Alg. 1: random Q_0 (n x l)
STREAM_LANCZOS_START = 2   # Alg. 2 S1: random Qbar_1 (m x b)
STREAM_BREAKDOWN = 0x100   # G17: replacement column t uses stream 0x100 + t


# ---------------------------------------------------------------------------
# Operator view of A: the products S1/S3 of Alg. 1 and S2/S4 of Alg. 2.
# ---------------------------------------------------------------------------
class _Op:
    """A (dense ndarray or scipy CSR) seen as an operator; ``transposed`` swaps roles."""

    def __init__(self, A, transposed: bool):
        self.A = A
        self.t = transposed
        m, n = A.shape
        self.m, self.n = (n, m) if transposed else (m, n)

    def mul(self, X):   # op(A) @ X
        return (self.A.T @ X) if self.t else (self.A @ X)

    def tmul(self, X):  # op(A)^T @ X
        return (self.A @ X) if self.t else (self.A.T @ X)


def as_operator(A):
    """Wrap A so that the methods always see m >= n (Sec. 2: otherwise work on A^T)."""
    if sp.issparse(A):
        A = sp.csr_matrix(A, dtype=np.float64)
    else:
        A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    return _Op(A, transposed=m < n)


# ---------------------------------------------------------------------------
# Small dense building blocks.
# ---------------------------------------------------------------------------
class Breakdown(Exception):
    """Cholesky pivot at or below the breakdown threshold (reading G17)."""


def cholesky_lower(W: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor L of W = L L^T, column by column (Golub & Van Loan Alg. 4.2.1).

    Raises ``Breakdown`` when a pivot d_j = W_jj - sum_k L_jk^2 is non-finite or
    <= b*eps*max_i W_ii (reading G17).
    """
    b = W.shape[0]
    L = np.zeros_like(W)
    wmax = float(np.max(np.diag(W))) if b else 0.0
    thresh = b * EPS * wmax
    if not np.isfinite(wmax) or wmax <= 0.0:
        raise Breakdown("zero or non-finite Gram diagonal")
    for j in range(b):
        d = W[j, j] - L[j, :j] @ L[j, :j]
        if not np.isfinite(d) or d <= thresh:
            raise Breakdown(f"pivot {j}: {d!r} <= {thresh!r}")
        L[j, j] = np.sqrt(d)
        L[j + 1:, j] = (W[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def _right_solve_lt(Q: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Q L^{-T}: the TRSM of Alg. 4 S3/S6 and Alg. 5 S5/S10."""
    # X L^T = Q  <=>  L X^T = Q^T
    return solve_triangular(L, Q.T, lower=True).T


@dataclasses.dataclass
class _Ctx:
    """Per-solve state shared by the orthogonalisation routines."""
    seed: int = 0
    replacements: int = 0   # Philox replacement columns drawn so far (stream 0x100 + t)
    fallbacks: int = 0      # Cholesky breakdowns sent to the CGS2 fallback


def _cgs2_columns(Y: np.ndarray, P: Optional[np.ndarray], ctx: _Ctx):
    """Column-wise classical Gram-Schmidt with one re-orthogonalisation pass (G17).

    Returns (Q, H, R) with Y = P H + Q R, Q^T Q = I, P^T Q = 0.  A column whose
    norm after both passes is below 1e-10 of its norm before them is numerically
    dependent: it keeps R_jj = that norm and its direction is replaced by a
    Philox N(0,1) column (stream 0x100 + t) orthogonalised the same way.
    """
    q, b = Y.shape
    s = 0 if P is None else P.shape[1]
    Q = np.zeros((q, b))
    H = np.zeros((s, b))
    R = np.zeros((b, b))

    def project(v, j, hcol, rcol):
        for _ in range(2):
            if s:
                h = P.T @ v
                v = v - P @ h
                if hcol is not None:
                    hcol += h
            if j:
                c = Q[:, :j].T @ v
                v = v - Q[:, :j] @ c
                if rcol is not None:
                    rcol += c
        return v

    for j in range(b):
        v = Y[:, j].copy()
        nrm0 = np.linalg.norm(v)
        hcol = np.zeros(s)
        rcol = np.zeros(j)
        v = project(v, j, hcol, rcol)
        nrm = np.linalg.norm(v)
        H[:, j] = hcol
        R[:j, j] = rcol
        R[j, j] = nrm
        if not (nrm > 1e-10 * nrm0) or nrm0 == 0.0:
            z = gaussian_block(q, 1, ctx.seed, STREAM_BREAKDOWN + ctx.replacements)[:, 0]
            ctx.replacements += 1
            z = project(z, j, None, None)
            v = z
            nrm = np.linalg.norm(z)
        Q[:, j] = v / nrm
    return Q, H, R


def cholqr2(Y: np.ndarray, ctx: Optional[_Ctx] = None):
    """Alg. 4 (CholeskyQR2): returns (Q, R) with Y = Q R, Q^T Q = I, R upper triangular."""
    ctx = ctx or _Ctx()
    try:
        Q = Y.copy()
        W = Q.T @ Q                       # S1
        L = cholesky_lower(W)             # S2
        Q = _right_solve_lt(Q, L)         # S3
        Wbar = Q.T @ Q                    # S4
        Lbar = cholesky_lower(Wbar)       # S5 (reading G9: factor Wbar)
        Q = _right_solve_lt(Q, Lbar)      # S6
        R = Lbar.T @ L.T                  # S7 (reading G7)
        return Q, R
    except Breakdown:
        ctx.fallbacks += 1
        Q, _, R = _cgs2_columns(Y, None, ctx)
        return Q, R


def cgs_cqr2(Y: np.ndarray, P: np.ndarray, ctx: Optional[_Ctx] = None):
    """Alg. 5 (CGS-CQR2): returns (Q, H, R) with Y = P H + Q R, P^T Q = 0, Q^T Q = I."""
    ctx = ctx or _Ctx()
    if P is None or P.shape[1] == 0:
        Q, R = cholqr2(Y, ctx)
        return Q, np.zeros((0, Y.shape[1])), R
    try:
        Q = Y.copy()
        H = P.T @ Q                       # S1
        Q = Q - P @ H                     # S2
        W = Q.T @ Q                       # S3
        L = cholesky_lower(W)             # S4
        Q = _right_solve_lt(Q, L)         # S5
        Hbar = P.T @ Q                    # S6
        Q = Q - P @ Hbar                  # S7
        W = Q.T @ Q                       # S8
        Lbar = cholesky_lower(W)          # S9
        Q = _right_solve_lt(Q, Lbar)      # S10
        R = Lbar.T @ L.T                  # S11 (reading G7)
        H = H + Hbar @ L.T                # S12 (reading G8)
        return Q, H, R
    except Breakdown:
        ctx.fallbacks += 1
        return _cgs2_columns(Y, P, ctx)


def cgs_qr(Y: np.ndarray, b: int, ctx: Optional[_Ctx] = None):
    """Alg. 3 (CGS-QR): QR of a q x r block by column blocks of width b.

    The last block is narrower when b does not divide r.  Returns (Q, R), R upper
    triangular r x r assembled by column blocks [H_j; R_j].
    """
    ctx = ctx or _Ctx()
    q, r = Y.shape
    b = max(1, min(b, r))
    Q = np.zeros((q, r))
    R = np.zeros((r, r))
    Q[:, :b], R[:b, :b] = cholqr2(Y[:, :b], ctx)                 # S1
    for c0 in range(b, r, b):                                    # S2
        c1 = min(c0 + b, r)
        Qj, Hj, Rj = cgs_cqr2(Y[:, c0:c1], Q[:, :c0], ctx)
        Q[:, c0:c1] = Qj
        R[:c0, c0:c1] = Hj
        R[c0:c1, c0:c1] = Rj
    return Q, R


def _fix_signs(Ubar: np.ndarray, Vbar: np.ndarray):
    """G19: flip (ubar_j, vbar_j) so that the largest-magnitude entry of vbar_j is positive."""
    idx = np.argmax(np.abs(Vbar), axis=0)
    sgn = np.where(Vbar[idx, np.arange(Vbar.shape[1])] < 0, -1.0, 1.0)
    return Ubar * sgn, Vbar * sgn


def small_svd(B: np.ndarray):
    """SVD of the small projected matrix (Alg. 1 S5, Alg. 2 S6; LAPACK GESVD in the paper).

    Returns (Ubar, sigma, Vbar) with B = Ubar diag(sigma) Vbar^T, sigma descending,
    signs fixed as in G19.
    """
    Ub, s, Vt = np.linalg.svd(B)
    order = np.argsort(-s, kind="stable")
    Ub, s, Vb = Ub[:, order], s[order], Vt.T[:, order]
    Ub, Vb = _fix_signs(Ub, Vb)
    return Ub, s, Vb


def _output_signs(U: np.ndarray, V: np.ndarray):
    """G19 on the returned vectors: largest-magnitude entry of each v_j positive."""
    return _fix_signs(U, V)


# ---------------------------------------------------------------------------
# Drivers.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class OracleInfo:
    iterations: int = 0
    restarts: int = 0
    breakdowns: int = 0
    converged: bool = False
    rho_hist: list = dataclasses.field(default_factory=list)
    resid_max: float = float("nan")
    transposed: bool = False


def _resid_max(op, sigma, U, V):
    """max_j of both one-sided residuals over sigma_1 (reading G1), in the m >= n orientation."""
    if not sigma[0] > 0:
        return float("nan")
    av = np.linalg.norm(op.mul(V) - U * sigma, axis=0)
    atu = np.linalg.norm(op.tmul(U) - V * sigma, axis=0)
    return float(max(np.max(av), np.max(atu)) / sigma[0])


def residuals(A, sigma, U, V):
    """Per-triplet residual norms for the metric of Sec. 4 (reading G1).

    Returns a dict with ``av`` = ||A v_j - sigma_j u_j||_2 and ``atu`` =
    ||A^T u_j - sigma_j v_j||_2 (arrays of length k).
    """
    av = A @ V - U * sigma
    atu = A.T @ U - V * sigma
    return {"av": np.linalg.norm(av, axis=0), "atu": np.linalg.norm(atu, axis=0)}


def rsvd(A, k: int, p: int, q: int, seed: int = 0, qr_block: int = 0,
         start_block: Optional[np.ndarray] = None):
    """Alg. 1 (RandSVD) with block width l = k + p and q + 1 iterations of S1-S4.

    ``start_block`` (n x l) replaces the Philox draw when given.  Returns
    (sigma[k], U[m x k], V[n x k], OracleInfo).
    """
    op = as_operator(A)
    m, n = op.m, op.n
    ell = k + p
    if not (1 <= k <= ell <= n):
        raise ValueError("need 1 <= k <= k+p <= min(m, n)")
    b_qr = ell if qr_block <= 0 else min(qr_block, ell)
    ctx = _Ctx(seed=seed)
    Qn = gaussian_block(n, ell, seed, STREAM_RSVD_START) if start_block is None \
        else np.array(start_block, dtype=np.float64, copy=True)       # Q_0 (G23: raw)
    info = OracleInfo(transposed=op.t)
    Qm = None
    R = None
    for _ in range(q + 1):
        Ybar = op.mul(Qn)                        # S1
        Qm, _ = cgs_qr(Ybar, b_qr, ctx)          # S2
        Y = op.tmul(Qm)                          # S3
        Qn, R = cgs_qr(Y, b_qr, ctx)             # S4
        info.iterations += 1
    Ub, s, Vb = small_svd(R)                     # S5
    U = Qm @ Vb[:, :k]                           # S6
    V = Qn @ Ub[:, :k]                           # S7
    sigma = s[:k].copy()
    U, V = _output_signs(U, V)
    info.breakdowns = ctx.fallbacks
    info.resid_max = _resid_max(op, sigma, U, V)
    if op.t:
        U, V = V, U
    return sigma, U, V, info


def blanczos(A, k: int, b: int, r: int, seed: int = 0, tol: float = 1e-6,
             max_restarts: int = 50, start_block: Optional[np.ndarray] = None,
             return_state: bool = False, keep: int = 0):
    """Alg. 2 (LancSVD): block Golub-Kahan-Lanczos with full two-sided block
    re-orthogonalisation (reading G6) and basic restart (Golub, Luk, Overton 1981).

    ``r`` blocks of width ``b`` give a Krylov dimension r*b; the restart loop stops
    when the residual test of G21 passes or after ``max_restarts`` restarts.
    ``start_block`` (m x b) replaces the Philox draw when given.  Returns
    (sigma[k], U[m x k], V[n x k], OracleInfo) and, with ``return_state``, the
    last cycle's (P, Pbar, B, Rr, Qbar_{r+1}) in the orientation m >= n.

    ``keep`` = s > 0 selects the thick (augmented) restart that the paper names as
    future work (Sec. 5; Baglama and Reichel's augmented restarting): a cycle
    ending with A P = Pbar B + Qbar R E^T and B = Ubar S Vbar^T keeps the s leading
    Ritz pairs, P~ = P Vbar_s and Pbar~ = Pbar Ubar_s, for which
        A P~ = Pbar~ S_s + Qbar G,   A^T Pbar~ = P~ S_s,   G = R E^T Vbar_s,
    and continues the same recurrence from the residual block Qbar: the next right
    block is A^T Qbar orthogonalised against P~ (its coefficients there are G^T),
    then the usual steps.  The new cycle's basis is [P~, Q'_1 ... Q'_r'] and
    [Pbar~, Qbar, Qbar'_2 ...] with r' = (r b - s) / b blocks, and its B is
        [ S_s   0    0  ... ]
        [ G     L'_1 0  ... ]
        [ 0     R'_1 L'_2 ..]   (block lower bidiagonal after the first s columns),
    so the same Ritz, residual-estimate and output steps apply.  The first cycle
    is the basic method's.
    """
    op = as_operator(A)
    m, n = op.m, op.n
    rb = r * b
    if not (b >= 1 and r >= 1 and 1 <= k <= rb <= n):
        raise ValueError("need b, r >= 1 and 1 <= k <= r*b <= min(m, n)")
    if keep and not (k <= keep and keep + b <= rb):
        raise ValueError("thick restart needs k <= keep and keep + b <= r*b")
    ctx = _Ctx(seed=seed)
    info = OracleInfo(transposed=op.t)
    Omega = gaussian_block(m, b, seed, STREAM_LANCZOS_START) if start_block is None \
        else np.array(start_block, dtype=np.float64, copy=True)
    Qbar1, _ = cholqr2(Omega, ctx)                               # S1
    s0 = 0                        # Ritz pairs kept from the previous cycle (thick restart)
    Pk = Pbk = Sk = Qlast = None
    while True:
        nblk = r if s0 == 0 else (rb - s0) // b
        d = s0 + nblk * b
        P = np.zeros((n, d))
        Pbar = np.zeros((m, d))
        B = np.zeros((d, d))
        if s0 == 0:
            Pbar[:, :b] = Qbar1
        else:
            P[:, :s0] = Pk
            Pbar[:, :s0] = Pbk
            B[:s0, :s0] = np.diag(Sk)
            Pbar[:, s0:s0 + b] = Qlast
        Rr = None
        for i in range(nblk):
            c0, c1 = s0 + i * b, s0 + (i + 1) * b
            Qi = op.tmul(Pbar[:, c0:c1])                          # S2
            if c0 == 0:
                Qi, T = cholqr2(Qi, ctx)                          # S3a
            else:
                Qi, H, T = cgs_cqr2(Qi, P[:, :c0], ctx)           # S3b
                if i == 0:                                        # coupling with the kept pairs
                    B[c0:c1, :s0] = H.T
            P[:, c0:c1] = Qi
            B[c0:c1, c0:c1] = T.T                                 # L_i
            Qn = op.mul(Qi)                                       # S4
            Qn, _, Ri = cgs_cqr2(Qn, Pbar[:, :c1], ctx)           # S5
            if i + 1 < nblk:
                Pbar[:, c1:c1 + b] = Qn
                B[c1:c1 + b, c0:c1] = Ri                          # R_i
            else:
                Rr, Qlast = Ri, Qn
        info.iterations += 1
        Ub, s, Vb = small_svd(B)                                  # S6
        rho = np.linalg.norm(Rr @ Vb[d - b:d, :k], axis=0)        # G21
        info.rho_hist.append(float(np.max(rho) / s[0]) if s[0] > 0 else float("nan"))
        done = info.rho_hist[-1] <= tol
        if done or info.restarts >= max_restarts:
            U = Pbar @ Ub[:, :k]                                  # S9
            V = P @ Vb[:, :k]                                     # S8 (reading G2)
            sigma = s[:k].copy()
            info.resid_max = _resid_max(op, sigma, U, V)
            if (done and info.resid_max <= tol) or info.restarts >= max_restarts:
                info.converged = bool(info.resid_max <= tol)
                break
        info.restarts += 1
        if keep:
            Pk, Pbk, Sk = P @ Vb[:, :keep], Pbar @ Ub[:, :keep], s[:keep].copy()
            s0 = keep
        else:
            Qbar1, _ = cholqr2(Pbar @ Ub[:, :b], ctx)             # S7 (reading G18)
    U, V = _output_signs(U, V)
    info.breakdowns = ctx.fallbacks
    if op.t:
        U, V = V, U
    out = (sigma, U, V, info)
    if return_state:
        out = out + ((P, Pbar, B, Rr, Qlast),)
    return out
