"""Seeded synthetic inputs for the truncated-SVD library and its tests.

This module only builds matrices (and nothing of the SVD methods' arithmetic), so
both the CUDA path and the CPU oracle may take their inputs from it.  Every
generator is deterministic in its seed (numpy PCG64).

Workloads (sizes as in the paper's experiments and the library's benchmark):

* ``dense_known_spectrum``: A = U0 diag(sigma) V0^T with U0, V0 the sign-fixed
  Q factors of seeded N(0,1) matrices; the synthetic dense benchmark of Sec. 4.2
  builds its test matrices this way.  Default spectrum sigma_i = 2^(-i/8).
* ``csr_uniform``: m x n CSR, exactly d distinct uniformly drawn columns per row
  (sorted), N(0,1) values: a stand-in for the rectangular SuiteSparse matrices of
  Sec. 4.1 (Table 2), which are not available here.
* ``csr_power_law``: rows with Zipf-distributed degrees and Zipf column
  popularity, U(0,1) values (heavy rows and heavy columns).
* ``dense_householder_spectrum``: A = H_U diag(sigma) H_V^T with H_U, H_V
  products of L seeded Householder reflectors (the large dense workload, whose
  factors are orthogonal "via Householder products"); default sigma_i =
  1/(1+i)^1.5.  ``householder_factors`` gives the reflectors so that a device
  can materialise the same A.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _orthonormal(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """Q factor of a seeded N(0,1) rows x cols matrix, signs fixed so diag(R) > 0."""
    G = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(G)
    return Q * np.where(np.diag(R) < 0, -1.0, 1.0)


def spectrum_pow2(n: int) -> np.ndarray:
    """sigma_i = 2^(-i/8), i = 0..n-1 (sigma_1 = 1, gaps of 2^(1/8))."""
    return 2.0 ** (-np.arange(n) / 8.0)


def spectrum_power(n: int, alpha: float = 1.5) -> np.ndarray:
    """sigma_i = 1 / (1 + i)^alpha, i = 0..n-1."""
    return 1.0 / (1.0 + np.arange(n)) ** alpha


def dense_known_spectrum(m: int, n: int, seed: int = 0, sigma=None):
    """Dense A = U0 diag(sigma) V0^T (m x n, m >= n is not required).

    Returns (A, sigma, U0, V0) with U0 (m x r), V0 (n x r), r = min(m, n), A C-contiguous FP64.
    """
    rng = np.random.default_rng(seed)
    r = min(m, n)
    if sigma is None:
        sigma = spectrum_pow2(r)
    sigma = np.asarray(sigma, dtype=np.float64)
    U0 = _orthonormal(rng, m, r)
    V0 = _orthonormal(rng, n, r)
    A = np.ascontiguousarray((U0 * sigma) @ V0.T)
    return A, sigma, U0, V0


def csr_uniform(m: int, n: int, d: int, seed: int = 1, dtype=np.float64) -> sp.csr_matrix:
    """CSR with exactly ``d`` distinct uniformly random columns per row (sorted), N(0,1) values."""
    if d > n:
        raise ValueError("d > n")
    rng = np.random.default_rng(seed)
    cols = np.sort(rng.integers(0, n, size=(m, d)), axis=1)
    while True:
        dup = np.any(cols[:, 1:] == cols[:, :-1], axis=1) if d > 1 else np.zeros(m, bool)
        bad = np.nonzero(dup)[0]
        if bad.size == 0:
            break
        cols[bad] = np.sort(rng.integers(0, n, size=(bad.size, d)), axis=1)
    vals = rng.standard_normal(m * d).astype(dtype)
    indptr = np.arange(0, m * d + 1, d, dtype=np.int32)
    return sp.csr_matrix((vals, cols.reshape(-1).astype(np.int32), indptr), shape=(m, n))


def _zipf_truncated(rng, size, a, lo, hi):
    """Samples of P(k) proportional to k^-a on the integers lo..hi (inverse CDF on a table)."""
    ks = np.arange(lo, hi + 1, dtype=np.float64)
    w = ks ** (-a)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    return (np.searchsorted(cdf, rng.random(size), side="right") + lo).astype(np.int64)


def _unique_sorted(keys: np.ndarray) -> np.ndarray:
    """Sorted distinct values of an int64 array (sort, then drop repeats)."""
    keys = np.sort(keys)
    if keys.size > 1:
        keep = np.empty(keys.size, dtype=bool)
        keep[0] = True
        np.not_equal(keys[1:], keys[:-1], out=keep[1:])
        keys = keys[keep]
    return keys


def _trim_to_degree(rng, keys, n, deg):
    """Keeps, for every row, at most deg[row] of its keys (the ones with the smallest
    seeded random priorities); keys = row * n + col, sorted."""
    m = deg.size
    r = keys // n
    have = np.bincount(r, minlength=m)
    if not np.any(have > deg):
        return keys
    pri = rng.integers(0, 2 ** 31, size=keys.size, dtype=np.int64)
    order = np.argsort(r * (2 ** 31) + pri)
    ks, rs = keys[order], r[order]
    start = np.searchsorted(rs, np.arange(m))
    rank = np.arange(ks.size) - start[rs]
    return np.sort(ks[rank < deg[rs]])


def csr_power_law(m: int, n: int, target_nnz: int, seed: int = 3, deg_exp: float = 2.1,
                  deg_max: int = 20000, col_exp: float = 1.5, dtype=np.float32) -> sp.csr_matrix:
    """Power-law CSR: row degrees d_i = min(deg_max, ceil(c z_i)), z_i ~ Zipf(deg_exp) on
    [1, deg_max], with c set by bisection so that sum d_i is within 0.5% of ``target_nnz``.
    Columns: each row draws 2 d_i + 4 columns with Zipf(col_exp) popularity over ranks
    (mapped to column ids by a seeded permutation) and keeps distinct ones; rows still
    short of d_i (heavy rows, whose degree approaches the popular support) are topped up
    with uniformly drawn distinct columns.  Values U(0, 1); columns sorted per row.
    """
    rng = np.random.default_rng(seed)
    deg_max = min(deg_max, n)
    z = _zipf_truncated(rng, m, deg_exp, 1, deg_max).astype(np.float64)
    lo, hi = 0.0, float(target_nnz)
    c = 1.0
    for _ in range(200):
        c = 0.5 * (lo + hi)
        tot = np.minimum(deg_max, np.ceil(c * z)).sum()
        if abs(tot - target_nnz) <= 0.005 * target_nnz:
            break
        if tot < target_nnz:
            lo = c
        else:
            hi = c
    deg = np.minimum(deg_max, np.ceil(c * z)).astype(np.int64)
    perm = rng.permutation(n).astype(np.int64)
    cdf = np.cumsum(np.arange(1, n + 1, dtype=np.float64) ** (-col_exp))
    cdf /= cdf[-1]
    cnt = 2 * deg + 4
    rows = np.repeat(np.arange(m, dtype=np.int64), cnt)
    cols = perm[np.minimum(np.searchsorted(cdf, rng.random(rows.size), side="right"), n - 1)]
    keys = _trim_to_degree(rng, _unique_sorted(rows * n + cols), n, deg)
    for _ in range(50):
        need = deg - np.bincount(keys // n, minlength=m)
        short = np.nonzero(need > 0)[0]
        if short.size == 0:
            break
        extra = need[short] + need[short] // 8 + 4
        rows = np.repeat(short, extra)
        new = rows * n + rng.integers(0, n, size=rows.size)
        keys = _trim_to_degree(rng, _unique_sorted(np.concatenate([keys, new])), n, deg)
    have = np.bincount(keys // n, minlength=m)
    indptr = np.zeros(m + 1, dtype=np.int64)
    indptr[1:] = np.cumsum(have)
    vals = rng.random(keys.size).astype(dtype)
    return sp.csr_matrix((vals, (keys % n).astype(np.int32), indptr), shape=(m, n))


def householder_factors(m: int, n: int, seed: int = 2, L: int = 16):
    """Unit vectors of the seeded reflectors: rows u_1..u_L (length m) and v_1..v_L
    (length n), each a normalised N(0,1) draw (u's first, then v's)."""
    rng = np.random.default_rng(seed)
    Uv = rng.standard_normal((L, m))
    Uv /= np.linalg.norm(Uv, axis=1, keepdims=True)
    Vv = rng.standard_normal((L, n))
    Vv /= np.linalg.norm(Vv, axis=1, keepdims=True)
    return Uv, Vv


def reflect_left(X: np.ndarray, Uv: np.ndarray) -> np.ndarray:
    """H_U X with H_U = (I - 2 u_1 u_1^T) ... (I - 2 u_L u_L^T): the reflectors are
    applied from u_L to u_1.  In place on a copy."""
    X = np.array(X, dtype=np.float64, copy=True)
    for u in Uv[::-1]:
        X -= 2.0 * np.outer(u, u @ X)
    return X


def dense_householder_spectrum(m: int, n: int, seed: int = 2, sigma=None, L: int = 16):
    """Dense A = H_U S H_V^T (m x n, FP64, C-contiguous): S is m x n with diagonal
    sigma (default sigma_i = 1/(1+i)^1.5, i = 0..min(m,n)-1), H_U and H_V the
    reflector products of ``householder_factors``.  The singular values are sigma
    and the singular vectors are the leading columns of H_U and H_V.

    Returns (A, sigma, Uv, Vv)."""
    r = min(m, n)
    sigma = spectrum_power(r) if sigma is None else np.asarray(sigma, dtype=np.float64)
    Uv, Vv = householder_factors(m, n, seed, L)
    S = np.zeros((m, n))
    S[np.arange(r), np.arange(r)] = sigma
    # (H_U S) H_V^T = ((H_V (H_U S)^T))^T since H_V is symmetric
    A = reflect_left(reflect_left(S, Uv).T, Vv).T
    return np.ascontiguousarray(A), sigma, Uv, Vv


def reflect_left_torch(X, Uv):
    """Device twin of ``reflect_left`` for a torch tensor X (modified in place)."""
    for i in range(Uv.shape[0] - 1, -1, -1):
        u = Uv[i]
        X.addr_(u, u @ X, alpha=-2.0)
    return X


def dense_householder_spectrum_torch(m: int, n: int, seed: int = 2, sigma=None, L: int = 16, device="cuda"):
    """The matrix of ``dense_householder_spectrum`` built with torch on ``device``
    (same reflectors, same formula; for sizes where numpy would take minutes).

    Returns (A, sigma) with A a C-contiguous float64 torch tensor."""
    import torch
    r = min(m, n)
    sigma = spectrum_power(r) if sigma is None else np.asarray(sigma, dtype=np.float64)
    Uv, Vv = householder_factors(m, n, seed, L)
    S = torch.zeros((m, n), dtype=torch.float64, device=device)
    idx = torch.arange(r, device=device)
    S[idx, idx] = torch.as_tensor(sigma, dtype=torch.float64, device=device)
    reflect_left_torch(S, torch.as_tensor(Uv, device=device))
    At = S.T.contiguous()
    del S
    reflect_left_torch(At, torch.as_tensor(Vv, device=device))
    return At.T.contiguous(), sigma


def spectrum_paper_dense(n: int) -> np.ndarray:
    """Singular values of the paper's dense experiment (Sec. 4.2), read as decreasing:
    sigma_i = 10^(1 - 15 i / (n/2)) for i < n/2 (10 down to ~1e-14), then 1e-14."""
    h = n // 2
    i = np.arange(n)
    return np.where(i < h, 10.0 ** (1.0 - 15.0 * i / h), 1e-14)
