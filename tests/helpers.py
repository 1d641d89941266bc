"""Shared numerical helpers of the test suite (test code only)."""

import numpy as np


def subspace_sin(X, X0):
    """sin of the largest principal angle between span(X) and span(X0), both with
    orthonormal columns: ||(I - X0 X0^T) X||_2, accurate down to rounding level
    (unlike sqrt(1 - cos^2))."""
    X = np.asarray(X, dtype=np.float64)
    X0 = np.asarray(X0, dtype=np.float64)
    return float(np.linalg.norm(X - X0 @ (X0.T @ X), 2))



def separated_prefix(s, rel_gap=1e-4):
    """The largest j < len(s) with (s[j-1] - s[j]) / s[0] >= rel_gap (0 if none):
    span of the first j singular vectors is well conditioned (its sensitivity to a
    perturbation of size e is about e / gap), unlike a subspace whose last value
    is nearly tied with the next."""
    s = np.asarray(s, dtype=np.float64)
    gaps = (s[:-1] - s[1:]) / s[0]
    idx = np.nonzero(gaps >= rel_gap)[0]
    return int(idx[-1] + 1) if idx.size else 0


def residual_gap_bound(sin_u, sin_v, sig_rel=0.0):
    """How far two residual maxima ||A v - s u|| / s_1 of nearby triplets may differ:
    |delta| <= ||A|| ||dv|| + |ds| + s ||du|| (in units of s_1), with ||dv||, ||du||
    at most 2 sin(angle) for sign-fixed unit vectors."""
    return 2.0 * (sin_u + sin_v) + sig_rel + 1e-12


class LowRankPlusSparse:
    """A = S + Us diag(sg) Vs^T (n x n): a flat random sparse bulk (25 N(0,1) entries a
    row, norm about 10) and eight separated leading singular values (25 down to 20),
    so that a thick-restart solve converges in a few cycles.  mul / tmul give A X and
    A^T X."""

    def __init__(self, n, seed):
        import workloads
        self.n = n
        self.S = workloads.csr_uniform(n, n, 25, seed=seed)
        rng = np.random.default_rng(seed + 1)
        self.Us = np.linalg.qr(rng.standard_normal((n, 8)))[0]
        self.Vs = np.linalg.qr(rng.standard_normal((n, 8)))[0]
        self.sg = np.linspace(25.0, 20.0, 8)[:, None]

    def mul(self, X):
        return self.S @ X + self.Us @ (self.sg * (self.Vs.T @ X))

    def tmul(self, X):
        return self.S.T @ X + self.Vs @ (self.sg * (self.Us.T @ X))


def emulated_thick_lanczos(A, k, b, r, keep, cycles, small_svd=None, restart_basis=None, orth_basis=None):
    """Thick-restart block Lanczos (FP64 numpy, the thick-restart reading of the
    library) with hooks for the design checks: ``small_svd(B) -> (Ubar, s, Vbar)``
    (default LAPACK), and the basis as the restart/Ritz products (``restart_basis``)
    and the CGS-CQR2 products (``orth_basis``) see it (default: exact).  Returns per
    cycle (rho, residual): the Lanczos estimate and max of both one-sided residuals
    of the k leading triplets, both over sigma_1."""
    n = A.n
    same = lambda X: X  # noqa: E731
    restart_basis = restart_basis or same
    orth_basis = orth_basis or same
    if small_svd is None:
        def small_svd(B):
            u, s, vt = np.linalg.svd(B)
            return u, s, vt.T

    def orth(Y, P):
        P = orth_basis(P) if P.shape[1] else P
        for _ in range(2):
            if P.shape[1]:
                Y = Y - P @ (P.T @ Y)
        return np.linalg.qr(Y)

    rb = r * b
    Q1 = np.linalg.qr(np.random.default_rng(0).standard_normal((n, b)))[0]
    s0, Pk, Pbk, Sk, Qlast = 0, None, None, None, None
    hist = []
    for _ in range(cycles):
        nblk = r if s0 == 0 else (rb - s0) // b
        d = s0 + nblk * b
        P, Pb, B = np.zeros((n, d)), np.zeros((n, d)), np.zeros((d, d))
        if s0 == 0:
            Pb[:, :b] = Q1
        else:
            P[:, :s0], Pb[:, :s0] = Pk, Pbk
            B[:s0, :s0] = np.diag(Sk)
            Pb[:, s0:s0 + b] = Qlast
        for i in range(nblk):
            c0, c1 = s0 + i * b, s0 + (i + 1) * b
            Y = A.tmul(Pb[:, c0:c1])
            H = P[:, :c0].T @ Y
            Qi, T = orth(Y, P[:, :c0])
            if i == 0 and s0:
                B[c0:c1, :s0] = H.T                         # coupling block
            P[:, c0:c1], B[c0:c1, c0:c1] = Qi, T.T
            Qn, Ri = orth(A.mul(Qi), Pb[:, :c1])
            if i + 1 < nblk:
                Pb[:, c1:c1 + b], B[c1:c1 + b, c0:c1] = Qn, Ri
            else:
                Rr, Qlast = Ri, Qn
        Ub, s, Vb = small_svd(B)
        rho = np.max(np.linalg.norm(Rr @ Vb[d - b:, :k], axis=0)) / s[0]
        Pm, Pbm = restart_basis(P), restart_basis(Pb)
        U, V, sg = Pbm @ Ub[:, :k], Pm @ Vb[:, :k], s[:k]
        res = max(np.linalg.norm(A.mul(V) - U * sg, axis=0).max(),
                  np.linalg.norm(A.tmul(U) - V * sg, axis=0).max()) / sg[0]
        hist.append((rho, res))
        Pk, Pbk, Sk, s0 = Pm @ Vb[:, :keep], Pbm @ Ub[:, :keep], s[:keep], keep
    return hist
