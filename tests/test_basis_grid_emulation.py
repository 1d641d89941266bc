"""Why the restart and Ritz products of the FP64 method slice the Lanczos basis
afresh: a numpy emulation of thick-restart LancSVD in FP64 in which the basis
enters chosen products as fixed-point values on one grid for all rows, as the
rows-layout digit planes of an orthonormal basis hold it (a fixed exponent for
every row).  The library's grid unit is 2^-54; here a coarser unit, 2^-44, makes the
effect visible at a CPU-sized matrix (the floor scales with the unit, sqrt(n) and
sqrt(r b)).

* exact: the solve converges to rounding level;
* basis on the grid in the restart products (P Vbar_s, Pbar Ubar_s, U, V): the
  kept Ritz vectors carry the grid's error, the next cycle takes them as exact, and
  the residual stops at a floor while the Lanczos estimate keeps falling;
* basis on the grid in the CGS-CQR2 products: a lower floor of the same origin.

Design check, not a pin of the oracle: the emulation is written here."""

import numpy as np

import workloads

UNIT = 2.0 ** -44


def _grid(X):
    return np.round(X / UNIT) * UNIT


class _LowRankPlusSparse:
    """A = S + Us diag(sg) Vs^T: a flat random sparse bulk (norm about 10) and eight
    separated leading singular values (20 .. 25), so that a few cycles converge."""

    def __init__(self, n, seed):
        self.S = workloads.csr_uniform(n, n, 25, seed=seed)
        rng = np.random.default_rng(seed + 1)
        self.Us = np.linalg.qr(rng.standard_normal((n, 8)))[0]
        self.Vs = np.linalg.qr(rng.standard_normal((n, 8)))[0]
        self.sg = np.linspace(25.0, 20.0, 8)[:, None]

    def mul(self, X):
        return self.S @ X + self.Us @ (self.sg * (self.Vs.T @ X))

    def tmul(self, X):
        return self.S.T @ X + self.Vs @ (self.sg * (self.Us.T @ X))


def _orth(Y, P, on_grid):
    if on_grid and P.shape[1]:
        P = _grid(P)
    for _ in range(2):
        if P.shape[1]:
            Y = Y - P @ (P.T @ Y)
    return np.linalg.qr(Y)


def _thick(A, n, k, b, r, keep, cycles, restart_grid, orth_grid):
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
            Qi, T = _orth(Y, P[:, :c0], orth_grid)
            if i == 0 and s0:
                B[c0:c1, :s0] = H.T                         # coupling block
            P[:, c0:c1], B[c0:c1, c0:c1] = Qi, T.T
            Qn, Ri = _orth(A.mul(Qi), Pb[:, :c1], orth_grid)
            if i + 1 < nblk:
                Pb[:, c1:c1 + b], B[c1:c1 + b, c0:c1] = Qn, Ri
            else:
                Rr, Qlast = Ri, Qn
        Ub, s, Vbt = np.linalg.svd(B)
        Vb = Vbt.T
        rho = np.max(np.linalg.norm(Rr @ Vb[d - b:, :k], axis=0)) / s[0]
        Pm, Pbm = (_grid(P), _grid(Pb)) if restart_grid else (P, Pb)
        U, V, sg = Pbm @ Ub[:, :k], Pm @ Vb[:, :k], s[:k]
        res = max(np.linalg.norm(A.mul(V) - U * sg, axis=0).max(),
                  np.linalg.norm(A.tmul(U) - V * sg, axis=0).max()) / sg[0]
        hist.append((rho, res))
        Pk, Pbk, Sk, s0 = Pm @ Vb[:, :keep], Pbm @ Ub[:, :keep], s[:keep], keep
    return hist


def test_basis_on_a_fixed_grid_in_the_restart_products_sets_a_residual_floor():
    n = 30_000
    A = _LowRankPlusSparse(n, seed=4)
    run = lambda rg, og: _thick(A, n, 8, 16, 8, 48, 5, rg, og)  # noqa: E731
    exact, restart, orth = run(False, False), run(True, False), run(False, True)
    res = lambda h: [r for _, r in h]  # noqa: E731
    # exact arithmetic of the products: converged to rounding level
    assert res(exact)[-1] < 3e-14
    # grid in the restart products: a flat floor far above it, while the Lanczos
    # estimate (computed from B, which takes the kept vectors as exact) keeps falling
    assert res(restart)[-1] > 100 * res(exact)[-1]
    assert max(res(restart)[-3:]) < 1.5 * min(res(restart)[-3:])
    assert restart[-1][0] < 1e-3 * res(restart)[-1]
    # grid in the CGS-CQR2 products: also above exact arithmetic
    assert res(orth)[-1] > 10 * res(exact)[-1]
