"""Why the small SVD tightens its sweep tolerance when LancSVD asks for very small
residuals: a numpy emulation of thick-restart LancSVD (FP64) whose small SVD is a
one-sided Jacobi SVD on the columns of B, rotations skipped when
|g_p . g_q| <= tau |g_p||g_q|, with the right vectors recovered as B^T Ubar Sigma^-1
and re-orthonormalised by QR, as the library's small SVD does.

With thick restart the converged kept Ritz pairs enter B as columns
[sigma_j e_j; G_j] whose couplings lie below tau = d eps: they are never rotated, the
last block rows of their left vectors stay exactly zero, so the Lanczos estimate
reads exactly 0, and the residual stops at a floor set by tau.  tau = sqrt(d) eps
(the level to which a computed coupling is known) lowers that floor; LAPACK's SVD
(no threshold) lower still.

Design check, not a pin of the oracle: the Jacobi SVD is written here."""

import numpy as np

from helpers import LowRankPlusSparse, emulated_thick_lanczos

EPS = 2.0 ** -52


def _jacobi_small_svd(tau_of_d):
    def svd(B):
        d = B.shape[1]
        tau = tau_of_d(d)
        npad = d + (d & 1)
        C = np.hstack([B, np.zeros((B.shape[0], npad - d))])
        order = list(range(npad))
        for _ in range(40):
            rotated = False
            for _ in range(npad - 1):  # one round-robin sweep, disjoint pairs per round
                p, q = np.array(order[:npad // 2]), np.array(order[npad // 2:][::-1])
                a = np.einsum("ij,ij->j", C[:, p], C[:, p])
                b = np.einsum("ij,ij->j", C[:, q], C[:, q])
                g = np.einsum("ij,ij->j", C[:, p], C[:, q])
                act = np.abs(g) > tau * np.sqrt(a * b)
                if act.any():
                    rotated = True
                    zeta = (b[act] - a[act]) / (2.0 * g[act])
                    t = np.where(zeta == 0, 1.0, np.sign(zeta) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta)))
                    c = 1.0 / np.sqrt(1.0 + t * t)
                    s = c * t
                    Cp, Cq = C[:, p[act]].copy(), C[:, q[act]].copy()
                    C[:, p[act]], C[:, q[act]] = c * Cp - s * Cq, s * Cp + c * Cq
                order = [order[0], order[-1]] + order[1:-1]
            if not rotated:
                break
        C = C[:, :d]
        sig = np.linalg.norm(C, axis=0)
        o = np.argsort(-sig)
        sig = sig[o]
        U = C[:, o] / np.where(sig > 0, sig, 1.0)
        V, R = np.linalg.qr((B.T @ U) / np.where(sig > 0, sig, 1.0))
        return U, sig, V * np.sign(np.diag(R))
    return svd


def test_sweep_tolerance_sets_the_floor_of_thick_restart():
    A = LowRankPlusSparse(30_000, seed=4)
    run = lambda svd: emulated_thick_lanczos(A, 8, 16, 8, 48, 6, small_svd=svd)  # noqa: E731
    loose = run(_jacobi_small_svd(lambda d: d * EPS))
    tight = run(_jacobi_small_svd(lambda d: np.sqrt(d) * EPS))
    lapack = run(None)
    # converged kept pairs are left unrotated at tau = d eps: the estimate reads exactly
    # zero while the residual stays above it
    assert any(rho == 0.0 for rho, _ in loose[2:])
    assert loose[-1][1] > 1e-14
    # the tighter tolerance lowers the floor, LAPACK's SVD lower still
    assert tight[-1][1] < 0.7 * loose[-1][1]
    assert lapack[-1][1] < 0.5 * tight[-1][1]
