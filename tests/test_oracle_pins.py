"""Pins of the FP64 oracle to facts fixed outside the oracle itself.

Each test ties one oracle function to a published value, a closed form, a
textbook method implemented independently here, an invariant of the algebra,
or a library routine run as a cross-check (never to a retyped copy of the
oracle's own formula).  CPU only.
"""

import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle
import workloads
from oracle import tsvd_oracle as O

from helpers import subspace_sin

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox / start block
def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answer_vectors():
    kat = _kat()
    assert len(kat) == 3
    for ctr, key, out in kat:
        got = oracle.philox4x32_10(np.array([ctr], dtype=np.uint32), key)[0]
        assert [int(x) for x in got] == out


def test_gaussian_block_box_muller_structure():
    # elements 2t and 2t+1 share the radius: z0^2 + z1^2 = -2 ln u1 with u1 from words (w0, w1)
    seed, stream = 12345, 7
    z = oracle.gaussian_block(1, 64, seed, stream)[0]
    t = np.arange(32, dtype=np.uint64)
    ctr = np.zeros((32, 4), dtype=np.uint32)
    ctr[:, 0] = t.astype(np.uint32)
    ctr[:, 2] = stream
    w = oracle.philox4x32_10(ctr, (seed, 0)).astype(np.uint64)
    k = ((w[:, 0] >> np.uint64(5)) << np.uint64(26)) + (w[:, 1] >> np.uint64(6))
    u1 = (k.astype(np.float64) + 1.0) * 2.0 ** -53
    np.testing.assert_allclose(z[0::2] ** 2 + z[1::2] ** 2, -2.0 * np.log(u1), rtol=1e-13)


def test_gaussian_block_moments_and_layout():
    z = oracle.gaussian_block(500, 2000, 3, 1)
    n = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    # fourth moment of N(0,1) is 3
    assert abs((z ** 4).mean() - 3.0) < 0.05
    # row-major element order: a 1 x (r*c) draw reshaped equals the r x c draw
    a = oracle.gaussian_block(7, 9, 11, 2)
    b = oracle.gaussian_block(1, 63, 11, 2).reshape(7, 9)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(oracle.gaussian_block(4, 4, 11, 2), oracle.gaussian_block(4, 4, 11, 3))


# ---------------------------------------------------------------- Cholesky / CholeskyQR2
def _rand_cond(rng, q, b, cond):
    U, _ = np.linalg.qr(rng.standard_normal((q, b)))
    V, _ = np.linalg.qr(rng.standard_normal((b, b)))
    s = np.logspace(0, -np.log10(cond), b)
    return (U * s) @ V.T


def test_cholesky_matches_lapack_and_detects_breakdown():
    rng = np.random.default_rng(0)
    for b in (1, 2, 7, 64):
        G = rng.standard_normal((b + 5, b))
        W = G.T @ G
        np.testing.assert_allclose(oracle.cholesky_lower(W), np.linalg.cholesky(W), rtol=1e-12, atol=1e-13)
    W = np.ones((3, 3))  # rank 1
    with pytest.raises(O.Breakdown):
        oracle.cholesky_lower(W)
    with pytest.raises(O.Breakdown):
        oracle.cholesky_lower(np.diag([1.0, -1.0]))


@pytest.mark.parametrize("cond", [1.0, 1e3, 1e6])
def test_cholqr2_equals_householder_qr(cond):
    rng = np.random.default_rng(1)
    Y = _rand_cond(rng, 300, 17, cond)
    Q, R = oracle.cholqr2(Y)
    # uniqueness of the QR factorisation with positive diag(R) (Golub & Van Loan Thm. 5.2.3)
    Qh, Rh = np.linalg.qr(Y)
    sgn = np.sign(np.diag(Rh))
    Qh, Rh = Qh * sgn, Rh * sgn[:, None]
    np.testing.assert_allclose(Q, Qh, atol=1e-13 * cond)
    np.testing.assert_allclose(R, Rh, atol=1e-13 * np.abs(Rh).max())
    assert np.abs(Q.T @ Q - np.eye(17)).max() < 1e-14
    assert np.abs(Q @ R - Y).max() < 1e-14 * np.abs(Y).max() * 10
    assert np.all(np.diag(R) > 0) and np.abs(np.tril(R, -1)).max() == 0.0


def test_cholqr2_breakdown_falls_back_to_cgs2():
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((200, 6))
    Y[:, 3] = Y[:, 0] + 2.0 * Y[:, 1]          # exactly dependent column
    Y[:, 5] = 0.0                              # zero column
    ctx = O._Ctx(seed=5)
    Q, R = oracle.cholqr2(Y, ctx)
    assert ctx.fallbacks == 1 and ctx.replacements == 2
    assert np.abs(Q.T @ Q - np.eye(6)).max() < 1e-14
    assert np.abs(Q @ R - Y).max() < 1e-12
    assert abs(R[3, 3]) < 1e-12 and R[5, 5] == 0.0


def test_cgs_cqr2_invariants():
    rng = np.random.default_rng(3)
    P, _ = np.linalg.qr(rng.standard_normal((500, 40)))
    Y = rng.standard_normal((500, 16)) + P @ rng.standard_normal((40, 16)) * 10
    Q, H, R = oracle.cgs_cqr2(Y, P)
    assert np.abs(P.T @ Q).max() < 1e-14
    assert np.abs(Q.T @ Q - np.eye(16)).max() < 1e-14
    assert np.abs(P @ H + Q @ R - Y).max() < 1e-13 * np.abs(Y).max()
    # H is the projection coefficient P^T Y (exact for orthonormal P)
    np.testing.assert_allclose(H, P.T @ Y, atol=1e-12)
    # Q R is then the QR of (I - P P^T) Y, unique with positive diag(R)
    Qh, Rh = np.linalg.qr(Y - P @ (P.T @ Y))
    sgn = np.sign(np.diag(Rh))
    np.testing.assert_allclose(R, Rh * sgn[:, None], atol=1e-12)


@pytest.mark.parametrize("b", [1, 4, 5, 24])
def test_cgs_qr_equals_householder_qr(b):
    rng = np.random.default_rng(4)
    Y = _rand_cond(rng, 400, 24, 1e4)
    Q, R = oracle.cgs_qr(Y, b)
    Qh, Rh = np.linalg.qr(Y)
    sgn = np.sign(np.diag(Rh))
    np.testing.assert_allclose(R, Rh * sgn[:, None], atol=1e-12 * np.abs(Rh).max())
    np.testing.assert_allclose(Q, Qh * sgn, atol=1e-10)
    assert np.abs(Q.T @ Q - np.eye(24)).max() < 1e-14


# ---------------------------------------------------------------- small SVD
def test_small_svd_known_spectrum_and_conventions():
    rng = np.random.default_rng(5)
    n = 40
    s_true = np.exp(rng.uniform(-5, 2, n))
    U0, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V0, _ = np.linalg.qr(rng.standard_normal((n, n)))
    B = (U0 * s_true) @ V0.T
    Ub, s, Vb = oracle.small_svd(B)
    np.testing.assert_allclose(s, np.sort(s_true)[::-1], rtol=1e-13)
    assert np.all(np.diff(s) <= 0)
    np.testing.assert_allclose((Ub * s) @ Vb.T, B, atol=1e-13 * s[0])
    idx = np.argmax(np.abs(Vb), axis=0)
    assert np.all(Vb[idx, np.arange(n)] > 0)
    # diagonal input: singular values are |d| sorted, vectors are signed unit vectors
    d = np.array([3.0, -7.0, 0.5, 2.0])
    Ub, s, Vb = oracle.small_svd(np.diag(d))
    np.testing.assert_allclose(s, [7.0, 3.0, 2.0, 0.5])
    np.testing.assert_allclose(np.abs(Vb), np.eye(4)[:, [1, 0, 3, 2]])


# ---------------------------------------------------------------- RandSVD
def test_rsvd_full_width_is_exact():
    # l = n: Q_p spans R^n, so A = Qbar Qbar^T A exactly and the SVD is exact
    A, s_true, U0, V0 = workloads.dense_known_spectrum(120, 60, seed=7)
    sig, U, V, info = oracle.rsvd(A, 10, 50, 0, seed=3)
    np.testing.assert_allclose(sig, s_true[:10], rtol=1e-12)
    assert info.resid_max < 1e-13


def test_rsvd_identity_and_monotone_power_iterations():
    A, s_true, U0, V0 = workloads.dense_known_spectrum(512, 256, seed=0)
    errs = []
    for q in range(5):
        sig, U, V, info = oracle.rsvd(A, 10, 10, q, seed=0)
        # A^T u_j = sigma_j v_j holds by construction (A^T Qbar = Q R, Sec. 2.1)
        assert np.abs(A.T @ U - V * sig).max() < 1e-13
        assert np.abs(U.T @ U - np.eye(10)).max() < 1e-13
        assert np.abs(V.T @ V - np.eye(10)).max() < 1e-13
        errs.append(np.max(np.abs(sig - s_true[:10]) / s_true[:10]))
    assert all(errs[i + 1] < errs[i] for i in range(4)), errs
    # subspace iteration on (A A^T)^q A: the relative error of sigma_k follows
    # (sigma_{l+1}/sigma_k)^(2(2q+1)) (Halko, Martinsson, Tropp 2011, Sec. 4.5); a
    # missing or extra product per trip would change the exponent by 2 per trip
    rate = s_true[20] / s_true[9]
    for q, e in enumerate(errs):
        assert 0.2 * rate ** (2 * (2 * q + 1)) < e < 1.5 * rate ** (2 * (2 * q + 1)), (q, e)


def test_rsvd_transposed_input():
    # m < n runs the method on A^T (Sec. 2): identical to calling it on A^T with U and V swapped
    A, s_true, U0, V0 = workloads.dense_known_spectrum(80, 200, seed=2)
    sig, U, V, info = oracle.rsvd(A, 5, 10, 3, seed=1)
    assert info.transposed and U.shape == (80, 5) and V.shape == (200, 5)
    sig_t, U_t, V_t, info_t = oracle.rsvd(np.ascontiguousarray(A.T), 5, 10, 3, seed=1)
    assert not info_t.transposed
    np.testing.assert_array_equal(sig, sig_t)
    rate = (s_true[15] / s_true[4]) ** 14
    np.testing.assert_allclose(sig, s_true[:5], rtol=5 * rate)
    # signs: the convention is applied in the transposed orientation, so columns agree up to sign
    np.testing.assert_allclose(np.abs(U), np.abs(V_t), atol=1e-14)
    np.testing.assert_allclose(np.abs(V), np.abs(U_t), atol=1e-14)


# ---------------------------------------------------------------- LancSVD
def _gkl_full_reorth(A, u1, steps):
    """Textbook Golub-Kahan-Lanczos lower bidiagonalisation (Golub & Kahan 1965),
    single vector, with full re-orthogonalisation of both vector sequences."""
    m, n = A.shape
    Us, Vs, alphas, betas = [u1 / np.linalg.norm(u1)], [], [], []
    for i in range(steps):
        v = A.T @ Us[-1]
        if Vs:
            v -= betas[-1] * Vs[-1]
        for _ in range(2):
            for x in Vs:
                v -= (x @ v) * x
        a = np.linalg.norm(v)
        v /= a
        Vs.append(v)
        alphas.append(a)
        w = A @ v - a * Us[-1]
        for _ in range(2):
            for x in Us:
                w -= (x @ w) * x
        bt = np.linalg.norm(w)
        Us.append(w / bt)
        betas.append(bt)
    B = np.diag(alphas) + np.diag(betas[:-1], -1)
    return B, betas[-1]


def test_blanczos_b1_is_golub_kahan_lanczos():
    A = workloads.csr_uniform(300, 200, 6, seed=9).toarray()
    r = 25
    Om = O.gaussian_block(300, 1, 4, O.STREAM_LANCZOS_START)
    sig, U, V, info, (P, Pbar, B, Rr, Ql) = oracle.blanczos(A, 3, 1, r, seed=4, tol=0.0, max_restarts=0,
                                                            return_state=True)
    Bg, beta_last = _gkl_full_reorth(A, Om[:, 0], r)
    np.testing.assert_allclose(B, Bg, atol=1e-11)
    assert abs(Rr[0, 0] - beta_last) < 1e-11


def test_blanczos_lanczos_relations_and_structure():
    A = workloads.csr_uniform(900, 600, 12, seed=11)
    b, r = 8, 6
    sig, U, V, info, (P, Pbar, B, Rr, Ql) = oracle.blanczos(A, 5, b, r, seed=2, tol=0.0, max_restarts=1,
                                                            return_state=True)
    Ad = A.toarray()
    nA = np.linalg.norm(Ad, 2)
    rb = r * b
    assert np.abs(P.T @ P - np.eye(rb)).max() < 1e-13
    assert np.abs(Pbar.T @ Pbar - np.eye(rb)).max() < 1e-13
    # A^T Pbar = P B^T and A P = Pbar B + Qbar_{r+1} R_r E_r^T (Sec. 2.2)
    assert np.abs(Ad.T @ Pbar - P @ B.T).max() < 1e-12 * nA
    E = np.zeros((rb, b))
    E[rb - b:, :] = np.eye(b)
    assert np.abs(Ad @ P - Pbar @ B - Ql @ Rr @ E.T).max() < 1e-12 * nA
    # lower block bidiagonal: L_i lower triangular on the diagonal, R_i upper triangular below it
    for i in range(r):
        for j in range(r):
            blk = B[i * b:(i + 1) * b, j * b:(j + 1) * b]
            if i == j:
                assert np.abs(np.triu(blk, 1)).max() == 0.0 and np.all(np.diag(blk) > 0)
            elif i == j + 1:
                assert np.abs(np.tril(blk, -1)).max() == 0.0
            else:
                assert np.abs(blk).max() == 0.0


def test_blanczos_residual_estimate_equals_explicit_residual():
    A = workloads.csr_uniform(700, 500, 9, seed=12)
    sig, U, V, info = oracle.blanczos(A, 6, 6, 5, seed=3, tol=0.0, max_restarts=2)
    explicit = np.linalg.norm(A @ V - U * sig, axis=0).max() / sig[0]
    assert abs(info.rho_hist[-1] - explicit) < 1e-10 * max(1.0, explicit) + 1e-14


def test_blanczos_exhausted_square_is_exact():
    # square A with r*b = n: Pbar spans R^n, R_r = 0 and B is an exact orthogonal transform of A
    A, s_true, _, _ = workloads.dense_known_spectrum(48, 48, seed=3)
    sig, U, V, info = oracle.blanczos(A, 6, 4, 12, seed=1, tol=1e-10, max_restarts=0)
    np.testing.assert_allclose(sig, s_true[:6], rtol=1e-13)
    assert info.converged and info.resid_max < 1e-12


def test_blanczos_converges_to_known_spectrum_cfg_small():
    A, s_true, U0, V0 = workloads.dense_known_spectrum(512, 256, seed=0)
    sig, U, V, info = oracle.blanczos(A, 10, 16, 4, seed=0, tol=1e-10, max_restarts=50)
    assert info.converged
    np.testing.assert_allclose(sig, s_true[:10], rtol=1e-12)
    # principal angles between the computed and true singular subspaces
    for X, X0 in ((U, U0[:, :10]), (V, V0[:, :10])):
        assert subspace_sin(X, X0) < 1e-10
    # the sign convention: largest-magnitude entry of each v_j positive
    idx = np.argmax(np.abs(V), axis=0)
    assert np.all(V[idx, np.arange(10)] > 0)


def test_blanczos_transposed_and_against_scipy_svds():
    A = workloads.csr_uniform(400, 1000, 15, seed=13)
    sig, U, V, info = oracle.blanczos(A, 4, 4, 10, seed=5, tol=1e-9, max_restarts=200)
    assert info.transposed and info.converged
    s_ref = np.linalg.svd(A.toarray(), compute_uv=False)[:4]
    np.testing.assert_allclose(sig, s_ref, rtol=1e-9)
    assert np.linalg.norm(A @ V - U * sig, axis=0).max() <= 1e-9 * sig[0] * 1.01


def test_blanczos_rank_deficient_uses_fallback():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((60, 3)) @ rng.standard_normal((3, 40))   # rank 3
    sig, U, V, info = oracle.blanczos(A, 3, 2, 4, seed=2, tol=1e-10, max_restarts=5)
    s_ref = np.linalg.svd(A, compute_uv=False)[:3]
    np.testing.assert_allclose(sig, s_ref, rtol=1e-10)
    assert info.breakdowns >= 1


# ---------------------------------------------------------------- residual helper and inputs
def test_residuals_zero_on_exact_triplets():
    A, s_true, U0, V0 = workloads.dense_known_spectrum(50, 30, seed=1)
    r = oracle.residuals(A, s_true[:5], U0[:, :5], V0[:, :5])
    assert r["av"].max() < 1e-14 and r["atu"].max() < 1e-14


def test_workload_generators():
    A = workloads.csr_uniform(1000, 500, 10, seed=1)
    assert A.nnz == 10000 and np.all(np.diff(A.indptr) == 10)
    for i in range(0, 1000, 97):
        c = A.indices[A.indptr[i]:A.indptr[i + 1]]
        assert np.all(np.diff(c) > 0) and c.min() >= 0 and c.max() < 500
    B = workloads.csr_uniform(1000, 500, 10, seed=1)
    assert np.array_equal(A.indices, B.indices) and np.array_equal(A.data, B.data)
    A, s, U0, V0 = workloads.dense_known_spectrum(64, 32, seed=4)
    np.testing.assert_allclose(np.linalg.svd(A, compute_uv=False), s, rtol=1e-13)
    np.testing.assert_allclose(s, 2.0 ** (-np.arange(32) / 8))


def test_householder_workload_has_its_spectrum_and_vectors():
    """The large dense workload's generator: singular values exactly sigma, singular
    vectors the leading columns of the reflector products, and the device twin of
    the construction (tests/helpers.py) gives the same matrix."""
    m, n = 300, 200
    A, s, Uv, Vv = workloads.dense_householder_spectrum(m, n, seed=2, L=16)
    np.testing.assert_allclose(s, 1.0 / (1.0 + np.arange(n)) ** 1.5)
    np.testing.assert_allclose(np.linalg.svd(A, compute_uv=False), s, rtol=1e-12, atol=1e-15)
    HU = workloads.reflect_left(np.eye(m), Uv)
    HV = workloads.reflect_left(np.eye(n), Vv)
    assert np.abs(HU.T @ HU - np.eye(m)).max() < 1e-13
    np.testing.assert_allclose(A, (HU[:, :n] * s) @ HV.T, atol=1e-14)
    # A v_j = sigma_j u_j for the generator's own vectors
    assert np.abs(A @ HV[:, :5] - HU[:, :5] * s[:5]).max() < 1e-14
    At, _ = workloads.dense_householder_spectrum_torch(m, n, seed=2, L=16, device="cpu")
    assert np.abs(At.numpy() - A).max() < 1e-14


# ------------------------------------------------------------------ thick restart (keep > 0)
def test_blanczos_thick_restart_relations_and_coupling_block():
    """After a thick restart the cycle still satisfies A P = Pbar B + Qbar R E^T and
    A^T Pbar = P B^T with orthonormal bases; B is diag(S_s) on the kept pairs, the
    coupling block below them equals G = R_r E^T Vbar_s of the previous cycle, and
    everything else outside the block lower bidiagonal part is zero."""
    A = workloads.csr_uniform(700, 400, 9, seed=11).toarray()
    k, b, r, keep = 6, 6, 5, 12
    # cycle 1 alone, then cycles 1-2 from the same start
    _, _, _, _, st1 = O.blanczos(A, k, b, r, seed=4, tol=0.0, max_restarts=0, keep=keep, return_state=True)
    _, _, _, info2, st2 = O.blanczos(A, k, b, r, seed=4, tol=0.0, max_restarts=1, keep=keep, return_state=True)
    assert info2.iterations == 2
    P1, Pb1, B1, R1, Q1 = st1
    P, Pb, B, R, Q = st2
    d = P.shape[1]
    assert d == keep + ((r * b - keep) // b) * b
    E = np.zeros((d, b))
    E[d - b:, :] = np.eye(b)
    assert np.abs(A @ P - Pb @ B - Q @ R @ E.T).max() < 1e-12 * np.abs(A).max() * d
    assert np.abs(A.T @ Pb - P @ B.T).max() < 1e-12 * np.abs(A).max() * d
    assert np.abs(P.T @ P - np.eye(d)).max() < 1e-13 and np.abs(Pb.T @ Pb - np.eye(d)).max() < 1e-13
    Ub1, s1, Vb1 = np.linalg.svd(B1)
    np.testing.assert_allclose(np.diag(B[:keep, :keep]), s1[:keep], rtol=1e-13)
    assert np.abs(B[:keep, :keep] - np.diag(np.diag(B[:keep, :keep]))).max() == 0.0
    G = R1 @ Vb1.T[B1.shape[0] - b:, :keep]          # R_r E^T Vbar_s (signs of the SVD vectors...)
    # singular vectors are unique up to sign: compare |G| column by column
    np.testing.assert_allclose(np.abs(B[keep:keep + b, :keep]), np.abs(G), atol=1e-12 * s1[0])
    assert np.abs(B[:keep, keep:]).max() == 0.0 and np.abs(B[keep + b:, :keep]).max() == 0.0
    for i in range(keep, d, b):  # nothing above the block diagonal in the bidiagonal part
        assert np.abs(B[i:i + b, i + b:]).max(initial=0.0) == 0.0
    # the kept right Ritz vectors span P Vbar_s of cycle 1
    assert subspace_sin(P[:, :keep], P1 @ Vb1.T[:, :keep]) < 1e-12


def test_blanczos_thick_restart_converges_to_known_spectrum_with_fewer_products():
    A, s_true, U0, V0 = workloads.dense_known_spectrum(512, 256, seed=0)
    tol = 1e-8
    s, U, V, info = O.blanczos(A, 10, 16, 4, seed=0, tol=tol, max_restarts=200, keep=32)
    assert info.converged and info.resid_max <= tol
    assert np.max(np.abs(s - s_true[:10])) <= 2 * tol * s_true[0]
    relgap = (s_true[9] - s_true[10]) / s_true[0]
    assert subspace_sin(U, U0[:, :10]) < 10 * tol / relgap and subspace_sin(V, V0[:, :10]) < 10 * tol / relgap
    assert np.abs(A.T @ U - V * s).max() < 1e-13  # exact by construction, as for basic restart
    # A-products: cycle 1 has r blocks, later cycles (r b - keep) / b; fewer in total than basic restart
    _, _, _, ib = O.blanczos(A, 10, 16, 4, seed=0, tol=tol, max_restarts=200)
    thick_blocks = 4 + (info.iterations - 1) * ((64 - 32) // 16)
    assert thick_blocks < 4 * ib.iterations, (thick_blocks, 4 * ib.iterations)


def test_power_law_generator_statistics():
    """The power-law workload's structure: row degrees follow Zipf(2.1) (the slope of
    their complementary distribution over degrees 60..2000 gives the exponent within
    0.1), every row has exactly its target degree of distinct sorted columns, the
    degree cap holds, and column popularity is heavy-tailed: the top column is in more
    rows than Zipf(1.5)'s first-rank probability 1/zeta(1.5) = 0.383 alone gives (it is
    drawn ~2d times per row), and the rank-frequency slope over ranks 2..2000 is between
    -1.6 and -1.1 (flatter than -1.5 because a column appears at most once per row)."""
    A = workloads.csr_power_law(200_000, 100_000, 5_000_000, seed=3)
    assert abs(A.nnz - 5_000_000) <= 0.005 * 5_000_000
    deg = np.diff(A.indptr)
    assert deg.max() <= 20_000 and deg.min() >= 1
    for i in range(0, 200_000, 9973):
        c = A.indices[A.indptr[i]:A.indptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    d = np.sort(deg)[::-1]
    ranks = np.arange(1, d.size + 1)
    sel = (d >= 60) & (d <= 2000)
    exponent = 1.0 - np.polyfit(np.log(d[sel]), np.log(ranks[sel]), 1)[0]
    assert abs(exponent - 2.1) < 0.1, exponent
    col = np.sort(np.bincount(A.indices, minlength=100_000))[::-1]
    assert col[0] / 200_000 > 0.383
    r = np.arange(1, col.size + 1)
    sel = (r >= 2) & (r <= 2000)
    slope = np.polyfit(np.log(r[sel]), np.log(col[sel]), 1)[0]
    assert -1.6 < slope < -1.1, slope
    assert A.dtype == np.float32 and 0.0 <= A.data.min() and A.data.max() <= 1.0  # U(0,1) rounded to FP32
