"""Gradient of a loss on the k leading triplets with respect to A
(tsvd_svd_backward and the differentiable truncated_svd) against the oracle's FP64
gradient and against central finite differences.

Losses: sum(sigma) + ||U^T X||_F^2 (the large sparse workload's loss: the
within-subspace terms cancel and everything sits in the complement solves), and
a loss with per-vector weights on U and V, whose within-subspace coupling terms
do not cancel."""

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _np(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


def _adjoints(s, U, V, X, wu, y, wv):
    """sigma_bar, U_bar, V_bar of L = sum s + sum_i wu_i ||X^T u_i||^2 + sum_i wv_i (v_i^T y)^2."""
    XtU = X.T @ U
    return np.ones_like(s), 2 * X @ (XtU * wu[None, :]), 2 * np.outer(y, wv * (V.T @ y))


@pytest.mark.parametrize("kind", ["csr", "dense", "csr_wide"])
def test_backward_matches_oracle_gradient(tsvd, torch_cuda, kind):
    torch = torch_cuda
    k = 6
    if kind == "dense":
        A, _, _, _ = workloads.dense_known_spectrum(300, 200, seed=5, sigma=1.0 / (1.0 + np.arange(200)) ** 1.2)
        Ad = torch.from_numpy(A).cuda()
    else:
        m, n = (2000, 1500) if kind == "csr" else (1200, 2500)
        A = workloads.csr_uniform(m, n, 12, seed=7)
        Ad = tsvd.CsrMatrix.from_scipy(A)
    res = tsvd.blanczos(Ad, k, 8, 8, seed=1, tol=1e-11, max_restarts=400)
    assert res.status == 0
    s, U, V = _np(res.sigma), _np(res.U), _np(res.V)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((U.shape[0], 4))
    y = rng.standard_normal(V.shape[0])
    wu, wv = rng.uniform(0.5, 2.0, k), rng.uniform(0.5, 2.0, k)
    sb, Ub, Vb = _adjoints(s, U, V, X, wu, y, wv)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    grad, info = tsvd.svd_backward(Ad, res.sigma, res.U, res.V, t(sb), t(Ub), t(Vb), cg_tol=1e-12)
    ref, _ = oracle.svd_backward(A, s, U, V, sb, Ub, Vb, solver="cg", cg_tol=1e-13)
    g = _np(grad)
    assert g.shape == ref.shape
    err = np.abs(g - ref).max() / np.abs(ref).max()
    print(f"backward {kind}: max rel err {err:.2e}, CG iterations {info['cg_iters_u']}/{info['cg_iters_v']}")
    assert err < 1e-8, err


def test_sum_of_sigma_gradient_is_u_vt_on_the_pattern(tsvd, torch_cuda):
    A = workloads.csr_uniform(3000, 2000, 9, seed=2)
    Ad = tsvd.CsrMatrix.from_scipy(A)
    res = tsvd.blanczos(Ad, 5, 8, 6, seed=0, tol=1e-10, max_restarts=400)
    import torch
    grad, info = tsvd.svd_backward(Ad, res.sigma, res.U, res.V, torch.ones(5, dtype=torch.float64, device="cuda"))
    U, V = _np(res.U), _np(res.V)
    rows = np.repeat(np.arange(3000), np.diff(A.indptr))
    ref = np.einsum("ij,ij->i", U[rows], V[A.indices])
    assert np.abs(_np(grad) - ref).max() < 1e-14 * 10
    assert info["cg_iters_u"] == 0 and info["cg_iters_v"] == 0


def _fd_check(tsvd, torch, A, k, b, r, X, n_picks, seed):
    """Autograd gradient of sum(sigma) + ||U^T X||^2 against central differences.

    The perturbed losses are evaluated after a fixed number of restart cycles from
    the same start block (the count the unperturbed solve needed to reach a
    residual of 1e-13), which makes the computed loss a smooth function of A: a
    tolerance-stopped solve could stop after a different number of cycles on the
    two sides, and its convergence error (amplified by 1/gap in U) would not
    cancel in the difference."""
    Ad = tsvd.CsrMatrix.from_scipy(A)
    ref = tsvd.blanczos(Ad, k, b, r, seed=0, tol=1e-13, max_restarts=1000)
    assert ref.status == 0
    cycles = ref.info["iterations"]
    vals = Ad.val.clone().requires_grad_(True)
    Av = tsvd.CsrMatrix(Ad.row_ptr, Ad.col_idx, vals, Ad.shape)
    s, U, V = tsvd.truncated_svd(Av, k, b, r, tol=1e-13, max_restarts=1000)
    loss = s.sum() + ((U.T @ X) ** 2).sum()
    loss.backward()
    g = _np(vals.grad)

    def L(v):
        Ap = tsvd.CsrMatrix(Ad.row_ptr, Ad.col_idx, v, Ad.shape)
        r_ = tsvd.blanczos(Ap, k, b, r, seed=0, tol=0.0, max_restarts=cycles - 1)
        assert r_.info["iterations"] == cycles
        return float(r_.sigma.sum() + ((r_.U.T @ X) ** 2).sum())

    picks = np.random.default_rng(seed).choice(A.nnz, n_picks, replace=False)
    base = Ad.val.detach()
    scale = np.abs(g).max()
    worst = 0.0
    for e in picks:
        h = 1e-4 * max(1.0, abs(float(base[e])))
        vp, vm = base.clone(), base.clone()
        vp[e] += h
        vm[e] -= h
        fd = (L(vp) - L(vm)) / (2 * h)
        worst = max(worst, abs(fd - g[e]) / max(abs(fd), 1e-2 * scale))
    return worst, cycles, ref.info["resid_max"]


def test_truncated_svd_autograd_central_differences(tsvd, torch_cuda):
    """2,000 x 2,000 sparse (10 nnz/row), k = b = 8, r = 8: 20 random nonzeros."""
    torch = torch_cuda
    A = workloads.csr_uniform(2000, 2000, 10, seed=11)
    X = torch.from_numpy(np.random.default_rng(1).standard_normal((2000, 4))).cuda()
    worst, cycles, resid = _fd_check(tsvd, torch, A, 8, 8, 8, X, 20, 5)
    print(f"autograd vs central differences (20 nonzeros, {cycles} cycles, resid {resid:.1e}): "
          f"worst relative difference {worst:.2e}")
    assert worst < 1e-5, worst


def test_backward_full_size_200k(tsvd, torch_cuda):
    """200,000 x 200,000 CSR, 5M nnz (25 uniform columns per row), N(0,1) FP64,
    k = b = 32, r = 16 (thick restart keeping 128), loss sum(sigma) + ||U^T X||^2
    with a seeded 200,000 x 32 X.  The top of this spectrum is tightly clustered
    (relative gap sigma_k - sigma_k+1 of order 1e-4), so the forward is converged to
    a residual of 1e-13 (12 cycles; the FP64 oracle's Lanczos estimate is 1.6e-14
    after 12 cycles on this matrix): a gradient built from triplets of residual e is
    accurate to about e / gap^2.  Each perturbed solve costs seconds, so the central difference is taken
    along one random +-1 direction supported on 100 random nonzeros (its
    directional derivative is the sum of those 100 gradient entries with the
    signs), plus 3 single nonzeros, each at the unperturbed solve's fixed cycle
    count.  The FP32-valued copy of the matrix must give the same gradient
    (returned in FP32)."""
    torch = torch_cuda
    A = workloads.csr_uniform(200_000, 200_000, 25, seed=4)
    X = torch.from_numpy(np.random.default_rng(4).standard_normal((200_000, 32))).cuda()
    k, b, r, keep, tol = 32, 32, 16, 128, 1e-13
    import time
    Ad = tsvd.CsrMatrix.from_scipy(A)
    t0 = time.perf_counter()
    vals = Ad.val.clone().requires_grad_(True)
    Av = tsvd.CsrMatrix(Ad.row_ptr, Ad.col_idx, vals, Ad.shape)
    s, U, V = tsvd.truncated_svd(Av, k, b, r, tol=tol, max_restarts=200, restart_keep=keep)
    loss = s.sum() + ((U.T @ X) ** 2).sum()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g = _np(vals.grad)
    ref = tsvd.blanczos(Ad, k, b, r, seed=0, tol=tol, max_restarts=200, restart_keep=keep)
    cycles = ref.info["iterations"]

    def L(v):
        Ap = tsvd.CsrMatrix(Ad.row_ptr, Ad.col_idx, v, Ad.shape)
        r_ = tsvd.blanczos(Ap, k, b, r, seed=0, tol=0.0, max_restarts=cycles - 1, restart_keep=keep)
        return float(r_.sigma.sum() + ((r_.U.T @ X) ** 2).sum())

    rng = np.random.default_rng(100)
    picks = rng.choice(A.nnz, 100, replace=False)
    signs = rng.choice([-1.0, 1.0], 100)
    base = Ad.val.detach()
    h = 1e-4
    d = torch.zeros_like(base)
    d[torch.from_numpy(picks).cuda()] = torch.from_numpy(signs).cuda()
    fd_dir = (L(base + h * d) - L(base - h * d)) / (2 * h)
    g_dir = float(np.dot(g[picks], signs))
    rel_dir = abs(fd_dir - g_dir) / abs(fd_dir)
    worst = rel_dir
    for e in picks[:3]:
        vp, vm = base.clone(), base.clone()
        vp[e] += h
        vm[e] -= h
        fd = (L(vp) - L(vm)) / (2 * h)
        worst = max(worst, abs(fd - g[e]) / max(abs(fd), 1e-2 * np.abs(g).max()))
    A32 = tsvd.CsrMatrix.from_scipy(A.astype(np.float32))
    v32 = A32.val.clone().requires_grad_(True)
    s32, U32, V32 = tsvd.truncated_svd(tsvd.CsrMatrix(A32.row_ptr, A32.col_idx, v32, A32.shape), k, b, r,
                                       tol=tol, max_restarts=200, restart_keep=keep)
    (s32.sum() + ((U32.T @ X) ** 2).sum()).backward()
    assert v32.grad.dtype == torch.float32
    d32 = float((v32.grad.double() - vals.grad).abs().max() / vals.grad.abs().max())
    print(f"200k backward: forward {(t1 - t0):.2f} s ({cycles} cycles), backward {(t2 - t1) * 1e3:.0f} ms; "
          f"directional central difference on 100 nonzeros: {fd_dir:.6e} vs {g_dir:.6e} (rel {rel_dir:.1e}); "
          f"worst incl. 3 single entries {worst:.1e}; FP32-valued copy vs FP64: {d32:.1e}")
    # the gap that conditions the gradient: sigma_k - sigma_{k+1}, from a solve for k + 1
    nxt = tsvd.blanczos(Ad, k + 1, b, r, seed=0, tol=1e-10, max_restarts=200, restart_keep=keep)
    gap = float((nxt.sigma[k - 1] - nxt.sigma[k]) / nxt.sigma[0])
    bound = ref.info["resid_max"] / gap ** 2
    print(f"   forward resid {ref.info['resid_max']:.1e}, relative gap at k {gap:.1e}, "
          f"conditioning bound resid / gap^2 = {bound:.1e}")
    assert ref.info["resid_max"] <= tol
    assert worst < 1e-5, (worst, bound)
    assert d32 < 1e-3
