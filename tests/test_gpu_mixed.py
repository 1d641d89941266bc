"""The mixed-precision form (FP32 products and bases, FP64 small algebra, final
FP64 Rayleigh-Ritz step) against FP64 ground truth.

Its arithmetic differs from the oracle's by design, so it is not compared step
by step: the returned triplets must meet the residual tolerance against the
FP64 A, their singular values must agree with the FP64 oracle's converged ones
within the residual bound (|sigma - sigma~| <= max residual), and their
subspaces must lie within tol / relative gap of the dense SVD's.  The measured
errors are printed for the record.
"""

import numpy as np
import pytest

import oracle
import workloads
from helpers import subspace_sin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _np(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


def _check(A, res, k, tol, s_ref, U_ref=None, V_ref=None, relgap=None):
    s, U, V = _np(res.sigma), _np(res.U), _np(res.V)
    resid = max(np.linalg.norm(A @ V - U * s, axis=0).max(), np.linalg.norm(A.T @ U - V * s, axis=0).max()) / s[0]
    assert resid <= tol * 1.0001, resid
    assert abs(res.info["resid_max"] - resid) <= 1e-3 * resid + 1e-15
    err_s = np.max(np.abs(s - s_ref[:k])) / s_ref[0]
    assert err_s <= 2 * tol, err_s
    assert np.abs(U.T @ U - np.eye(k)).max() < 1e-12
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-12
    out = {"resid": resid, "sigma_err": err_s}
    if U_ref is not None:
        out["sin_u"] = subspace_sin(U, U_ref[:, :k])
        out["sin_v"] = subspace_sin(V, V_ref[:, :k])
        assert out["sin_u"] < 10 * tol / relgap and out["sin_v"] < 10 * tol / relgap
    print("mixed vs FP64:", out)
    return out


def test_mixed_blanczos_dense_known_spectrum(tsvd, torch_cuda):
    torch = torch_cuda
    A, s_true, U0, V0 = workloads.dense_known_spectrum(512, 256, seed=0)
    res = tsvd.blanczos(torch.from_numpy(A).cuda(), 10, 16, 4, seed=0, tol=1e-6, precision="mixed")
    assert res.status == 0 and res.info["converged"] == 1
    relgap = (s_true[9] - s_true[10]) / s_true[0]
    _check(A, res, 10, 1e-6, s_true, U0, V0, relgap)


def test_mixed_blanczos_sparse_and_transposed(tsvd, torch_cuda):
    for (m, n) in ((3001, 1200), (700, 2500)):
        A = workloads.csr_uniform(m, n, 11, seed=m)
        res = tsvd.blanczos(tsvd.CsrMatrix.from_scipy(A), 8, 8, 6, seed=3, tol=1e-6, max_restarts=400,
                            precision="mixed")
        assert res.status == 0 and res.info["transposed"] == int(m < n)
        Ut, st_, Vt = np.linalg.svd(A.toarray(), full_matrices=False)
        relgap = (st_[7] - st_[8]) / st_[0]
        _check(A, res, 8, 1e-6, st_, Ut, Vt.T, relgap)


def test_mixed_rsvd_matches_fp64_method(tsvd, torch_cuda):
    torch = torch_cuda
    A, s_true, _, _ = workloads.dense_known_spectrum(512, 256, seed=0)
    At = torch.from_numpy(A).cuda()
    r64 = tsvd.rsvd(At, 10, 10, 2, seed=0)
    r32 = tsvd.rsvd(At, 10, 10, 2, seed=0, precision="mixed")
    s64, s32 = _np(r64.sigma), _np(r32.sigma)
    # same method, FP32 products: the Ritz values move by O(eps_32 * cond), far below the method's own error
    assert np.max(np.abs(s32 - s64)) / s64[0] < 1e-5
    so, _, _, _ = oracle.rsvd(A, 10, 10, 2, seed=0)
    assert np.max(np.abs(s32 - so)) / so[0] < 1e-5


def test_mixed_fp32_valued_input(tsvd, torch_cuda):
    # FP32 values (the power-law workload stores its matrix in FP32): the FP64 steps use them widened exactly
    A = workloads.csr_power_law(4000, 2000, 40_000, seed=3, deg_max=500)
    assert A.dtype == np.float32
    res = tsvd.blanczos(tsvd.CsrMatrix.from_scipy(A), 6, 8, 6, seed=1, tol=1e-6, max_restarts=400,
                        precision="mixed")
    A64 = A.astype(np.float64)
    st_ = np.linalg.svd(A64.toarray(), compute_uv=False)
    assert res.status == 0
    _check(A64, res, 6, 1e-6, st_)
    r64 = tsvd.blanczos(tsvd.CsrMatrix.from_scipy(A), 6, 8, 6, seed=1, tol=1e-6, max_restarts=400)
    _check(A64, r64, 6, 1e-6, st_)


def test_mixed_full_size_sparse_beats_fp64(tsvd, torch_cuda):
    """100,000 x 100,000, 10 nnz/row, k = b = 64, r = 16 to residual 1e-6: the mixed
    form meets the tolerance against the FP64 A and agrees with the FP64 method."""
    A = workloads.csr_uniform(100_000, 100_000, 10, seed=1)
    Ad = tsvd.CsrMatrix.from_scipy(A)
    r32 = tsvd.blanczos(Ad, 64, 64, 16, seed=1, tol=1e-6, precision="mixed")
    r64 = tsvd.blanczos(Ad, 64, 64, 16, seed=1, tol=1e-6)
    assert r32.status == 0 and r64.status == 0
    s32, s64 = _np(r32.sigma), _np(r64.sigma)
    U32, V32 = _np(r32.U), _np(r32.V)
    resid = max(np.linalg.norm(A @ V32 - U32 * s32, axis=0).max(),
                np.linalg.norm(A.T @ U32 - V32 * s32, axis=0).max()) / s32[0]
    assert resid <= 1e-6 * 1.0001
    assert np.max(np.abs(s32 - s64)) / s64[0] <= 2e-6
    print("full size: mixed %.3f s (%d cycles), fp64 %.3f s (%d cycles), sigma diff %.2e, resid %.2e" % (
        r32.info["ms_total"] / 1e3, r32.info["iterations"], r64.info["ms_total"] / 1e3, r64.info["iterations"],
        np.max(np.abs(s32 - s64)) / s64[0], resid))
    assert r32.info["ms_total"] < r64.info["ms_total"]
