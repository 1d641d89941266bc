"""Thick (augmented) restart of LancSVD (restart_keep = s > 0) against the oracle's
thick restart: element-wise on fixed cycle counts (sigma 1e-10, subspaces 1e-8),
converged against the dense SVD, and at full size against the basic method."""

import numpy as np
import pytest

import oracle
import workloads
from helpers import residual_gap_bound, subspace_sin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _np(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


@pytest.mark.parametrize("m,n,keep", [(3001, 1200, 16), (700, 2500, 10), (3001, 1200, 21)])
def test_thick_restart_matches_oracle_fixed_cycles(tsvd, torch_cuda, m, n, keep):
    A = workloads.csr_uniform(m, n, 11, seed=m)
    res = tsvd.blanczos(tsvd.CsrMatrix.from_scipy(A), 8, 8, 5, seed=3, tol=0.0, max_restarts=2, restart_keep=keep)
    so, Uo, Vo, info = oracle.blanczos(A, 8, 8, 5, seed=3, tol=0.0, max_restarts=2, keep=keep)
    assert res.info["iterations"] == 3 == info.iterations
    s, U, V = _np(res.sigma), _np(res.U), _np(res.V)
    np.testing.assert_allclose(s, so, rtol=1e-10)
    su, sv = subspace_sin(U, Uo), subspace_sin(V, Vo)
    assert su < 1e-8 and sv < 1e-8, (su, sv)
    assert abs(res.info["resid_max"] - info.resid_max) <= residual_gap_bound(su, sv, 1e-10)


def test_thick_restart_converges_dense_known_spectrum(tsvd, torch_cuda):
    torch = torch_cuda
    A, s_true, U0, V0 = workloads.dense_known_spectrum(512, 256, seed=0)
    res = tsvd.blanczos(torch.from_numpy(A).cuda(), 10, 16, 4, seed=0, tol=1e-6, max_restarts=100,
                        restart_keep=32)
    assert res.status == 0 and res.info["converged"] == 1
    s, U, V = _np(res.sigma), _np(res.U), _np(res.V)
    assert np.max(np.abs(s - s_true[:10])) <= 2e-6
    relgap = (s_true[9] - s_true[10]) / s_true[0]
    assert subspace_sin(U, U0[:, :10]) < 10e-6 / relgap and subspace_sin(V, V0[:, :10]) < 10e-6 / relgap
    # mixed form (tensor-core products, FP32 bases with FP64 masters of the kept vectors)
    rm = tsvd.blanczos(torch.from_numpy(A).cuda(), 10, 16, 4, seed=0, tol=1e-6, max_restarts=100,
                       restart_keep=32, precision="mixed")
    assert rm.status == 0 and rm.info["converged"] == 1
    assert np.max(np.abs(_np(rm.sigma) - s_true[:10])) <= 2e-6
    so, _, _, info = oracle.blanczos(A, 10, 16, 4, seed=0, tol=1e-6, max_restarts=100, keep=32)
    np.testing.assert_allclose(_np(res.sigma), so, rtol=2e-6)


def test_thick_restart_rejects_bad_keep(tsvd, torch_cuda):
    A = workloads.csr_uniform(300, 200, 5, seed=1)
    Ad = tsvd.CsrMatrix.from_scipy(A)
    with pytest.raises(tsvd.TsvdError):
        tsvd.blanczos(Ad, 8, 8, 4, restart_keep=4)      # keep < k
    with pytest.raises(tsvd.TsvdError):
        tsvd.blanczos(Ad, 8, 8, 4, restart_keep=28)     # keep + b > r b
    with pytest.raises(tsvd.TsvdError):
        tsvd.blanczos(Ad, 8, 8, 4, restart_keep=-1)


def test_thick_restart_full_size_sparse(tsvd, torch_cuda):
    """100,000 x 100,000 CSR, k = b = 64, r = 9, keep 128 (the benchmark's launch
    configuration), to residual 1e-6: the same singular values as the basic method
    (r = 16) within the residual bound, with fewer products with A."""
    A = workloads.csr_uniform(100_000, 100_000, 10, seed=1)
    Ad = tsvd.CsrMatrix.from_scipy(A)
    rt = tsvd.blanczos(Ad, 64, 64, 9, seed=1, tol=1e-6, restart_keep=128)
    rb_ = tsvd.blanczos(Ad, 64, 64, 16, seed=1, tol=1e-6)
    assert rt.status == 0 and rb_.status == 0
    st, sb = _np(rt.sigma), _np(rb_.sigma)
    assert np.max(np.abs(st - sb)) / sb[0] <= 2e-6
    blocks_thick = 9 + (rt.info["iterations"] - 1) * ((576 - 128) // 64)
    blocks_basic = 16 * rb_.info["iterations"]
    print(f"full size thick restart: {rt.info['ms_total'] / 1e3:.3f} s, {rt.info['iterations']} cycles "
          f"({blocks_thick} blocks), basic {rb_.info['ms_total'] / 1e3:.3f} s, {rb_.info['iterations']} cycles "
          f"({blocks_basic} blocks), resid {rt.info['resid_max']:.2e}")
    assert blocks_thick < blocks_basic


def test_thick_restart_mixed_form_converges_where_fp32_kept_vectors_stall(tsvd, torch_cuda):
    """The mixed form with thick restart keeps FP64 master copies of the kept Ritz
    vectors (their FP32 rounding alone stalls the FP64 residual just above 1e-6 on
    the 100,000^2 matrix): it must reach tol against the FP64 A and agree with the
    FP64 method, at the benchmark's thick-restart configuration."""
    A = workloads.csr_uniform(100_000, 100_000, 10, seed=1)
    Ad = tsvd.CsrMatrix.from_scipy(A)
    rm = tsvd.blanczos(Ad, 64, 64, 9, seed=1, tol=1e-6, restart_keep=128, precision="mixed")
    rd = tsvd.blanczos(Ad, 64, 64, 9, seed=1, tol=1e-6, restart_keep=128)
    assert rm.status == 0 and rm.info["converged"] == 1 and rm.info["resid_max"] <= 1e-6
    s32, s64 = _np(rm.sigma), _np(rd.sigma)
    assert np.max(np.abs(s32 - s64)) / s64[0] <= 2e-6
    U, V = _np(rm.U), _np(rm.V)
    resid = max(np.linalg.norm(A @ V - U * s32, axis=0).max(), np.linalg.norm(A.T @ U - V * s32, axis=0).max())
    assert resid / s32[0] <= 1e-6 * 1.0001
    print(f"mixed thick: {rm.info['ms_total'] / 1e3:.3f} s ({rm.info['iterations']} cycles), "
          f"FP64 thick {rd.info['ms_total'] / 1e3:.3f} s ({rd.info['iterations']} cycles), resid {resid / s32[0]:.2e}")
