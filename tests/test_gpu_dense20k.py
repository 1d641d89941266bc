"""The large dense workload at full size: A = H_U diag(sigma) H_V^T, 20,000 x
20,000 FP64, sigma_i = 1/(1+i)^1.5, k = 100, LancSVD b = 128, r = 4, to residual
1e-6, in the FP64 method and in the mixed form (split-BF16 tensor-core products).

No oracle run at this size: the singular values are known in closed form, so
each run must (i) meet the residual bound on both sides against the FP64 A,
(ii) return the k largest singular values to within 2 tol sigma_1 (a triplet
with residual eps lies within eps of a singular value), (iii) return
orthonormal U and V.  The mixed form's errors against the exact values and
against the FP64 run are printed for the record.
"""

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

M = N = 20_000
K, B, R, TOL = 100, 128, 4, 1e-6


@pytest.fixture(scope="module")
def dense20k():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A, sigma = workloads.dense_householder_spectrum_torch(M, N, seed=2, L=16, device="cuda")
    yield torch, A, sigma
    del A
    torch.cuda.empty_cache()


def _check(torch, A, res, sigma, label):
    s = res.sigma.double()
    U, V = res.U, res.V
    R1 = torch.linalg.vector_norm(A @ V - U * s, dim=0).max()
    R2 = torch.linalg.vector_norm(A.T @ U - V * s, dim=0).max()
    resid = float(max(R1, R2) / s[0])
    assert resid <= TOL * 1.0001, resid
    err = float(np.max(np.abs(s.cpu().numpy() - sigma[:K])) / sigma[0])
    assert err <= 2 * TOL, err
    I = torch.eye(K, dtype=torch.float64, device=A.device)
    assert float((U.T @ U - I).abs().max()) < 1e-12 and float((V.T @ V - I).abs().max()) < 1e-12
    print(f"{label}: {res.info['ms_total'] / 1e3:.3f} s, {res.info['iterations']} cycles, resid {resid:.2e}, "
          f"max |sigma - exact| / sigma_1 = {err:.2e}")
    return s.cpu().numpy()


def test_dense20k_lanczos_fp64_and_mixed(tsvd, dense20k):
    torch, A, sigma = dense20k
    r64 = tsvd.blanczos(A, K, B, R, seed=2, tol=TOL, max_restarts=300)
    assert r64.status == 0 and r64.info["converged"] == 1
    s64 = _check(torch, A, r64, sigma, "fp64")
    r32 = tsvd.blanczos(A, K, B, R, seed=2, tol=TOL, max_restarts=300, precision="mixed")
    assert r32.status == 0 and r32.info["converged"] == 1
    s32 = _check(torch, A, r32, sigma, "mixed")
    print(f"mixed vs fp64: max |sigma diff| / sigma_1 = {np.max(np.abs(s32 - s64)) / s64[0]:.2e}")
    assert r32.info["ms_total"] < r64.info["ms_total"]


def test_dense20k_rsvd_mixed_matches_fp64_method(tsvd, dense20k):
    """RandSVD, l = 128 (p = 28), q = 2: the same method in both precisions, so the
    Ritz values agree far below the method's own error."""
    torch, A, sigma = dense20k
    r64 = tsvd.rsvd(A, K, 28, 2, seed=2)
    r32 = tsvd.rsvd(A, K, 28, 2, seed=2, precision="mixed")
    s64, s32 = r64.sigma.double().cpu().numpy(), r32.sigma.double().cpu().numpy()
    d = np.max(np.abs(s32 - s64)) / s64[0]
    print(f"rsvd q=2: fp64 {r64.info['ms_total']:.1f} ms, mixed {r32.info['ms_total']:.1f} ms, sigma diff {d:.2e}, "
          f"sigma_1 error {abs(s64[0] - sigma[0]):.2e}")
    assert d < 1e-6
