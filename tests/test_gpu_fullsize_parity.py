"""Element-wise parity with the FP64 oracle at the full sizes and launch
configurations the benchmark times (Alg. 1 and Alg. 2 from the same Philox start
block):

* the 100,000 x 100,000 CSR matrix (10 nnz per row), LancSVD k = b = 64, r = 9
  with thick restart keeping 128 Ritz pairs: two cycles element-wise (sigma to
  1e-10, subspaces to 1e-8, the Lanczos estimate rho and the explicit residual
  within the residual bound), and the converged solve (tol 1e-6): the same number
  of cycles and the same residual as the oracle's;
* the same matrix, RandSVD k = 64, p = 64, q = 3;
* the dense 20,000 x 20,000 Householder matrix (sigma_i = 1/(1+i)^1.5),
  LancSVD k = 100, b = 128, r = 4, one cycle in FP64.
"""

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


@pytest.fixture(scope="module")
def sparse100k():
    return workloads.csr_uniform(100_000, 100_000, 10, seed=1)


def _np(t):
    return t.detach().cpu().numpy()


def test_thick_restart_two_cycles_full_size_matches_oracle(tsvd, torch_cuda, sparse100k):
    A = sparse100k
    res = tsvd.blanczos(tsvd.CsrMatrix.from_scipy(A), 64, 64, 9, seed=1, tol=0.0, max_restarts=1,
                        restart_keep=128)
    so, Uo, Vo, info = oracle.blanczos(A, 64, 64, 9, seed=1, tol=0.0, max_restarts=1, keep=128)
    assert res.info["iterations"] == 2 == info.iterations
    s, U, V = _np(res.sigma), _np(res.U), _np(res.V)
    np.testing.assert_allclose(s, so, rtol=1e-10)
    su, sv = subspace_sin(U, Uo), subspace_sin(V, Vo)
    print(f"thick, 2 cycles: max rel sigma diff {np.max(np.abs(s - so) / so):.1e}, sin U {su:.1e}, sin V {sv:.1e}, "
          f"rho {res.info['rho_last']:.4e} (oracle {info.rho_hist[-1]:.4e})")
    assert su < 1e-8 and sv < 1e-8, (su, sv)
    bound = residual_gap_bound(su, sv, 1e-10)
    assert abs(res.info["rho_last"] - info.rho_hist[-1]) <= bound
    assert abs(res.info["resid_max"] - info.resid_max) <= bound


def test_thick_restart_converged_full_size_matches_oracle(tsvd, torch_cuda, sparse100k):
    """The benchmark's step: the oracle's converged solve takes the same cycle count
    as the GPU solve and stops at the same residual."""
    A = sparse100k
    res = tsvd.blanczos(tsvd.CsrMatrix.from_scipy(A), 64, 64, 9, seed=1, tol=1e-6, max_restarts=50,
                        restart_keep=128)
    so, Uo, Vo, info = oracle.blanczos(A, 64, 64, 9, seed=1, tol=1e-6, max_restarts=50, keep=128)
    assert res.status == 0 and res.info["converged"] == 1 and info.converged
    s, U, V = _np(res.sigma), _np(res.U), _np(res.V)
    su, sv = subspace_sin(U, Uo), subspace_sin(V, Vo)
    print(f"thick converged: {res.info['iterations']} cycles (oracle {info.iterations}), resid "
          f"{res.info['resid_max']:.4e} (oracle {info.resid_max:.4e}), max rel sigma diff "
          f"{np.max(np.abs(s - so) / so):.1e}, sin U {su:.1e}, sin V {sv:.1e}")
    assert res.info["iterations"] == info.iterations
    assert res.info["resid_max"] <= 1e-6 and info.resid_max <= 1e-6
    np.testing.assert_allclose(s, so, rtol=1e-9)
    assert abs(res.info["resid_max"] - info.resid_max) <= residual_gap_bound(su, sv, 1e-9)


def test_rsvd_full_size_matches_oracle(tsvd, torch_cuda, sparse100k):
    A = sparse100k
    res = tsvd.rsvd(tsvd.CsrMatrix.from_scipy(A), 64, 64, 3, seed=1)
    so, Uo, Vo, info = oracle.rsvd(A, 64, 64, 3, seed=1)
    assert res.info["iterations"] == 4 == info.iterations
    s, U, V = _np(res.sigma), _np(res.U), _np(res.V)
    su, sv = subspace_sin(U, Uo), subspace_sin(V, Vo)
    print(f"rsvd q=3: max rel sigma diff {np.max(np.abs(s - so) / so):.1e}, sin U {su:.1e}, sin V {sv:.1e}")
    np.testing.assert_allclose(s, so, rtol=1e-10)
    assert su < 1e-8 and sv < 1e-8, (su, sv)
    assert abs(res.info["resid_max"] - info.resid_max) <= residual_gap_bound(su, sv, 1e-10)


def test_dense20k_one_cycle_fp64_matches_oracle(tsvd, torch_cuda):
    torch = torch_cuda
    A, sigma = workloads.dense_householder_spectrum_torch(20_000, 20_000, seed=2, L=16, device="cuda")
    res = tsvd.blanczos(A, 100, 128, 4, seed=2, tol=0.0, max_restarts=0)
    An = A.cpu().numpy()
    del A
    torch.cuda.empty_cache()
    so, Uo, Vo, info = oracle.blanczos(An, 100, 128, 4, seed=2, tol=0.0, max_restarts=0)
    assert res.info["iterations"] == 1 == info.iterations
    s, U, V = _np(res.sigma), _np(res.U), _np(res.V)
    su, sv = subspace_sin(U, Uo), subspace_sin(V, Vo)
    print(f"dense 20k, 1 cycle: max rel sigma diff {np.max(np.abs(s - so) / so):.1e}, sin U {su:.1e}, "
          f"sin V {sv:.1e}, resid {res.info['resid_max']:.3e} (oracle {info.resid_max:.3e})")
    np.testing.assert_allclose(s, so, rtol=1e-10)
    assert su < 1e-8 and sv < 1e-8, (su, sv)
    assert abs(res.info["resid_max"] - info.resid_max) <= residual_gap_bound(su, sv, 1e-10)
