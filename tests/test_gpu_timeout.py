"""Bounded device waits driven to their limit (no fault, no hang): with a wait
limit of a few SM clock cycles set on the handle, the pipelined split-BF16
product, the FP64-accurate sliced product and the block Jacobi SVD give up their
first wait, stop their pipelines and return TSVD_ERR_TIMEOUT; with the default
limit restored the same calls on the same handle succeed and give the right
result (the context stays usable)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _timeout(tsvd):
    from paper_2403_06218_gb300 import _capi
    return _capi.TSVD_ERR_TIMEOUT


def test_split_bf16_product_times_out_then_recovers(tsvd, torch_cuda):
    torch = torch_cuda
    g = torch.Generator(device="cuda").manual_seed(11)
    A = torch.randn(20_000, 512, dtype=torch.float64, device="cuda", generator=g)
    X = torch.randn(512, 64, dtype=torch.float32, device="cuda", generator=g)
    P = tsvd.bf16x3_split(A)
    with tsvd.wait_limit(2):
        with pytest.raises(tsvd.TsvdError) as e:
            tsvd.mm_bf16x6(P, X)
    assert e.value.code == _timeout(tsvd)
    Y = tsvd.mm_bf16x6(P, X)
    ref = A @ X.double()
    err = float(((Y.double() - ref).abs() / (A.abs() @ X.double().abs())).max())
    assert err < 1e-5, err


def test_sliced_fp64_product_times_out_then_recovers(tsvd, torch_cuda):
    torch = torch_cuda
    g = torch.Generator(device="cuda").manual_seed(12)
    A = torch.randn(20_000, 600, dtype=torch.float64, device="cuda", generator=g)
    X = torch.randn(600, 64, dtype=torch.float64, device="cuda", generator=g)
    with tsvd.wait_limit(2):
        with pytest.raises(tsvd.TsvdError) as e:
            tsvd.dense_mm(A, X, tensor_cores=True)
    assert e.value.code == _timeout(tsvd)
    Y = tsvd.dense_mm(A, X, tensor_cores=True)
    bound = 2 * 600 * np.finfo(np.float64).eps * (A.abs() @ X.abs())
    assert bool(((Y - A @ X).abs() <= bound).all())


def test_block_jacobi_grid_barrier_times_out_then_recovers(tsvd, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(13)
    n = 300  # above the one-CTA sweep size: the cooperative block Jacobi with its grid barrier
    B = torch.from_numpy(rng.standard_normal((n, n))).cuda()
    with tsvd.wait_limit(2):
        with pytest.raises(tsvd.TsvdError) as e:
            tsvd.small_svd(B)
    assert e.value.code == _timeout(tsvd)
    U, s, V, _ = tsvd.small_svd(B)
    ref = np.linalg.svd(B.cpu().numpy(), compute_uv=False)
    assert np.max(np.abs(s.cpu().numpy() - ref)) < 1e-12 * ref[0] * n
