"""The allocation-free A^T X entry point (tsvd_dense_mm_t_noalloc).

Callers that cannot allocate device memory (their application's memory pool
already holds the whole GPU, or they must never risk the device-wide
synchronisation cudaMalloc/cudaFree can cause) use this variant, whose split-K
scratch is a fixed array inside the library.  It must give the same result as
the workspace-based tsvd_dense_mm(trans=1), call after call.  This file is
collected last so that a failure here comes after every other test ran.
"""

import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _noalloc(tsvd, torch, A, X):
    from paper_2403_06218_gb300 import _capi, api
    lib = tsvd.load()
    m, n = A.shape
    w = X.shape[1]
    Y = torch.full((n, w), float("nan"), dtype=torch.float64, device=A.device)
    rc = lib.tsvd_dense_mm_t_noalloc(api.handle(A.device), m, n, A.data_ptr(), A.stride(0), w, X.data_ptr(),
                                     X.stride(0), Y.data_ptr(), Y.stride(0),
                                     torch.cuda.current_stream(A.device).cuda_stream)
    return rc, Y


@pytest.mark.parametrize("m,n,w", [(100_000, 64, 16), (3000, 300, 64), (512, 256, 20)])
def test_noalloc_matches_workspace_entry_point(tsvd, torch_cuda, m, n, w):
    torch = torch_cuda
    g = torch.Generator(device="cuda").manual_seed(m + n + w)
    A = torch.randn(m, n, dtype=torch.float64, device="cuda", generator=g)
    X = torch.randn(m, w, dtype=torch.float64, device="cuda", generator=g)
    ref = tsvd.dense_mm(A, X, trans=True).cpu().numpy()
    An, Xn = A.cpu().numpy(), X.cpu().numpy()
    bound = 2 * m * np.finfo(np.float64).eps * (np.abs(An.T) @ np.abs(Xn))
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        rc, Y = _noalloc(tsvd, torch, A, X)
        assert rc == 0
        Yn = Y.cpu().numpy()
        # same kernels, same split of the sum, fixed-order reduction: the same bits
        assert np.array_equal(Yn, ref)
        assert np.all(np.abs(Yn - ref) <= bound)
        assert np.all(np.abs(Yn - An.T @ Xn) <= bound)


def test_noalloc_rejects_shapes_beyond_its_scratch(tsvd, torch_cuda):
    torch = torch_cuda
    from paper_2403_06218_gb300 import _capi
    # 96 x 32 outputs split over 354 row slabs need 8.7 MB of partial sums (> 4 MiB)
    A = torch.zeros(200_000, 96, dtype=torch.float64, device="cuda")
    X = torch.zeros(200_000, 32, dtype=torch.float64, device="cuda")
    rc, _ = _noalloc(tsvd, torch, A, X)
    assert rc == _capi.TSVD_ERR_UNSUPPORTED
