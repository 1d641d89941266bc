"""The Python binding's argument checks, on CPU.  The C entry points take plain
pointers and cannot see a tensor's length, so the binding checks every shape a
kernel would index by (CSR array lengths, the rows of X and P, the start block)
before any launch; these tests run those checks without a GPU."""

import numpy as np
import pytest
import torch


def _csr(tsvd, m=6, n=5, nnz=9, idx=torch.int32, val=torch.float64):
    rng = np.random.default_rng(0)
    rp = torch.tensor(np.linspace(0, nnz, m + 1).astype(np.int64), dtype=idx)
    ci = torch.tensor(rng.integers(0, n, nnz), dtype=idx)
    return tsvd.CsrMatrix(rp, ci, torch.ones(nnz, dtype=val), (m, n))


def test_csr_structure_is_checked_before_any_launch(tsvd):
    X = torch.zeros((5, 3), dtype=torch.float64)
    A = _csr(tsvd)
    bad_rp = tsvd.CsrMatrix(A.row_ptr[:-1], A.col_idx, A.val, A.shape)
    with pytest.raises(ValueError, match="row_ptr"):
        tsvd.spmm(bad_rp, X)
    bad_val = tsvd.CsrMatrix(A.row_ptr, A.col_idx, A.val[:-1], A.shape)
    with pytest.raises(ValueError, match="nnz"):
        tsvd.spmm(bad_val, X)
    with pytest.raises(TypeError, match="int32"):
        tsvd.spmm(_csr(tsvd, idx=torch.int64), X)
    with pytest.raises(TypeError, match="values"):
        tsvd.spmm(_csr(tsvd, val=torch.float16), X)
    with pytest.raises(TypeError, match="CsrMatrix"):
        tsvd.spmm(torch.zeros((6, 5), dtype=torch.float64), X)
    # the gradient and the drivers build their descriptors through the same check
    with pytest.raises(ValueError, match="row_ptr"):
        tsvd.svd_backward(bad_rp, torch.ones(1), torch.zeros(6, 1), torch.zeros(5, 1))


def test_spmm_checks_the_rows_of_x(tsvd):
    A = _csr(tsvd)
    with pytest.raises(ValueError, match="5 rows"):
        tsvd.spmm(A, torch.zeros((6, 3), dtype=torch.float64))
    with pytest.raises(ValueError, match="5 rows"):
        tsvd.spmm(A, torch.zeros(5, dtype=torch.float64))
    # right shape, but host memory: rejected before the library is called
    with pytest.raises(TypeError, match="CUDA"):
        tsvd.spmm(A, torch.zeros((5, 3), dtype=torch.float64))


def test_csr_transpose_takes_fp64_values_on_the_gpu(tsvd):
    with pytest.raises(TypeError, match="float64 values on the GPU"):
        tsvd.csr_transpose(_csr(tsvd, val=torch.float32))
    with pytest.raises(TypeError, match="float64 values on the GPU"):
        tsvd.csr_transpose(_csr(tsvd))


@pytest.mark.parametrize("trans,rows", [(False, 4), (True, 7)])
def test_dense_mm_checks_the_rows_of_x(tsvd, trans, rows):
    A = torch.zeros((7, 4), dtype=torch.float64)
    with pytest.raises(ValueError, match=f"{rows} rows"):
        tsvd.dense_mm(A, torch.zeros((rows + 1, 2), dtype=torch.float64), trans=trans)
    with pytest.raises(TypeError, match="CUDA"):
        tsvd.dense_mm(A, torch.zeros((rows, 2), dtype=torch.float64), trans=trans)
    with pytest.raises(TypeError, match="2-D"):
        tsvd.dense_mm(torch.zeros(7, dtype=torch.float64), torch.zeros((rows, 2)), trans=trans)


def test_cgs_cqr2_checks_the_rows_of_p(tsvd):
    Y = torch.zeros((10, 2), dtype=torch.float64)
    with pytest.raises(ValueError, match="10 rows"):
        tsvd.cgs_cqr2(Y, torch.zeros((9, 3), dtype=torch.float64))
    with pytest.raises(TypeError, match="CUDA"):
        tsvd.cgs_cqr2(Y, torch.zeros((10, 3), dtype=torch.float64))


@pytest.mark.parametrize("m,n", [(40, 30), (30, 40)])
def test_start_block_shape_follows_the_method(tsvd, monkeypatch, m, n):
    """LancSVD takes a max(m, n) x b block, RandSVD a min(m, n) x (k + p) block."""
    from paper_2403_06218_gb300 import api
    monkeypatch.setattr(api, "_dev_index", lambda device=None: 0)   # no CUDA call on this host
    A = np.zeros((m, n))
    big, small = max(m, n), min(m, n)
    with pytest.raises(ValueError, match=rf"\({big}, 4\)"):
        tsvd.blanczos(A, 3, 4, 2, start_block=torch.zeros((small, 4), dtype=torch.float64))
    with pytest.raises(ValueError, match=rf"\({big}, 4\)"):
        tsvd.blanczos(A, 3, 4, 2, start_block=torch.zeros((big, 5), dtype=torch.float64))
    with pytest.raises(TypeError, match="CUDA"):
        tsvd.blanczos(A, 3, 4, 2, start_block=torch.zeros((big, 4), dtype=torch.float64))
    with pytest.raises(ValueError, match=rf"\({small}, 7\)"):
        tsvd.rsvd(A, 3, 4, 1, start_block=torch.zeros((big, 7), dtype=torch.float64))
    with pytest.raises(TypeError, match="CUDA"):
        tsvd.rsvd(A, 3, 4, 1, start_block=torch.zeros((small, 7), dtype=torch.float64))
