"""Truncated SVD on one NVIDIA GB300: RandSVD and block LancSVD (Tomas,
Quintana-Orti, Anzt, "Fast Truncated SVD of Sparse and Dense Matrices on
Graphics Processors") as hand-written sm_103a CUDA behind the C ABI of
``include/tsvd.h``.  This package is a thin ctypes binding: it marshals
arguments, PyTorch supplies device memory and streams, and every step of the
methods runs in ``libtsvd.so``.  Importing the computational entry points
fails loudly when the library has not been built.
"""

from ._capi import TsvdError, LIB_PATH, load  # noqa: F401
from .api import (  # noqa: F401
    CsrMatrix,
    SvdResult,
    blanczos,
    rsvd,
    gaussian_block,
    csr_transpose,
    spmm,
    dense_mm,
    svd_backward,
    truncated_svd,
    Bf16x3,
    bf16x3_split,
    mm_bf16x6,
    cholqr2,
    cgs_cqr2,
    update_gram_f32,
    cgs_qr,
    small_svd,
    handle,
    wait_limit,
    RowPartition,
    torch_allreduce,
    row_block,
)

__all__ = [
    "TsvdError", "CsrMatrix", "SvdResult", "blanczos", "rsvd", "gaussian_block", "csr_transpose", "spmm",
    "dense_mm", "svd_backward", "truncated_svd", "Bf16x3", "bf16x3_split", "mm_bf16x6", "cholqr2", "cgs_cqr2", "update_gram_f32", "cgs_qr", "small_svd", "handle", "wait_limit", "RowPartition", "torch_allreduce",
    "row_block", "load",
    "LIB_PATH",
]
