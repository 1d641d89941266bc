"""ctypes declarations of the C ABI in ``include/tsvd.h`` (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "libtsvd.so"

TSVD_OK = 0
TSVD_NOT_CONVERGED = 1
TSVD_ERR_INVALID_ARG = -1
TSVD_ERR_NONFINITE = -2
TSVD_ERR_CUDA = -3
TSVD_ERR_WORKSPACE = -4
TSVD_ERR_TIMEOUT = -5
TSVD_ERR_UNSUPPORTED = -6
TSVD_ERR_COMM = -7

TSVD_DENSE = 0
TSVD_CSR = 1
TSVD_F64 = 0
TSVD_F32 = 1
TSVD_PREC_FP64 = 0
TSVD_PREC_MIXED = 1
TSVD_DEVICE = 0
TSVD_HOST = 1
TSVD_METHOD_RSVD = 0
TSVD_METHOD_BLANCZOS = 1
TSVD_MAX_BLOCK = 128
TSVD_MAX_SMALL_SVD = 2048
TSVD_FLAG_PROFILE = 1
TSVD_FLAG_ROW_PARTITION = 2
TSVD_NOALLOC_SCRATCH_BYTES = 4 * 1024 * 1024
KERNEL_CLASSES = ("a_products", "gemm_tn", "gemm_nn", "chol", "svd", "other", "upd_gram")


class TsvdMatrix(C.Structure):
    _fields_ = [
        ("m", C.c_int64), ("n", C.c_int64),
        ("format", C.c_int32), ("dtype", C.c_int32), ("location", C.c_int32), ("reserved", C.c_int32),
        ("val", C.c_void_p), ("ld", C.c_int64),
        ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("nnz", C.c_int64),
    ]


class TsvdOpts(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("max_restarts", C.c_int32), ("qr_block", C.c_int32),
        ("output_location", C.c_int32), ("flags", C.c_int32),
        ("start_block", C.c_void_p), ("stream", C.c_void_p),
        ("precision", C.c_int32), ("restart_keep", C.c_int32),
    ]


class TsvdInfo(C.Structure):
    _fields_ = [
        ("iterations", C.c_int32), ("restarts", C.c_int32), ("breakdowns", C.c_int32),
        ("converged", C.c_int32), ("transposed", C.c_int32), ("svd_sweeps", C.c_int32),
        ("resid_max", C.c_double), ("rho_last", C.c_double),
        ("ms_total", C.c_double), ("ms_transpose", C.c_double), ("kernel_launches", C.c_int64),
        ("prof_launches", C.c_int64 * 7), ("prof_ms", C.c_double * 7),
        ("prof_flops", C.c_double * 7), ("prof_bytes", C.c_double * 7),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name.startswith("prof_") else v
        return out


class TsvdBackwardOpts(C.Structure):
    _fields_ = [("cg_tol", C.c_double), ("cg_max_iter", C.c_int32), ("check_every", C.c_int32),
                ("stream", C.c_void_p)]


class TsvdBackwardInfo(C.Structure):
    _fields_ = [("cg_iters_u", C.c_int32), ("cg_iters_v", C.c_int32), ("cg_resid_u", C.c_double),
                ("cg_resid_v", C.c_double), ("ms_total", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


# int (*tsvd_allreduce_fn)(void* ctx, double* buf, int64_t count)
ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_int64)

# (name, restype, argtypes); every symbol listed here is declared in include/tsvd.h.
_P = C.c_void_p
_I = C.c_int
_I64 = C.c_int64
_SZ = C.c_size_t
_PSZ = C.POINTER(C.c_size_t)
_PI = C.POINTER(C.c_int)
SIGNATURES = [
    ("tsvd_default_opts", None, [C.POINTER(TsvdOpts)]),
    ("tsvd_create", _I, [C.POINTER(_P), _I]),
    ("tsvd_destroy", _I, [_P]),
    ("tsvd_set_wait_limit", _I, [_P, C.c_longlong]),
    ("tsvd_set_row_partition", _I, [_P, _I64, _I64, ALLREDUCE_FN, _P]),
    ("tsvd_status_string", C.c_char_p, [_I]),
    ("tsvd_workspace_size", _I, [C.POINTER(TsvdMatrix), _I, _I, _I, _I, C.POINTER(TsvdOpts), _PSZ]),
    ("tsvd_rsvd", _I, [_P, C.POINTER(TsvdMatrix), _I, _I, _I, C.c_uint64, C.POINTER(TsvdOpts), _P, _SZ,
                       _P, _P, _P, C.POINTER(TsvdInfo)]),
    ("tsvd_blanczos", _I, [_P, C.POINTER(TsvdMatrix), _I, _I, _I, C.c_uint64, C.POINTER(TsvdOpts), _P, _SZ,
                           _P, _P, _P, C.POINTER(TsvdInfo)]),
    ("tsvd_gaussian_block", _I, [_I64, _I64, C.c_uint64, C.c_uint32, _P, _I64, _P]),
    ("tsvd_csr_transpose_workspace", _I, [_I64, _I64, _I64, _PSZ]),
    ("tsvd_csr_transpose", _I, [_P, _I64, _I64, _I64, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    ("tsvd_spmm_workspace", _I, [_I64, _I64, _I, _PSZ]),
    ("tsvd_spmm_f32", _I, [_P, _I64, _I64, _I64, _P, _P, _P, _I, _P, _I64, _P, _I64, _P, _SZ, _P]),
    ("tsvd_spmm", _I, [_P, _I64, _I64, _I64, _P, _P, _P, _I, _P, _I64, _P, _I64, _P, _SZ, _P]),
    ("tsvd_dense_mm_workspace", _I, [_I, _I64, _I64, _I, _PSZ]),
    ("tsvd_dense_mm", _I, [_P, _I, _I64, _I64, _P, _I64, _I, _P, _I64, _P, _I64, _P, _SZ, _P]),
    ("tsvd_dense_mm_f32", _I, [_P, _I, _I64, _I64, _P, _I64, _I, _P, _I64, _P, _I64, _P, _SZ, _P]),
    ("tsvd_dense_mm_f64tc_workspace", _I, [_I, _I64, _I64, _I, _PSZ]),
    ("tsvd_dense_mm_f64tc", _I, [_P, _I, _I64, _I64, _P, _I64, _I, _P, _I64, _P, _I64, _P, _SZ, _P]),
    ("tsvd_default_backward_opts", None, [_P]),
    ("tsvd_svd_backward_workspace", _I, [_P, _I, _P, _PSZ]),
    ("tsvd_svd_backward", _I, [_P, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    ("tsvd_bf16x3_bytes", _I, [_I64, _I64, _PSZ]),
    ("tsvd_bf16x3_split", _I, [_P, _I, _I64, _I64, _P, _I64, _P, _P]),
    ("tsvd_mm_bf16x6_workspace", _I, [_I64, _I64, _I, _PSZ]),
    ("tsvd_mm_bf16x6", _I, [_P, _I64, _I64, _P, _I, _P, _I64, _P, _I64, _P, _SZ, _P]),
    ("tsvd_orth_workspace", _I, [_I64, _I64, _I, _PSZ]),
    ("tsvd_cholqr2", _I, [_P, _I64, _I, _P, _I64, _P, C.c_uint64, _PI, _PI, _P, _SZ, _P]),
    ("tsvd_cgs_cqr2", _I, [_P, _I64, _I64, _I, _P, _I64, _P, _I64, _P, _P, C.c_uint64, _PI, _PI, _P, _SZ, _P]),
    ("tsvd_cgs_cqr2_f32", _I, [_P, _I64, _I64, _I, _P, _I64, _P, _I64, _P, _P, C.c_uint64, _PI, _PI, _P, _SZ,
                               _P]),
    ("tsvd_update_gram_f32_workspace", _I, [_I64, _I, _PSZ]),
    ("tsvd_update_gram_f32", _I, [_P, _I64, _I64, _I, C.c_double, _P, _I64, _P, _I64, C.c_double, _P, _I64, _I,
                                  _P, _P, _SZ, _P]),
    ("tsvd_cgs_qr", _I, [_P, _I64, _I, _I, _P, _I64, _P, C.c_uint64, _PI, _PI, _P, _SZ, _P]),
    ("tsvd_small_svd_workspace", _I, [_I, _PSZ]),
    ("tsvd_small_svd", _I, [_P, _I, _P, _I64, _I, _P, _P, _P, _PI, _P, _SZ, _P]),
    ("tsvd_dense_mm_t_noalloc", _I, [_P, _I64, _I64, _P, _I64, _I, _P, _I64, _P, _I64, _P]),
]


class TsvdError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


_lib = None


def load():
    """Loads libtsvd.so; raises ImportError (never falls back) when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -m paper_2403_06218_gb300.build, or __graft_entry__.build())")
    import torch  # noqa: F401  (loads the CUDA runtime torch links against first)
    lib = C.CDLL(str(LIB_PATH), mode=os.RTLD_LOCAL if hasattr(os, "RTLD_LOCAL") else 0)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().tsvd_status_string(code).decode()
    except ImportError:
        return "status"


def check(code: int, where: str, allow_not_converged: bool = False) -> int:
    if code == TSVD_OK or (allow_not_converged and code == TSVD_NOT_CONVERGED):
        return code
    raise TsvdError(code, where)
