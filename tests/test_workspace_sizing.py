"""Workspace sizing on CPU (host-only calls): the sizes cover the Lanczos bases
and the digit planes of the FP64 tensor-core products,
grow linearly with the tall dimension, and stay in 64-bit arithmetic at sizes
beyond 2^31 rows and 2^31 - 1 stored entries."""

import ctypes as C

import pytest

from paper_2403_06218_gb300 import _capi


def _ws(lib, m, n, fmt, nnz, method, k, a, c, keep=0, prec=_capi.TSVD_PREC_FP64):
    d = _capi.TsvdMatrix()
    d.m, d.n, d.format, d.dtype, d.location = m, n, fmt, _capi.TSVD_F64, _capi.TSVD_DEVICE
    d.val, d.ld, d.row_ptr, d.col_idx, d.nnz = 1, n, 1, 1, nnz   # sizing never dereferences them
    o = _capi.TsvdOpts()
    lib.tsvd_default_opts(C.byref(o))
    o.restart_keep, o.precision = keep, prec
    nb = C.c_size_t()
    rc = lib.tsvd_workspace_size(C.byref(d), method, k, a, c, C.byref(o), C.byref(nb))
    assert rc == _capi.TSVD_OK
    return nb.value


@pytest.mark.parametrize("keep", [0, 128])
def test_lanczos_workspace_holds_both_bases(tsvd, keep):
    lib = tsvd.load()
    m = n = 100_000
    r = 9 if keep else 16
    ws = _ws(lib, m, n, _capi.TSVD_CSR, 1_000_000, _capi.TSVD_METHOD_BLANCZOS, 64, 64, r, keep=keep)
    bases = 8 * (m + n) * r * 64                       # P (n x rb) and Pbar (m x rb), FP64
    # BF16 digit planes (7 x 2 bytes an entry) of the tensor-core products: scratch for
    # the largest operands (a q x rb basis prefix and a q x max(b, k, keep) block) and
    # the kept planes of both bases in both layouts
    planes = 14 * max(m, n) * (r * 64 + max(64, keep)) + 2 * 14 * (m + n) * r * 64
    assert bases + planes < ws < 1.25 * (bases + planes)


@pytest.mark.parametrize("method,a,c", [(_capi.TSVD_METHOD_BLANCZOS, 64, 4), (_capi.TSVD_METHOD_RSVD, 64, 2)])
def test_sizes_grow_linearly_and_stay_64_bit(tsvd, method, a, c):
    lib = tsvd.load()
    n = 1000
    small = _ws(lib, 3_000_000, n, _capi.TSVD_DENSE, 0, method, 64, a, c)
    huge = _ws(lib, 3_000_000_000, n, _capi.TSVD_DENSE, 0, method, 64, a, c)
    assert 0.99e3 * small < huge < 1.01e3 * small       # linear in m: no 32-bit wrap-around
    width = a * c if method == _capi.TSVD_METHOD_BLANCZOS else 64 + a
    assert huge > 8 * 3_000_000_000 * width             # at least the m-side basis / block


def test_csr_sizing_at_the_int32_index_limit(tsvd):
    lib = tsvd.load()
    nnz = 2 ** 31 - 1
    ws = _ws(lib, 1_500_000_000, 1_000_000_000, _capi.TSVD_CSR, nnz, _capi.TSVD_METHOD_BLANCZOS, 64, 64, 4)
    # CSR(A^T): n + 1 row pointers, nnz column indices and values, plus the m-side basis
    assert ws > 4 * (10 ** 9 + 1) + 12 * nnz + 8 * 1_500_000_000 * 256
