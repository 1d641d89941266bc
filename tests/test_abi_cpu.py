"""The C-ABI library builds, loads and exports every entry point include/tsvd.h
declares; host-side argument validation works without a GPU.  No compute calls."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tsvd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s+(tsvd_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("tsvd_rsvd", "tsvd_blanczos", "tsvd_create", "tsvd_destroy", "tsvd_workspace_size",
                 "tsvd_spmm", "tsvd_csr_transpose", "tsvd_cholqr2", "tsvd_cgs_cqr2", "tsvd_cgs_qr",
                 "tsvd_small_svd", "tsvd_gaussian_block", "tsvd_dense_mm", "tsvd_dense_mm_f32",
                 "tsvd_dense_mm_f64tc", "tsvd_dense_mm_f64tc_workspace",
                 "tsvd_spmm_workspace", "tsvd_bf16x3_split", "tsvd_mm_bf16x6", "tsvd_svd_backward",
                 "tsvd_svd_backward_workspace"):
        assert must in names


def test_library_exports_every_declared_symbol(tsvd):
    lib = tsvd.load()
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_2403_06218_gb300 import _capi
    bound = {n for n, _, _ in _capi.SIGNATURES}
    assert bound == set(_declared())


def test_host_side_validation_without_gpu(tsvd):
    from paper_2403_06218_gb300 import _capi
    lib = tsvd.load()
    opts = _capi.TsvdOpts()
    lib.tsvd_default_opts(C.byref(opts))
    assert opts.tol == 1e-6 and opts.max_restarts == 50 and opts.qr_block == 0
    assert lib.tsvd_status_string(_capi.TSVD_ERR_WORKSPACE).decode().startswith("workspace")
    d = _capi.TsvdMatrix()
    d.m, d.n, d.format, d.location, d.ld = 100, 50, _capi.TSVD_DENSE, _capi.TSVD_DEVICE, 50
    d.val = 1  # never dereferenced by the sizing call
    nb = C.c_size_t()
    # k > min(m, n), l > n, b > TSVD_MAX_BLOCK, r*b > n are rejected before any device work
    assert lib.tsvd_workspace_size(C.byref(d), 0, 60, 0, 1, None, C.byref(nb)) == _capi.TSVD_ERR_INVALID_ARG
    assert lib.tsvd_workspace_size(C.byref(d), 0, 10, 41, 1, None, C.byref(nb)) == _capi.TSVD_ERR_INVALID_ARG
    assert lib.tsvd_workspace_size(C.byref(d), 1, 10, 129, 1, None, C.byref(nb)) == _capi.TSVD_ERR_UNSUPPORTED
    assert lib.tsvd_workspace_size(C.byref(d), 1, 10, 16, 4, None, C.byref(nb)) == _capi.TSVD_ERR_INVALID_ARG
    assert lib.tsvd_workspace_size(C.byref(d), 1, 10, 8, 4, None, C.byref(nb)) == _capi.TSVD_OK
    small = nb.value
    d.m, d.n, d.ld = 1000, 500, 500
    assert lib.tsvd_workspace_size(C.byref(d), 1, 10, 8, 4, None, C.byref(nb)) == _capi.TSVD_OK
    assert nb.value > small
    # bad dtype / format
    d.dtype = 7
    assert lib.tsvd_workspace_size(C.byref(d), 1, 10, 8, 4, None, C.byref(nb)) == _capi.TSVD_ERR_UNSUPPORTED
    d.dtype, d.format = 0, 9
    assert lib.tsvd_workspace_size(C.byref(d), 1, 10, 8, 4, None, C.byref(nb)) == _capi.TSVD_ERR_INVALID_ARG
    # a call without a handle is rejected
    assert lib.tsvd_blanczos(None, C.byref(d), 1, 1, 1, 0, None, None, 0, None, None, None, None) == \
        _capi.TSVD_ERR_INVALID_ARG
    assert lib.tsvd_small_svd_workspace(0, C.byref(nb)) == _capi.TSVD_ERR_INVALID_ARG
    assert lib.tsvd_small_svd_workspace(4096, C.byref(nb)) == _capi.TSVD_ERR_UNSUPPORTED


def test_validation_of_the_newer_entry_points_without_gpu(tsvd):
    """Thick restart, the gradient, the tensor-core product and the SpMM plan reject
    bad arguments (or size their workspace) before any device work."""
    from paper_2403_06218_gb300 import _capi
    lib = tsvd.load()
    d = _capi.TsvdMatrix()
    d.m, d.n, d.format, d.location, d.ld = 1000, 500, _capi.TSVD_DENSE, _capi.TSVD_DEVICE, 500
    d.val = 1
    nb = C.c_size_t()
    opts = _capi.TsvdOpts()
    lib.tsvd_default_opts(C.byref(opts))
    assert opts.restart_keep == 0
    for keep, code in ((4, _capi.TSVD_ERR_INVALID_ARG),    # keep < k
                       (28, _capi.TSVD_ERR_INVALID_ARG),   # keep + b > r b
                       (-1, _capi.TSVD_ERR_INVALID_ARG),
                       (16, _capi.TSVD_OK)):
        opts.restart_keep = keep
        assert lib.tsvd_workspace_size(C.byref(d), 1, 8, 8, 4, C.byref(opts), C.byref(nb)) == code, keep
    base = nb.value
    opts.restart_keep = 0
    assert lib.tsvd_workspace_size(C.byref(d), 1, 8, 8, 4, C.byref(opts), C.byref(nb)) == _capi.TSVD_OK
    assert base > nb.value  # the kept Ritz vectors need room
    opts.restart_keep, opts.precision = 16, _capi.TSVD_PREC_MIXED
    assert lib.tsvd_workspace_size(C.byref(d), 1, 8, 8, 4, C.byref(opts), C.byref(nb)) == _capi.TSVD_OK
    # gradient: k in [1, min(m, n)], k <= TSVD_MAX_BLOCK, positive tolerance
    bo = _capi.TsvdBackwardOpts()
    lib.tsvd_default_backward_opts(C.byref(bo))
    assert bo.cg_tol == 1e-12 and bo.cg_max_iter > 0
    assert lib.tsvd_svd_backward_workspace(C.byref(d), 0, C.byref(bo), C.byref(nb)) == _capi.TSVD_ERR_INVALID_ARG
    assert lib.tsvd_svd_backward_workspace(C.byref(d), 129, C.byref(bo), C.byref(nb)) == \
        _capi.TSVD_ERR_UNSUPPORTED
    assert lib.tsvd_svd_backward_workspace(C.byref(d), 8, C.byref(bo), C.byref(nb)) == _capi.TSVD_OK and nb.value > 0
    bo.cg_tol = 0.0
    assert lib.tsvd_svd_backward_workspace(C.byref(d), 8, C.byref(bo), C.byref(nb)) == _capi.TSVD_ERR_INVALID_ARG
    # split-BF16 product and SpMM workspaces
    assert lib.tsvd_mm_bf16x6_workspace(-1, 10, 4, C.byref(nb)) == _capi.TSVD_ERR_INVALID_ARG
    assert lib.tsvd_mm_bf16x6_workspace(1000, 500, 64, C.byref(nb)) == _capi.TSVD_OK and nb.value > 0
    assert lib.tsvd_bf16x3_bytes(1000, 501, C.byref(nb)) == _capi.TSVD_OK
    assert nb.value >= 3 * 1000 * 504 * 2 and nb.value % 256 == 0  # rows padded to a multiple of 8
    small = C.c_size_t()
    assert lib.tsvd_spmm_workspace(100, 1000, 64, C.byref(small)) == _capi.TSVD_OK
    assert lib.tsvd_spmm_workspace(100, 10 ** 7, 64, C.byref(nb)) == _capi.TSVD_OK and nb.value > small.value


def test_fused_update_gram_and_fp32_orthogonalisation_entry_points_without_gpu(tsvd):
    """The fused update + Gram pass and the FP32-block CGS-CQR2 reject bad arguments
    before any device work; the fused pass's workspace holds one b x b FP64 partial
    Gram matrix per row slab (at most one wave of slabs, so it stops growing with q),
    and the orthogonalisation workspace covers it."""
    from paper_2403_06218_gb300 import _capi
    lib = tsvd.load()
    nb = C.c_size_t()
    assert lib.tsvd_update_gram_f32_workspace(-1, 64, C.byref(nb)) == _capi.TSVD_ERR_INVALID_ARG
    assert lib.tsvd_update_gram_f32_workspace(1000, 0, C.byref(nb)) == _capi.TSVD_ERR_INVALID_ARG
    assert lib.tsvd_update_gram_f32_workspace(1000, 129, C.byref(nb)) == _capi.TSVD_ERR_UNSUPPORTED
    sizes = {}
    for q, b in ((64, 64), (10 ** 5, 64), (10 ** 6, 64), (10 ** 7, 64), (10 ** 7, 128)):
        assert lib.tsvd_update_gram_f32_workspace(q, b, C.byref(nb)) == _capi.TSVD_OK
        sizes[q, b] = nb.value
        assert nb.value % 256 == 0 and nb.value >= 8 * b * b
    assert sizes[64, 64] < sizes[10 ** 5, 64] <= sizes[10 ** 6, 64]
    # at most one wave of slabs: 4 CTAs an SM for b <= 64, 2 for b = 128 (152 SMs)
    for (q, b), v in sizes.items():
        assert v <= 8 * b * b * 152 * (4 if b <= 64 else 2) + 256, (q, b, v)
    assert sizes[10 ** 7, 64] > 0.95 * 8 * 64 * 64 * 152 * 4
    orth = C.c_size_t()
    for q, s_, b in ((10 ** 5, 576, 64), (2 * 10 ** 6, 1024, 128)):
        assert lib.tsvd_orth_workspace(q, s_, b, C.byref(orth)) == _capi.TSVD_OK
        assert lib.tsvd_update_gram_f32_workspace(q, b, C.byref(nb)) == _capi.TSVD_OK
        assert orth.value > nb.value
    # no handle
    assert lib.tsvd_update_gram_f32(None, 100, 10, 8, 1.0, 1, 10, 1, 8, 0.0, 1, 8, 0, 1, None, 0, None) == \
        _capi.TSVD_ERR_INVALID_ARG
    assert lib.tsvd_cgs_cqr2_f32(None, 100, 10, 8, 1, 10, 1, 8, None, 1, 0, None, None, None, 0, None) == \
        _capi.TSVD_ERR_INVALID_ARG


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2403_06218_gb300 import _capi
    monkeypatch.setattr(_capi, "LIB_PATH", tmp_path / "libtsvd.so")
    monkeypatch.setattr(_capi, "_lib", None)
    with pytest.raises(ImportError):
        _capi.load()
