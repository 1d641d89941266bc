"""Python entry points over the C ABI: argument marshalling only.

Every computation runs in ``libtsvd.so``; this module only builds descriptors,
allocates outputs and workspace with PyTorch (device memory) or numpy (host
memory), passes the current CUDA stream, and raises ``TsvdError`` on failure.
Matrices:

* ``CsrMatrix`` (int32 ``row_ptr``/``col_idx`` and float64 ``val`` tensors, on the
  GPU or in host memory), a ``torch.sparse_csr`` tensor, or a ``scipy.sparse``
  matrix (host);
* a dense float64 ``torch.Tensor`` (GPU or host) or ``numpy.ndarray`` (host),
  row-major.

Host inputs are staged onto the GPU by the library inside the call; ``output="host"``
returns numpy arrays copied back inside the call.
"""

from __future__ import annotations

import contextlib
import ctypes as C
import dataclasses
from typing import Optional

import numpy as np
import torch

from . import _capi as capi

_handles: dict = {}


def _dev_index(device=None) -> int:
    if device is None:
        return torch.cuda.current_device()
    d = torch.device(device)
    return d.index if d.index is not None else torch.cuda.current_device()


def handle(device=None):
    """Library handle of a CUDA device (created once per device)."""
    lib = capi.load()
    idx = _dev_index(device)
    h = _handles.get(idx)
    if h is None:
        hp = C.c_void_p()
        capi.check(lib.tsvd_create(C.byref(hp), idx), "tsvd_create")
        h = hp
        _handles[idx] = h
    return h


@contextlib.contextmanager
def wait_limit(cycles: int, device=None):
    """Within the block, every bounded device-side wait of the kernels launched through
    this device's handle gives up after ``cycles`` SM clock cycles (a test hook: the
    calls then return TSVD_ERR_TIMEOUT).  The default limit is restored on exit."""
    lib = capi.load()
    h = handle(device)
    capi.check(lib.tsvd_set_wait_limit(h, int(cycles)), "tsvd_set_wait_limit")
    try:
        yield
    finally:
        capi.check(lib.tsvd_set_wait_limit(h, 0), "tsvd_set_wait_limit")


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


@dataclasses.dataclass
class CsrMatrix:
    """CSR matrix with int32 indices and float64 values (GPU or host tensors)."""
    row_ptr: torch.Tensor
    col_idx: torch.Tensor
    val: torch.Tensor
    shape: tuple

    @property
    def nnz(self) -> int:
        return int(self.col_idx.numel())

    @property
    def device(self):
        return self.val.device

    @staticmethod
    def from_scipy(A, device="cuda", pin_memory: bool = False) -> "CsrMatrix":
        """Copies a scipy CSR matrix (float64 or float32 values are kept as they are)."""
        import scipy.sparse as sp
        A = sp.csr_matrix(A)
        rp = torch.from_numpy(np.ascontiguousarray(A.indptr, dtype=np.int32))
        ci = torch.from_numpy(np.ascontiguousarray(A.indices, dtype=np.int32))
        vdt = np.float32 if A.data.dtype == np.float32 else np.float64
        va = torch.from_numpy(np.ascontiguousarray(A.data, dtype=vdt))
        if str(device) == "cpu":
            if pin_memory:
                rp, ci, va = rp.pin_memory(), ci.pin_memory(), va.pin_memory()
            return CsrMatrix(rp, ci, va, tuple(A.shape))
        return CsrMatrix(rp.to(device), ci.to(device), va.to(device), tuple(A.shape))

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val.cpu().numpy(), self.col_idx.cpu().numpy(), self.row_ptr.cpu().numpy()),
                             shape=self.shape)


def _ptr(t) -> int:
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _check_csr(A: "CsrMatrix"):
    """The structure checks a pointer-based entry point cannot make: contiguous int32
    index arrays of lengths m + 1 and nnz, float values of length nnz, one device."""
    m, n = A.shape
    for t, dt, name in ((A.row_ptr, torch.int32, "row_ptr"), (A.col_idx, torch.int32, "col_idx")):
        if t.dtype != dt or not t.is_contiguous():
            raise TypeError(f"CsrMatrix needs a contiguous int32 {name}")
    if A.val.dtype not in (torch.float64, torch.float32) or not A.val.is_contiguous():
        raise TypeError("CsrMatrix needs contiguous float64 or float32 values")
    if A.row_ptr.dim() != 1 or A.row_ptr.numel() != m + 1:
        raise ValueError(f"row_ptr must have m + 1 = {m + 1} entries")
    if A.col_idx.dim() != 1 or A.val.dim() != 1 or A.val.numel() != A.col_idx.numel():
        raise ValueError("col_idx and val must be 1-D with nnz entries each")
    if not (A.row_ptr.device == A.col_idx.device == A.val.device):
        raise ValueError("row_ptr, col_idx and val must be on one device")


def _check_rows(t, rows: int, name: str):
    if not isinstance(t, torch.Tensor) or t.dim() != 2 or t.shape[0] != rows:
        shape = tuple(t.shape) if isinstance(t, torch.Tensor) else type(t).__name__
        raise ValueError(f"{name} must be a 2-D tensor with {rows} rows (got {shape})")


def _same_device(dev, *named):
    for t, name in named:
        if t.device != dev:
            raise ValueError(f"{name} is on {t.device}, expected {dev}")


def _desc(A):
    """(TsvdMatrix, keep-alive list, torch.device or None for host)."""
    import scipy.sparse as sp
    d = capi.TsvdMatrix()
    keep = []
    if isinstance(A, torch.Tensor) and A.layout == torch.sparse_csr:
        A = CsrMatrix(A.crow_indices().to(torch.int32), A.col_indices().to(torch.int32),
                      A.values().to(torch.float64), tuple(A.shape))
    if sp.issparse(A):
        A = sp.csr_matrix(A)
        f32 = A.data.dtype == np.float32
        rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
        ci = np.ascontiguousarray(A.indices, dtype=np.int32)
        va = np.ascontiguousarray(A.data, dtype=np.float32 if f32 else np.float64)
        keep += [rp, ci, va]
        d.m, d.n = A.shape
        d.format, d.location = capi.TSVD_CSR, capi.TSVD_HOST
        d.dtype = capi.TSVD_F32 if f32 else capi.TSVD_F64
        d.val, d.row_ptr, d.col_idx, d.nnz = va.ctypes.data, rp.ctypes.data, ci.ctypes.data, ci.size
        return d, keep, None
    if isinstance(A, CsrMatrix):
        _check_csr(A)
        keep += [A.row_ptr, A.col_idx, A.val]
        d.m, d.n = A.shape
        d.format = capi.TSVD_CSR
        d.dtype = capi.TSVD_F32 if A.val.dtype == torch.float32 else capi.TSVD_F64
        dev = A.val.device
        d.location = capi.TSVD_DEVICE if dev.type == "cuda" else capi.TSVD_HOST
        d.val, d.row_ptr, d.col_idx, d.nnz = A.val.data_ptr(), A.row_ptr.data_ptr(), A.col_idx.data_ptr(), A.nnz
        return d, keep, (dev if dev.type == "cuda" else None)
    if isinstance(A, np.ndarray):
        A = np.ascontiguousarray(A, dtype=np.float32 if A.dtype == np.float32 else np.float64)
        keep.append(A)
        d.m, d.n = A.shape
        d.format, d.location = capi.TSVD_DENSE, capi.TSVD_HOST
        d.dtype = capi.TSVD_F32 if A.dtype == np.float32 else capi.TSVD_F64
        d.val, d.ld = A.ctypes.data, A.shape[1]
        return d, keep, None
    if isinstance(A, torch.Tensor):
        if A.dtype not in (torch.float64, torch.float32) or A.dim() != 2 or A.stride(1) != 1:
            raise TypeError("dense A must be a 2-D float64/float32 tensor with unit column stride")
        keep.append(A)
        d.m, d.n = A.shape
        d.format = capi.TSVD_DENSE
        d.dtype = capi.TSVD_F32 if A.dtype == torch.float32 else capi.TSVD_F64
        d.location = capi.TSVD_DEVICE if A.is_cuda else capi.TSVD_HOST
        d.val, d.ld = A.data_ptr(), A.stride(0)
        return d, keep, (A.device if A.is_cuda else None)
    raise TypeError(f"unsupported matrix type {type(A)!r}")


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


@dataclasses.dataclass
class SvdResult:
    sigma: object
    U: object
    V: object
    info: dict
    status: int


_PRECISIONS = {"fp64": capi.TSVD_PREC_FP64, "mixed": capi.TSVD_PREC_MIXED}


class RowPartition:
    """This process's share of a row-partitioned LancSVD: its matrix holds rows
    [row0, row0 + m) of a rows_total x n matrix that other processes hold the rest of.
    ``allreduce(buf)`` sums a float64 numpy array in place over the processes (see
    :func:`torch_allreduce`); the library calls it, through the C ABI's callback, for
    every Gram matrix, projection and A^T product it sums over the rows."""

    def __init__(self, row0: int, rows_total: int, allreduce):
        if not (0 <= int(row0) < int(rows_total)):
            raise ValueError("row0 must lie in [0, rows_total)")
        self.row0, self.rows_total, self.allreduce = int(row0), int(rows_total), allreduce
        self.error = None
        self._cb = capi.ALLREDUCE_FN(self._call)

    def _call(self, ctx, buf, count):
        try:
            self.allreduce(np.ctypeslib.as_array(buf, shape=(int(count),)))
            return 0
        except Exception as e:  # reported to the library as a failed reduction
            self.error = e
            return 1


def torch_allreduce(group=None):
    """A RowPartition allreduce over a torch.distributed process group (CPU tensors:
    a gloo group, or any backend that reduces host memory)."""
    import torch.distributed as dist

    def allreduce(arr):
        dist.all_reduce(torch.from_numpy(arr), op=dist.ReduceOp.SUM, group=group)

    return allreduce


def row_block(rows_total: int, world: int, rank: int):
    """[lo, hi) of rank's rows in an even split of rows_total rows over world ranks."""
    base, extra = divmod(int(rows_total), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _run_driver(fn_name, method, A, k, a, c, seed, tol, max_restarts, qr_block, start_block, output, device,
                profile=False, precision="fp64", restart_keep=0, partition: Optional[RowPartition] = None):
    lib = capi.load()
    desc, keep, dev = _desc(A)
    if dev is None:
        dev = torch.device("cuda", _dev_index(device))
    opts = capi.TsvdOpts()
    lib.tsvd_default_opts(C.byref(opts))
    opts.tol = float(tol)
    opts.max_restarts = int(max_restarts)
    opts.qr_block = int(qr_block)
    opts.output_location = capi.TSVD_HOST if output == "host" else capi.TSVD_DEVICE
    opts.flags = capi.TSVD_FLAG_PROFILE if profile else 0
    if partition is not None:
        if start_block is not None:
            raise ValueError("a row-partitioned solve draws its own start block")
        if int(desc.m) + partition.row0 > partition.rows_total:
            raise ValueError("the matrix's rows do not fit in the partition")
        opts.flags |= capi.TSVD_FLAG_ROW_PARTITION
    if precision not in _PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(_PRECISIONS)}")
    opts.precision = _PRECISIONS[precision]
    opts.restart_keep = int(restart_keep)
    if start_block is not None:
        # LancSVD: max(m, n) x b; RandSVD: min(m, n) x (k + p) (the dimensions after the m < n transpose)
        m_, n_ = int(desc.m), int(desc.n)
        rows = max(m_, n_) if method == capi.TSVD_METHOD_BLANCZOS else min(m_, n_)
        cols = a if method == capi.TSVD_METHOD_BLANCZOS else k + a
        if not isinstance(start_block, torch.Tensor) or tuple(start_block.shape) != (rows, cols):
            raise ValueError(f"start_block must have shape ({rows}, {cols})")
        if not (start_block.is_cuda and start_block.dtype == torch.float64 and start_block.is_contiguous()):
            raise TypeError("start_block must be a contiguous float64 CUDA tensor")
        _same_device(dev, (start_block, "start_block"))
        keep.append(start_block)
        opts.start_block = start_block.data_ptr()
    with torch.cuda.device(dev):
        opts.stream = _stream_ptr(dev)
        nbytes = C.c_size_t()
        capi.check(lib.tsvd_workspace_size(C.byref(desc), method, k, a, c, C.byref(opts), C.byref(nbytes)),
                   "tsvd_workspace_size")
        ws = _ws(nbytes.value, dev)
        m, n = int(desc.m), int(desc.n)
        if output == "host":
            sigma = np.empty(k)
            U = np.empty((m, k))
            V = np.empty((n, k))
        else:
            sigma = torch.empty(k, dtype=torch.float64, device=dev)
            U = torch.empty((m, k), dtype=torch.float64, device=dev)
            V = torch.empty((n, k), dtype=torch.float64, device=dev)
        info = capi.TsvdInfo()
        h = handle(dev)
        if partition is not None:
            capi.check(lib.tsvd_set_row_partition(h, partition.row0, partition.rows_total, partition._cb, None),
                       "tsvd_set_row_partition")
        try:
            rc = getattr(lib, fn_name)(h, C.byref(desc), k, a, c, C.c_uint64(seed), C.byref(opts),
                                       ws.data_ptr(), ws.numel(), _ptr(sigma), _ptr(U), _ptr(V), C.byref(info))
        finally:
            if partition is not None:
                lib.tsvd_set_row_partition(h, 0, 0, capi.ALLREDUCE_FN(), None)
        if partition is not None and partition.error is not None and rc == capi.TSVD_ERR_COMM:
            raise capi.TsvdError(rc, fn_name) from partition.error
        capi.check(rc, fn_name, allow_not_converged=True)
    del keep
    return SvdResult(sigma, U, V, info.as_dict(), rc)


def blanczos(A, k: int, b: int, r: int, seed: int = 0, tol: float = 1e-6, max_restarts: int = 50,
             start_block: Optional[torch.Tensor] = None, output: str = "device", device=None,
             profile: bool = False, precision: str = "fp64", restart_keep: int = 0,
             partition: Optional[RowPartition] = None) -> SvdResult:
    """LancSVD (Alg. 2): k triplets with blocks of width b, r blocks per restart cycle.
    ``profile`` times every kernel class with CUDA events (``info['prof_*']``);
    ``precision="mixed"`` selects the FP32-product form with FP64 small algebra
    and a final FP64 Rayleigh-Ritz step; ``restart_keep=s > 0`` selects the thick
    restart that keeps the s leading Ritz pairs (0: the paper's basic restart).
    ``partition``: A is this process's row block of a row-partitioned matrix
    (FP64; sigma and V replicated, U this process's rows)."""
    return _run_driver("tsvd_blanczos", capi.TSVD_METHOD_BLANCZOS, A, k, b, r, seed, tol, max_restarts, 0,
                       start_block, output, device, profile, precision, restart_keep, partition)


def rsvd(A, k: int, p: int, q: int, seed: int = 0, qr_block: int = 0, start_block: Optional[torch.Tensor] = None,
         output: str = "device", device=None, profile: bool = False, precision: str = "fp64") -> SvdResult:
    """RandSVD (Alg. 1): k triplets, oversampling p, q power steps (q + 1 trips)."""
    return _run_driver("tsvd_rsvd", capi.TSVD_METHOD_RSVD, A, k, p, q, seed, 0.0, 0, qr_block, start_block, output,
                       device, profile, precision)


# ---------------------------------------------------------------------------
# Building blocks (GPU tensors in, GPU tensors out).
# ---------------------------------------------------------------------------
def _cuda_f64(t: torch.Tensor, name: str):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.dim() == 2
            and t.stride(1) == 1):
        raise TypeError(f"{name} must be a 2-D float64 CUDA tensor with unit column stride")


def gaussian_block(rows: int, cols: int, seed: int, stream_id: int, device=None) -> torch.Tensor:
    """N(0,1) block from Philox4x32-10 + Box-Muller (the library's start blocks)."""
    lib = capi.load()
    dev = torch.device("cuda", _dev_index(device))
    out = torch.empty((rows, cols), dtype=torch.float64, device=dev)
    with torch.cuda.device(dev):
        capi.check(lib.tsvd_gaussian_block(rows, cols, C.c_uint64(seed), C.c_uint32(stream_id), out.data_ptr(),
                                           max(cols, 1), _stream_ptr(dev)), "tsvd_gaussian_block")
    return out


def csr_transpose(A: CsrMatrix) -> CsrMatrix:
    """CSR of A^T (rows of A^T list original rows in increasing order)."""
    lib = capi.load()
    _check_csr(A)
    if A.val.dtype != torch.float64 or not A.val.is_cuda:
        raise TypeError("csr_transpose takes a CsrMatrix with float64 values on the GPU")
    dev = A.val.device
    m, n = A.shape
    nnz = A.nnz
    trp = torch.empty(n + 1, dtype=torch.int32, device=dev)
    tci = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    tva = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
    with torch.cuda.device(dev):
        nb = C.c_size_t()
        capi.check(lib.tsvd_csr_transpose_workspace(m, n, nnz, C.byref(nb)), "tsvd_csr_transpose_workspace")
        ws = _ws(nb.value, dev)
        capi.check(lib.tsvd_csr_transpose(handle(dev), m, n, nnz, A.row_ptr.data_ptr(), A.col_idx.data_ptr(),
                                          A.val.data_ptr(), trp.data_ptr(), tci.data_ptr(), tva.data_ptr(),
                                          ws.data_ptr(), ws.numel(), _stream_ptr(dev)), "tsvd_csr_transpose")
    return CsrMatrix(trp, tci[:nnz], tva[:nnz], (n, m))


def spmm(A: CsrMatrix, X: torch.Tensor) -> torch.Tensor:
    """Y = A X for CSR A on the GPU: FP64 values and block (tsvd_spmm), or FP32 values
    and block (tsvd_spmm_f32, the mixed form's SpMM)."""
    lib = capi.load()
    if not isinstance(A, CsrMatrix):
        raise TypeError("A must be a CsrMatrix")
    _check_csr(A)
    _check_rows(X, A.shape[1], "X")
    f32 = A.val.dtype == torch.float32
    if f32:
        if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1):
            raise TypeError("X must be a 2-D float32 CUDA tensor with unit column stride")
    else:
        _cuda_f64(X, "X")
    dev = X.device
    _same_device(dev, (A.val, "A"))
    m, n = A.shape
    w = X.shape[1]
    Y = torch.empty((m, w), dtype=A.val.dtype, device=dev)
    fn = lib.tsvd_spmm_f32 if f32 else lib.tsvd_spmm
    with torch.cuda.device(dev):
        nb = C.c_size_t()
        capi.check(lib.tsvd_spmm_workspace(m, A.nnz, w, C.byref(nb)), "tsvd_spmm_workspace")
        ws = _ws(nb.value, dev)
        capi.check(fn(handle(dev), m, n, A.nnz, A.row_ptr.data_ptr(), A.col_idx.data_ptr(), A.val.data_ptr(), w,
                      X.data_ptr(), X.stride(0), Y.data_ptr(), max(w, 1), ws.data_ptr(), ws.numel(),
                      _stream_ptr(dev)), "tsvd_spmm_f32" if f32 else "tsvd_spmm")
    return Y


def dense_mm(A: torch.Tensor, X: torch.Tensor, trans: bool = False, tensor_cores: bool = False) -> torch.Tensor:
    """op(A) X for dense row-major A on the GPU: FP64 operands (tsvd_dense_mm, or
    with ``tensor_cores=True`` the FP64-accurate sliced product on the tensor cores,
    tsvd_dense_mm_f64tc), or FP32 operands (tsvd_dense_mm_f32, the mixed-precision
    form's kernels)."""
    lib = capi.load()
    if not (isinstance(A, torch.Tensor) and A.dim() == 2):
        raise TypeError("A must be a 2-D tensor")
    _check_rows(X, A.shape[0] if trans else A.shape[1], "X")
    f32 = A.dtype == torch.float32
    if f32:
        for t, name in ((A, "A"), (X, "X")):
            if not (t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.stride(1) == 1):
                raise TypeError(f"{name} must be a 2-D float32 CUDA tensor with unit column stride")
    else:
        _cuda_f64(A, "A")
        _cuda_f64(X, "X")
    dev = A.device
    _same_device(dev, (X, "X"))
    m, n = A.shape
    w = X.shape[1]
    Y = torch.empty(((n if trans else m), w), dtype=A.dtype, device=dev)
    if tensor_cores and f32:
        raise TypeError("the tensor-core product takes float64 operands")
    if tensor_cores:
        fn, name, wsfn = lib.tsvd_dense_mm_f64tc, "tsvd_dense_mm_f64tc", lib.tsvd_dense_mm_f64tc_workspace
    elif f32:
        fn, name, wsfn = lib.tsvd_dense_mm_f32, "tsvd_dense_mm_f32", lib.tsvd_dense_mm_workspace
    else:
        fn, name, wsfn = lib.tsvd_dense_mm, "tsvd_dense_mm", lib.tsvd_dense_mm_workspace
    with torch.cuda.device(dev):
        nb = C.c_size_t()
        capi.check(wsfn(int(trans), m, n, w, C.byref(nb)), name + "_workspace")
        ws = _ws(nb.value, dev)
        capi.check(fn(handle(dev), int(trans), m, n, A.data_ptr(), A.stride(0), w, X.data_ptr(), X.stride(0),
                      Y.data_ptr(), max(w, 1), ws.data_ptr(), ws.numel(), _stream_ptr(dev)), name)
    return Y


# ---------------------------------------------------------------------------
# Gradient with respect to A, and a differentiable truncated SVD.
# ---------------------------------------------------------------------------
def svd_backward(A, sigma: torch.Tensor, U: torch.Tensor, V: torch.Tensor, sigma_bar=None, U_bar=None, V_bar=None,
                 cg_tol: float = 1e-12, cg_max_iter: int = 20000):
    """dL/dA of a loss on the k leading triplets (sigma, U, V) of A, given the
    adjoints dL/dsigma, dL/dU, dL/dV (None = 0): the values on A's pattern for a
    CsrMatrix (CSR order), the dense m x n gradient for a dense A.  Returns
    (grad, info)."""
    lib = capi.load()
    desc, keep, dev = _desc(A)
    if dev is None:
        raise TypeError("A must be on the GPU")
    k = int(sigma.numel())
    m, n = int(desc.m), int(desc.n)

    def f64(t, shape, name):
        if t is None:
            return None
        t = t.detach().to(device=dev, dtype=torch.float64).contiguous()
        if tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {shape}")
        return t

    s_, U_, V_ = f64(sigma, (k,), "sigma"), f64(U, (m, k), "U"), f64(V, (n, k), "V")
    sb, Ub, Vb = f64(sigma_bar, (k,), "sigma_bar"), f64(U_bar, (m, k), "U_bar"), f64(V_bar, (n, k), "V_bar")
    opts = capi.TsvdBackwardOpts()
    lib.tsvd_default_backward_opts(C.byref(opts))
    opts.cg_tol = float(cg_tol)
    opts.cg_max_iter = int(cg_max_iter)
    sparse = isinstance(A, CsrMatrix)
    grad = torch.empty((A.nnz,) if sparse else (m, n), dtype=torch.float64, device=dev)
    info = capi.TsvdBackwardInfo()
    with torch.cuda.device(dev):
        opts.stream = _stream_ptr(dev)
        nb = C.c_size_t()
        capi.check(lib.tsvd_svd_backward_workspace(C.byref(desc), k, C.byref(opts), C.byref(nb)),
                   "tsvd_svd_backward_workspace")
        ws = _ws(nb.value, dev)
        rc = lib.tsvd_svd_backward(handle(dev), C.byref(desc), k, _ptr(s_), _ptr(U_), _ptr(V_),
                                   _ptr(sb) if sb is not None else None, _ptr(Ub) if Ub is not None else None,
                                   _ptr(Vb) if Vb is not None else None, grad.data_ptr(), C.byref(opts),
                                   ws.data_ptr(), ws.numel(), C.byref(info))
        capi.check(rc, "tsvd_svd_backward", allow_not_converged=True)
    del keep
    return grad, info.as_dict()


class _TruncatedSVD(torch.autograd.Function):
    @staticmethod
    def forward(ctx, data, structure, k, solve, bwd):
        A = data if structure is None else CsrMatrix(structure[0], structure[1], data, structure[2])
        res = blanczos(A, k, **solve)
        if res.status != 0:
            raise capi.TsvdError(res.status, "truncated_svd (LancSVD did not converge)")
        ctx.structure = structure
        ctx.bwd = bwd
        ctx.save_for_backward(data, res.sigma, res.U, res.V)
        return res.sigma, res.U, res.V

    @staticmethod
    def backward(ctx, gs, gU, gV):
        data, sigma, U, V = ctx.saved_tensors
        st = ctx.structure
        A = data if st is None else CsrMatrix(st[0], st[1], data, st[2])
        grad, _ = svd_backward(A, sigma, U, V, gs, gU, gV, **ctx.bwd)
        return grad.to(data.dtype), None, None, None, None


def truncated_svd(A, k: int, b: int, r: int, seed: int = 0, tol: float = 1e-10, max_restarts: int = 200,
                  restart_keep: int = 0, cg_tol: float = 1e-12):
    """Differentiable k leading singular triplets (sigma, U, V) by LancSVD (FP64).

    A: a dense CUDA tensor, or a CsrMatrix whose ``val`` may require grad.
    Gradients with respect to A (dense) or to the CSR values flow through
    tsvd_svd_backward (exact for the truncated SVD; complement terms by CG).
    The loss should not depend on the signs of the singular vectors (the sign
    convention makes them locally constant)."""
    solve = dict(b=b, r=r, seed=seed, tol=tol, max_restarts=max_restarts, restart_keep=restart_keep)
    bwd = dict(cg_tol=cg_tol)
    if isinstance(A, CsrMatrix):
        return _TruncatedSVD.apply(A.val, (A.row_ptr, A.col_idx, A.shape), k, solve, bwd)
    return _TruncatedSVD.apply(A, None, k, solve, bwd)


@dataclasses.dataclass
class Bf16x3:
    """Three BF16 pieces of a rows x cols matrix (A = A0 + A1 + A2), as stored by
    tsvd_bf16x3_split: ``data`` is the device buffer [3][rows][ld] (ld = cols
    rounded up to a multiple of 8)."""
    data: torch.Tensor
    rows: int
    cols: int

    @property
    def ld(self) -> int:
        return (self.cols + 7) // 8 * 8

    def pieces(self) -> torch.Tensor:
        """The pieces as a (3, rows, cols) bfloat16 tensor (a view of ``data``)."""
        n = 3 * self.rows * self.ld
        return self.data[: 2 * n].view(torch.bfloat16).view(3, self.rows, self.ld)[:, :, : self.cols]


def bf16x3_split(A: torch.Tensor, trans: bool = False) -> Bf16x3:
    """BF16 pieces of FP64 A (or of A^T) for the tensor-core products."""
    lib = capi.load()
    _cuda_f64(A, "A")
    dev = A.device
    m, n = A.shape
    rows, cols = (n, m) if trans else (m, n)
    nb = C.c_size_t()
    capi.check(lib.tsvd_bf16x3_bytes(rows, cols, C.byref(nb)), "tsvd_bf16x3_bytes")
    buf = _ws(nb.value, dev)
    with torch.cuda.device(dev):
        capi.check(lib.tsvd_bf16x3_split(handle(dev), int(trans), m, n, A.data_ptr(), A.stride(0), buf.data_ptr(),
                                         _stream_ptr(dev)), "tsvd_bf16x3_split")
    return Bf16x3(buf, rows, cols)


def mm_bf16x6(P: Bf16x3, X: torch.Tensor) -> torch.Tensor:
    """Y = P X on the tensor cores (six BF16 cross terms, FP32 accumulation); X FP32."""
    lib = capi.load()
    if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1):
        raise TypeError("X must be a 2-D float32 CUDA tensor with unit column stride")
    if X.shape[0] != P.cols:
        raise ValueError("X must have P.cols rows")
    dev = X.device
    _same_device(dev, (P.data, "P"))
    w = X.shape[1]
    Y = torch.empty((P.rows, w), dtype=torch.float32, device=dev)
    nb = C.c_size_t()
    capi.check(lib.tsvd_mm_bf16x6_workspace(P.rows, P.cols, w, C.byref(nb)), "tsvd_mm_bf16x6_workspace")
    ws = _ws(nb.value, dev)
    with torch.cuda.device(dev):
        capi.check(lib.tsvd_mm_bf16x6(handle(dev), P.rows, P.cols, P.data.data_ptr(), w, X.data_ptr(), X.stride(0),
                                      Y.data_ptr(), max(w, 1), ws.data_ptr(), ws.numel(), _stream_ptr(dev)),
                   "tsvd_mm_bf16x6")
    return Y


def _orth_ws(q, s, b, dev):
    nb = C.c_size_t()
    capi.check(capi.load().tsvd_orth_workspace(q, s, b, C.byref(nb)), "tsvd_orth_workspace")
    return _ws(nb.value + 256 * 4 + 8 * (s + b) * b, dev)


def cholqr2(Y: torch.Tensor, seed: int = 0):
    """CholeskyQR2 (Alg. 4) of a copy of Y: returns (Q, R, breakdowns)."""
    lib = capi.load()
    _cuda_f64(Y, "Y")
    dev = Y.device
    Q = Y.clone()
    q, b = Q.shape
    R = torch.empty((b, b), dtype=torch.float64, device=dev)
    rep, bd = C.c_int(0), C.c_int(0)
    with torch.cuda.device(dev):
        ws = _orth_ws(q, 0, b, dev)
        capi.check(lib.tsvd_cholqr2(handle(dev), q, b, Q.data_ptr(), Q.stride(0), R.data_ptr(), C.c_uint64(seed),
                                    C.byref(rep), C.byref(bd), ws.data_ptr(), ws.numel(), _stream_ptr(dev)),
                   "tsvd_cholqr2")
    return Q, R, bd.value


def _cuda_f32(t: torch.Tensor, name: str):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.dim() == 2
            and t.stride(1) == 1):
        raise TypeError(f"{name} must be a row-major float32 CUDA matrix")


def cgs_cqr2(Y: torch.Tensor, P: torch.Tensor, seed: int = 0):
    """CGS-CQR2 (Alg. 5) of a copy of Y against P: returns (Q, H, R, breakdowns).
    float32 Y and P run the mixed form's FP32-block variant (tsvd_cgs_cqr2_f32;
    H and R are float64 either way); P may have 0 columns (CholeskyQR2)."""
    lib = capi.load()
    if not (isinstance(Y, torch.Tensor) and Y.dim() == 2):
        raise TypeError("Y must be a 2-D tensor")
    _check_rows(P, Y.shape[0], "P")
    if Y.dtype == torch.float32:
        _cuda_f32(Y, "Y")
        _cuda_f32(P, "P")
        fn, name = lib.tsvd_cgs_cqr2_f32, "tsvd_cgs_cqr2_f32"
    else:
        _cuda_f64(Y, "Y")
        _cuda_f64(P, "P")
        fn, name = lib.tsvd_cgs_cqr2, "tsvd_cgs_cqr2"
    dev = Y.device
    _same_device(dev, (P, "P"))
    Q = Y.clone()
    q, b = Q.shape
    s = P.shape[1]
    R = torch.empty((b, b), dtype=torch.float64, device=dev)
    H = torch.empty((max(s, 1), b), dtype=torch.float64, device=dev)
    rep, bd = C.c_int(0), C.c_int(0)
    with torch.cuda.device(dev):
        ws = _orth_ws(q, s, b, dev)
        capi.check(fn(handle(dev), q, s, b, P.data_ptr(), max(P.stride(0), s), Q.data_ptr(), Q.stride(0),
                      H.data_ptr(), R.data_ptr(), C.c_uint64(seed), C.byref(rep), C.byref(bd),
                      ws.data_ptr(), ws.numel(), _stream_ptr(dev)), name)
    return Q, H[:s], R, bd.value


def update_gram_f32(X: torch.Tensor, M: torch.Tensor, Y: Optional[torch.Tensor] = None, alpha: float = 1.0,
                    beta: float = 0.0, upper: bool = False, in_place: bool = False, overwrite_y: bool = False):
    """Fused update + Gram of FP32 blocks (tsvd_update_gram_f32): returns (Y', W) with
    Y' = beta Y + alpha X M (FP32) and W = Y'^T Y' (float64).  Y' is a new tensor
    (a copy of Y, or zeros when Y is None) unless ``overwrite_y`` (Y itself is updated)
    or ``in_place`` (X itself is updated; M square, Y unused)."""
    lib = capi.load()
    _cuda_f32(X, "X")
    _cuda_f64(M, "M")
    dev = X.device
    _same_device(dev, (M, "M"))
    q, s = X.shape
    if M.shape[0] != s:
        raise ValueError(f"M must have {s} rows")
    b = M.shape[1]
    if in_place:
        if s != b:
            raise ValueError("an in-place update needs a square M")
        Yo = X
    elif Y is None:
        Yo = torch.zeros((q, b), dtype=torch.float32, device=dev)
    else:
        _cuda_f32(Y, "Y")
        _check_rows(Y, q, "Y")
        if Y.shape[1] != b:
            raise ValueError(f"Y must have {b} columns")
        Yo = Y if overwrite_y else Y.clone()
    W = torch.empty((b, b), dtype=torch.float64, device=dev)
    nb = C.c_size_t()
    capi.check(lib.tsvd_update_gram_f32_workspace(q, b, C.byref(nb)), "tsvd_update_gram_f32_workspace")
    with torch.cuda.device(dev):
        ws = _ws(nb.value, dev)
        capi.check(lib.tsvd_update_gram_f32(handle(dev), q, s, b, float(alpha), X.data_ptr(), X.stride(0),
                                            M.data_ptr(), M.stride(0), float(beta), Yo.data_ptr(), Yo.stride(0),
                                            int(bool(upper)), W.data_ptr(), ws.data_ptr(), ws.numel(),
                                            _stream_ptr(dev)), "tsvd_update_gram_f32")
    return Yo, W


def cgs_qr(Y: torch.Tensor, b: int, seed: int = 0):
    """CGS-QR (Alg. 3) of a copy of Y with column blocks of width b: returns (Q, R, breakdowns)."""
    lib = capi.load()
    _cuda_f64(Y, "Y")
    dev = Y.device
    Q = Y.clone()
    q, r = Q.shape
    R = torch.empty((r, r), dtype=torch.float64, device=dev)
    rep, bd = C.c_int(0), C.c_int(0)
    with torch.cuda.device(dev):
        ws = _orth_ws(q, r, min(b, r), dev)
        capi.check(lib.tsvd_cgs_qr(handle(dev), q, r, b, Q.data_ptr(), Q.stride(0), R.data_ptr(), C.c_uint64(seed),
                                   C.byref(rep), C.byref(bd), ws.data_ptr(), ws.numel(), _stream_ptr(dev)),
                   "tsvd_cgs_qr")
    return Q, R, bd.value


def small_svd(B: torch.Tensor, nv: Optional[int] = None):
    """SVD of a small square matrix by the device Jacobi kernels: (Ubar, sigma, Vbar, sweeps).
    ``nv`` < n returns only the leading nv right vectors (the methods' mode)."""
    lib = capi.load()
    _cuda_f64(B, "B")
    dev = B.device
    n = B.shape[0]
    if B.shape[1] != n:
        raise ValueError("B must be square")
    nv = n if nv is None else int(nv)
    U = torch.empty((n, n), dtype=torch.float64, device=dev)
    V = torch.empty((n, n), dtype=torch.float64, device=dev)
    s = torch.empty(n, dtype=torch.float64, device=dev)
    sweeps = C.c_int(0)
    with torch.cuda.device(dev):
        nb = C.c_size_t()
        capi.check(lib.tsvd_small_svd_workspace(n, C.byref(nb)), "tsvd_small_svd_workspace")
        ws = _ws(nb.value, dev)
        capi.check(lib.tsvd_small_svd(handle(dev), n, B.data_ptr(), B.stride(0), nv, U.data_ptr(), s.data_ptr(),
                                      V.data_ptr(), C.byref(sweeps), ws.data_ptr(), ws.numel(), _stream_ptr(dev)),
                   "tsvd_small_svd")
    return U, s, V, sweeps.value
