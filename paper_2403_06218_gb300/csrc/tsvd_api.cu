// C ABI (include/tsvd.h): handle, workspace sizing, argument checks, the entry
// points of RandSVD and LancSVD (the methods themselves are in drivers.cu) and
// the building-block entry points.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <algorithm>

#include "tsvd_internal.cuh"

namespace tsvd {
int jacobi_coop_capacity(int device, int sm_count);
template <typename T>
int rsvd_run(tsvd_handle* h, const tsvd_matrix* A, int k, int p, int q, int bq, uint64_t seed, const tsvd_opts* o,
             char* ws, size_t ws_bytes, size_t* sizing, double* sigma, double* U, double* V, tsvd_info* info);
template <typename T>
int blanczos_run(tsvd_handle* h, const tsvd_matrix* A, int k, int b, int r, uint64_t seed, const tsvd_opts* o,
                 char* ws, size_t ws_bytes, size_t* sizing, double* sigma, double* U, double* V, tsvd_info* info);
}

using namespace tsvd;

int tsvd::part_sum(tsvd_handle* h, double* d, int64_t rows, int64_t cols, int64_t ld, cudaStream_t st) {
    if (!h->part_fn || rows * cols == 0) return TSVD_OK;
    const size_t cnt = (size_t)rows * (size_t)cols;
    h->part_host.resize(cnt);
    double* hb = h->part_host.data();
    const size_t w = sizeof(double) * (size_t)cols;
    TSVD_TRY_CUDA(cudaMemcpy2DAsync(hb, w, d, sizeof(double) * (size_t)ld, w, (size_t)rows, cudaMemcpyDeviceToHost,
                                    st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    if (h->part_fn(h->part_ctx, hb, (int64_t)cnt) != 0) return TSVD_ERR_COMM;
    TSVD_TRY_CUDA(cudaMemcpy2DAsync(d, sizeof(double) * (size_t)ld, hb, w, w, (size_t)rows, cudaMemcpyHostToDevice,
                                    st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}

void tsvd::prof_collect(tsvd_handle* h, tsvd_info* info) {
    for (auto& r : h->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        if (info && r.cls >= 0 && r.cls < TSVD_K_COUNT) {
            info->prof_launches[r.cls] += 1;
            info->prof_ms[r.cls] += ms;
            info->prof_flops[r.cls] += r.flops;
            info->prof_bytes[r.cls] += r.bytes;
        }
        h->pool.push_back(r.e0);
        h->pool.push_back(r.e1);
    }
    h->recs.clear();
}

namespace {

// Turns kernel-class profiling on for one driver call and off again on every exit path.
struct ProfileGuard {
    tsvd_handle* h;
    ProfileGuard(tsvd_handle* hh, bool on) : h(hh) {
        h->recs.clear();
        h->profiling = on;
    }
    ~ProfileGuard() {
        h->profiling = false;
        for (auto& r : h->recs) {
            h->pool.push_back(r.e0);
            h->pool.push_back(r.e1);
        }
        h->recs.clear();
    }
};

int validate_matrix(const tsvd_matrix* A) {
    if (A == nullptr) return TSVD_ERR_INVALID_ARG;
    if (A->m < 1 || A->n < 1) return TSVD_ERR_INVALID_ARG;
    if (A->dtype != TSVD_F64 && A->dtype != TSVD_F32) return TSVD_ERR_UNSUPPORTED;
    if (A->location != TSVD_DEVICE && A->location != TSVD_HOST) return TSVD_ERR_INVALID_ARG;
    if (A->val == nullptr) return TSVD_ERR_INVALID_ARG;
    if (A->format == TSVD_DENSE) {
        if (A->ld < A->n) return TSVD_ERR_INVALID_ARG;
    } else if (A->format == TSVD_CSR) {
        if (A->row_ptr == nullptr || A->col_idx == nullptr) return TSVD_ERR_INVALID_ARG;
        if (A->nnz < 0 || A->nnz > 2147483647LL) return TSVD_ERR_UNSUPPORTED;
        if (A->m > 2147483647LL || A->n > 2147483647LL) return TSVD_ERR_UNSUPPORTED;
    } else {
        return TSVD_ERR_INVALID_ARG;
    }
    return TSVD_OK;
}

int check_rsvd_args(const tsvd_matrix* A, int k, int p, int q, const tsvd_opts* o) {
    TSVD_TRY(validate_matrix(A));
    const int64_t mn = A->m < A->n ? A->m : A->n;
    if (k < 1 || p < 0 || q < 0 || (int64_t)k + p > mn) return TSVD_ERR_INVALID_ARG;
    if (k + p > TSVD_MAX_SMALL_SVD) return TSVD_ERR_UNSUPPORTED;
    if (o->qr_block < 0) return TSVD_ERR_INVALID_ARG;
    if (o->precision != TSVD_PREC_FP64 && o->precision != TSVD_PREC_MIXED) return TSVD_ERR_INVALID_ARG;
    if (o->precision == TSVD_PREC_MIXED && k > TSVD_MAX_BLOCK) return TSVD_ERR_UNSUPPORTED;
    return TSVD_OK;
}

int check_lanc_args(const tsvd_matrix* A, int k, int b, int r, const tsvd_opts* o) {
    TSVD_TRY(validate_matrix(A));
    const int64_t mn = A->m < A->n ? A->m : A->n;
    if (b < 1 || r < 1 || k < 1) return TSVD_ERR_INVALID_ARG;
    if (b > TSVD_MAX_BLOCK) return TSVD_ERR_UNSUPPORTED;
    if ((int64_t)r * b > mn || k > r * b) return TSVD_ERR_INVALID_ARG;
    if (r * b > TSVD_MAX_SMALL_SVD) return TSVD_ERR_UNSUPPORTED;
    if (o->max_restarts < 0 || !(o->tol >= 0.0)) return TSVD_ERR_INVALID_ARG;
    if (o->precision != TSVD_PREC_FP64 && o->precision != TSVD_PREC_MIXED) return TSVD_ERR_INVALID_ARG;
    if (o->precision == TSVD_PREC_MIXED && k > TSVD_MAX_BLOCK) return TSVD_ERR_UNSUPPORTED;
    if (o->restart_keep < 0) return TSVD_ERR_INVALID_ARG;
    if (o->restart_keep > 0 && (o->restart_keep < k || o->restart_keep + b > r * b)) return TSVD_ERR_INVALID_ARG;
    return TSVD_OK;
}

int qr_block_of(const tsvd_opts* o, int ell) {
    int bq = (o->qr_block > 0) ? o->qr_block : ell;
    if (bq > ell) bq = ell;
    if (bq > TSVD_MAX_BLOCK) bq = TSVD_MAX_BLOCK;
    return bq;
}

// Handle for sizing without a device call that needs one (SM count of the current device, else 152).
tsvd_handle sizing_handle() {
    tsvd_handle hh{};
    hh.sm_count = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        int sm = 0;
        if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sm > 0) hh.sm_count = sm;
    }
    hh.jacobi_coop_blocks = 1 << 20;
    return hh;
}

}  // namespace

// ===========================================================================
extern "C" {

void tsvd_default_opts(tsvd_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->max_restarts = 50;
    o->qr_block = 0;
    o->output_location = TSVD_DEVICE;
}

const char* tsvd_status_string(int s) {
    switch (s) {
        case TSVD_OK: return "ok";
        case TSVD_NOT_CONVERGED: return "not converged";
        case TSVD_ERR_INVALID_ARG: return "invalid argument";
        case TSVD_ERR_NONFINITE: return "non-finite value";
        case TSVD_ERR_CUDA: return "CUDA error";
        case TSVD_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
        case TSVD_ERR_TIMEOUT: return "device wait timed out";
        case TSVD_ERR_UNSUPPORTED: return "unsupported size";
        case TSVD_ERR_COMM: return "row-partition reduction failed";
        default: return "unknown status";
    }
}

int tsvd_create(tsvd_handle** out, int device) {
    if (!out) return TSVD_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return TSVD_ERR_CUDA;
    int prev = 0;
    TSVD_TRY_CUDA(cudaGetDevice(&prev));
    TSVD_TRY_CUDA(cudaSetDevice(device));
    tsvd_handle* h = new (std::nothrow) tsvd_handle();
    if (!h) return TSVD_ERR_CUDA;
    h->device = device;
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    h->jacobi_coop_blocks = jacobi_coop_capacity(device, h->sm_count);
    h->launches = 0;
    cudaSetDevice(prev);
    *out = h;
    return TSVD_OK;
}

int tsvd_destroy(tsvd_handle* h) {
    delete h;
    return TSVD_OK;
}

int tsvd_set_row_partition(tsvd_handle* h, int64_t row0, int64_t rows_total, tsvd_allreduce_fn fn, void* ctx) {
    if (!h) return TSVD_ERR_INVALID_ARG;
    if (fn && (row0 < 0 || rows_total < 1 || row0 >= rows_total)) return TSVD_ERR_INVALID_ARG;
    h->part_fn = fn;
    h->part_ctx = fn ? ctx : nullptr;
    h->part_row0 = fn ? row0 : 0;
    h->part_rows = fn ? rows_total : 0;
    return TSVD_OK;
}

int tsvd_set_wait_limit(tsvd_handle* h, long long cycles) {
    if (!h) return TSVD_ERR_INVALID_ARG;
    h->max_wait = cycles > 0 ? cycles : tsvd_handle{}.max_wait;
    return TSVD_OK;
}

int tsvd_workspace_size(const tsvd_matrix* A, int method, int k, int a, int c, const tsvd_opts* opts, size_t* bytes) {
    if (!bytes) return TSVD_ERR_INVALID_ARG;
    tsvd_opts o;
    tsvd_default_opts(&o);
    if (opts) o = *opts;
    tsvd_handle hh = sizing_handle();
    const bool mixed = o.precision == TSVD_PREC_MIXED;
    if (method == TSVD_METHOD_RSVD) {
        TSVD_TRY(check_rsvd_args(A, k, a, c, &o));
        const int bq = qr_block_of(&o, k + a);
        return mixed ? rsvd_run<float>(&hh, A, k, a, c, bq, 0, &o, nullptr, 0, bytes, nullptr, nullptr, nullptr, nullptr)
                     : rsvd_run<double>(&hh, A, k, a, c, bq, 0, &o, nullptr, 0, bytes, nullptr, nullptr, nullptr,
                                        nullptr);
    }
    if (method == TSVD_METHOD_BLANCZOS) {
        TSVD_TRY(check_lanc_args(A, k, a, c, &o));
        return mixed ? blanczos_run<float>(&hh, A, k, a, c, 0, &o, nullptr, 0, bytes, nullptr, nullptr, nullptr, nullptr)
                     : blanczos_run<double>(&hh, A, k, a, c, 0, &o, nullptr, 0, bytes, nullptr, nullptr, nullptr,
                                            nullptr);
    }
    return TSVD_ERR_INVALID_ARG;
}

int tsvd_rsvd(tsvd_handle* h, const tsvd_matrix* A, int k, int p, int q, uint64_t seed, const tsvd_opts* opts,
              void* ws, size_t ws_bytes, double* sigma, double* U, double* V, tsvd_info* info) {
    if (!h || !sigma || !U || !V) return TSVD_ERR_INVALID_ARG;
    tsvd_opts o;
    tsvd_default_opts(&o);
    if (opts) o = *opts;
    TSVD_TRY(check_rsvd_args(A, k, p, q, &o));
    size_t need = 0;
    TSVD_TRY(tsvd_workspace_size(A, TSVD_METHOD_RSVD, k, p, q, &o, &need));
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    DeviceGuard dg(h->device);
    if (!dg.ok()) return TSVD_ERR_CUDA;
    ProfileGuard pg(h, (o.flags & TSVD_FLAG_PROFILE) != 0);
    const int bq = qr_block_of(&o, k + p);
    char* w = static_cast<char*>(ws);
    if (o.precision == TSVD_PREC_MIXED)
        return rsvd_run<float>(h, A, k, p, q, bq, seed, &o, w, ws_bytes, nullptr, sigma, U, V, info);
    return rsvd_run<double>(h, A, k, p, q, bq, seed, &o, w, ws_bytes, nullptr, sigma, U, V, info);
}

int tsvd_blanczos(tsvd_handle* h, const tsvd_matrix* A, int k, int b, int r, uint64_t seed, const tsvd_opts* opts,
                  void* ws, size_t ws_bytes, double* sigma, double* U, double* V, tsvd_info* info) {
    if (!h || !sigma || !U || !V) return TSVD_ERR_INVALID_ARG;
    tsvd_opts o;
    tsvd_default_opts(&o);
    if (opts) o = *opts;
    TSVD_TRY(check_lanc_args(A, k, b, r, &o));
    size_t need = 0;
    TSVD_TRY(tsvd_workspace_size(A, TSVD_METHOD_BLANCZOS, k, b, r, &o, &need));
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    DeviceGuard dg(h->device);
    if (!dg.ok()) return TSVD_ERR_CUDA;
    ProfileGuard pg(h, (o.flags & TSVD_FLAG_PROFILE) != 0);
    char* w = static_cast<char*>(ws);
    if (o.precision == TSVD_PREC_MIXED)
        return blanczos_run<float>(h, A, k, b, r, seed, &o, w, ws_bytes, nullptr, sigma, U, V, info);
    return blanczos_run<double>(h, A, k, b, r, seed, &o, w, ws_bytes, nullptr, sigma, U, V, info);
}

// ---------------------------------------------------------------------------
// Gradient with respect to A.
// ---------------------------------------------------------------------------
void tsvd_default_backward_opts(tsvd_backward_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->cg_tol = 1e-12;
    o->cg_max_iter = 20000;
    o->check_every = 10;
    o->stream = nullptr;
}

static int check_backward_args(const tsvd_matrix* A, int k, const tsvd_backward_opts* o) {
    TSVD_TRY(validate_matrix(A));
    const int64_t mn = A->m < A->n ? A->m : A->n;
    if (k < 1 || k > mn) return TSVD_ERR_INVALID_ARG;
    if (k > TSVD_MAX_BLOCK) return TSVD_ERR_UNSUPPORTED;  // 2k factor columns per SDDMM row
    if (!(o->cg_tol > 0.0) || o->cg_max_iter < 0) return TSVD_ERR_INVALID_ARG;
    return TSVD_OK;
}

int tsvd_svd_backward_workspace(const tsvd_matrix* A, int k, const tsvd_backward_opts* opts, size_t* bytes) {
    if (!A || !bytes) return TSVD_ERR_INVALID_ARG;
    tsvd_backward_opts o;
    tsvd_default_backward_opts(&o);
    if (opts) o = *opts;
    TSVD_TRY(check_backward_args(A, k, &o));
    tsvd_handle hh = sizing_handle();
    return svd_backward_run(&hh, A, k, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, &o, nullptr, 0,
                            bytes, nullptr);
}

int tsvd_svd_backward(tsvd_handle* h, const tsvd_matrix* A, int k, const double* sigma, const double* U,
                      const double* V, const double* sigma_bar, const double* U_bar, const double* V_bar,
                      double* grad, const tsvd_backward_opts* opts, void* ws, size_t ws_bytes,
                      tsvd_backward_info* info) {
    if (!h || !A || !sigma || !U || !V || !grad) return TSVD_ERR_INVALID_ARG;
    tsvd_backward_opts o;
    tsvd_default_backward_opts(&o);
    if (opts) o = *opts;
    TSVD_TRY(check_backward_args(A, k, &o));
    size_t need = 0;
    TSVD_TRY(tsvd_svd_backward_workspace(A, k, &o, &need));
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    DeviceGuard dg(h->device);
    if (!dg.ok()) return TSVD_ERR_CUDA;
    if (info) std::memset(info, 0, sizeof(*info));
    return svd_backward_run(h, A, k, sigma, U, V, sigma_bar, U_bar, V_bar, grad, &o, static_cast<char*>(ws), ws_bytes,
                            nullptr, info);
}

// ---------------------------------------------------------------------------
// Building blocks.
// ---------------------------------------------------------------------------
int tsvd_gaussian_block(int64_t rows, int64_t cols, uint64_t seed, uint32_t stream_id, double* out, int64_t ld,
                        void* stream) {
    if (rows < 0 || cols < 0 || (rows * cols > 0 && (out == nullptr || ld < cols))) return TSVD_ERR_INVALID_ARG;
    tsvd_handle hh{};
    int dev = 0;
    TSVD_TRY_CUDA(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&hh.sm_count, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TSVD_TRY_CUDA(gaussian(&hh, rows, cols, seed, stream_id, out, ld, st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}

int tsvd_csr_transpose_workspace(int64_t m, int64_t n, int64_t nnz, size_t* bytes) {
    if (!bytes || m < 0 || n < 0 || nnz < 0) return TSVD_ERR_INVALID_ARG;
    *bytes = align256(sizeof(int) * kStCount) + csr_transpose_ws(m, n, nnz);
    return TSVD_OK;
}

int tsvd_csr_transpose(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr,
                       const int32_t* col_idx, const double* val, int32_t* t_row_ptr, int32_t* t_col_idx,
                       double* t_val, void* ws, size_t ws_bytes, void* stream) {
    if (!h || m < 0 || n < 0 || nnz < 0 || nnz > 2147483647LL || !row_ptr || !t_row_ptr) return TSVD_ERR_INVALID_ARG;
    if (nnz > 0 && (!col_idx || !val || !t_col_idx || !t_val)) return TSVD_ERR_INVALID_ARG;
    size_t need = 0;
    TSVD_TRY(tsvd_csr_transpose_workspace(m, n, nnz, &need));
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Arena ar{static_cast<char*>(ws), ws_bytes, 0};
    int* status = ar.take<int>(kStCount);
    TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    TSVD_TRY(csr_transpose<double>(h, m, n, nnz, row_ptr, col_idx, val, t_row_ptr, t_col_idx, t_val, ar, status, st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}

int tsvd_spmm_workspace(int64_t m, int64_t nnz, int w, size_t* bytes) {
    if (!bytes || m < 0 || nnz < 0 || w < 0) return TSVD_ERR_INVALID_ARG;
    *bytes = align256(sizeof(int) * kStCount) + spmm_plan_ws(m, nnz, w, sizeof(double));
    return TSVD_OK;
}

extern "C++" template <typename T>
int spmm_entry(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr,
                      const int32_t* col_idx, const T* val, int w, const T* X, int64_t ldx, T* Y, int64_t ldy,
                      void* ws, size_t ws_bytes, void* stream) {
    if (!h || m < 0 || n < 0 || nnz < 0 || w < 0 || ldx < w || ldy < w || !row_ptr) return TSVD_ERR_INVALID_ARG;
    if (m * (int64_t)w > 0 && (!X || !Y)) return TSVD_ERR_INVALID_ARG;
    size_t need = 0;
    TSVD_TRY(tsvd_spmm_workspace(m, nnz, w, &need));
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* status = static_cast<int*>(ws);
    TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    Arena ar{static_cast<char*>(ws), ws_bytes, align256(sizeof(int) * kStCount)};
    SpmmPlan plan;
    TSVD_TRY(spmm_plan(h, m, nnz, row_ptr, w, sizeof(double), ar, &plan, st));
    TSVD_TRY_CUDA(launch_spmm<T>(h, m, n, nnz, row_ptr, col_idx, val, w, X, ldx, Y, ldy, status, st, &plan));
    int hs[kStCount];
    TSVD_TRY(read_status(st, status, hs));
    return hs[kStBadCsr] ? TSVD_ERR_INVALID_ARG : TSVD_OK;
}

int tsvd_spmm_f32(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                  const float* val, int w, const float* X, int64_t ldx, float* Y, int64_t ldy, void* ws,
                  size_t ws_bytes, void* stream) {
    return spmm_entry<float>(h, m, n, nnz, row_ptr, col_idx, val, w, X, ldx, Y, ldy, ws, ws_bytes, stream);
}

int tsvd_spmm(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
              const double* val, int w, const double* X, int64_t ldx, double* Y, int64_t ldy, void* ws,
              size_t ws_bytes, void* stream) {
    return spmm_entry<double>(h, m, n, nnz, row_ptr, col_idx, val, w, X, ldx, Y, ldy, ws, ws_bytes, stream);
}

int tsvd_dense_mm_workspace(int trans, int64_t m, int64_t n, int w, size_t* bytes) {
    if (!bytes || m < 0 || n < 0 || w < 0) return TSVD_ERR_INVALID_ARG;
    tsvd_handle hh{};
    hh.sm_count = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&hh.sm_count, cudaDevAttrMultiProcessorCount, dev);
    *bytes = trans ? std::max(gemm_tn_ws(&hh, m, n, w, false, 8), gemm_tn_ws(&hh, m, n, w, false, 4)) : 0;
    return TSVD_OK;
}

int tsvd_dense_mm(tsvd_handle* h, int trans, int64_t m, int64_t n, const double* A, int64_t lda, int w,
                  const double* X, int64_t ldx, double* Y, int64_t ldy, void* ws, size_t ws_bytes, void* stream) {
    if (!h || m < 0 || n < 0 || w < 0 || lda < n || !A || !X || !Y) return TSVD_ERR_INVALID_ARG;
    if (ldx < w || ldy < w) return TSVD_ERR_INVALID_ARG;
    size_t need = trans ? gemm_tn_ws(h, m, n, w, false) : 0;
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (trans)
        TSVD_TRY_CUDA((gemm_tn<double, double>(h, m, n, w, A, lda, X, ldx, Y, ldy, false, static_cast<double*>(ws), st)));
    else
        TSVD_TRY_CUDA((gemm_nn<double, double, double>(h, m, n, w, 1.0, A, lda, X, ldx, 0.0, Y, ldy, false, st)));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}

int tsvd_dense_mm_f64tc_workspace(int trans, int64_t m, int64_t n, int w, size_t* bytes) {
    if (!bytes || m < 0 || n < 0 || w < 0) return TSVD_ERR_INVALID_ARG;
    // 256 bytes of status words, then the product's scratch
    *bytes = 256 + (trans ? oz_tn_ws(m, n, w, false) : oz_nn_ws(m, n, w));
    return TSVD_OK;
}

int tsvd_dense_mm_f64tc(tsvd_handle* h, int trans, int64_t m, int64_t n, const double* A, int64_t lda, int w,
                        const double* X, int64_t ldx, double* Y, int64_t ldy, void* ws, size_t ws_bytes,
                        void* stream) {
    if (!h || m < 0 || n < 0 || w < 0 || lda < n || ldx < w || ldy < w) return TSVD_ERR_INVALID_ARG;
    // empty operands may come with null pointers
    if ((m * n > 0 && !A) || ((trans ? m : n) * w > 0 && !X) || ((trans ? n : m) * w > 0 && !Y))
        return TSVD_ERR_INVALID_ARG;
    size_t need = 0;
    TSVD_TRY(tsvd_dense_mm_f64tc_workspace(trans, m, n, w, &need));
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    DeviceGuard dg(h->device);
    if (!dg.ok()) return TSVD_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t rows = trans ? n : m;
    if (rows == 0 || w == 0) return TSVD_OK;
    if ((trans ? m : n) == 0) {
        for (int64_t i = 0; i < rows; ++i) TSVD_TRY_CUDA(cudaMemsetAsync(Y + i * ldy, 0, sizeof(double) * w, st));
        TSVD_TRY_CUDA(cudaStreamSynchronize(st));
        return TSVD_OK;
    }
    int* status = static_cast<int*>(ws);
    char* scratch = static_cast<char*>(ws) + 256;
    TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    if (trans)
        TSVD_TRY(oz_gemm_tn(h, m, n, w, A, lda, X, ldx, Y, ldy, false, scratch, need - 256, status, st));
    else
        TSVD_TRY(oz_gemm_nn(h, m, n, w, 1.0, A, lda, X, ldx, 0.0, Y, ldy, false, scratch, need - 256, status, st));
    int hs[kStCount];
    TSVD_TRY(read_status(st, status, hs));
    if (hs[kStTimeout]) return TSVD_ERR_TIMEOUT;
    return TSVD_OK;
}

int tsvd_dense_mm_f32(tsvd_handle* h, int trans, int64_t m, int64_t n, const float* A, int64_t lda, int w,
                      const float* X, int64_t ldx, float* Y, int64_t ldy, void* ws, size_t ws_bytes, void* stream) {
    if (!h || m < 0 || n < 0 || w < 0 || lda < n || !A || !X || !Y) return TSVD_ERR_INVALID_ARG;
    if (ldx < w || ldy < w) return TSVD_ERR_INVALID_ARG;
    size_t need = trans ? gemm_tn_ws(h, m, n, w, false, 4) : 0;
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (trans)
        TSVD_TRY_CUDA((gemm_tn<float, float>(h, m, n, w, A, lda, X, ldx, Y, ldy, false, static_cast<double*>(ws), st)));
    else
        TSVD_TRY_CUDA((gemm_nn<float, float, float>(h, m, n, w, 1.0, A, lda, X, ldx, 0.0, Y, ldy, false, st)));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}

int tsvd_bf16x3_bytes(int64_t rows, int64_t cols, size_t* bytes) {
    if (!bytes || rows < 0 || cols < 0) return TSVD_ERR_INVALID_ARG;
    *bytes = bf16x3_bytes(rows, cols);
    return TSVD_OK;
}

int tsvd_bf16x3_split(tsvd_handle* h, int trans, int64_t m, int64_t n, const double* A, int64_t lda, void* pieces,
                      void* stream) {
    if (!h || m < 0 || n < 0 || lda < n || (m * n > 0 && (!A || !pieces))) return TSVD_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TSVD_TRY_CUDA(bf16x3_split<double>(h, m, n, A, lda, trans != 0, pieces, st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}

int tsvd_mm_bf16x6_workspace(int64_t rows, int64_t cols, int w, size_t* bytes) {
    if (!bytes || rows < 0 || cols < 0 || w < 0) return TSVD_ERR_INVALID_ARG;
    *bytes = align256(sizeof(int) * kStCount) + tc_mm_ws(rows, cols, w);
    return TSVD_OK;
}

int tsvd_mm_bf16x6(tsvd_handle* h, int64_t rows, int64_t cols, const void* pieces, int w, const float* X,
                   int64_t ldx, float* Y, int64_t ldy, void* ws, size_t ws_bytes, void* stream) {
    if (!h || rows < 0 || cols < 0 || w < 0 || ldx < w || ldy < w) return TSVD_ERR_INVALID_ARG;
    if (rows * (int64_t)w > 0 && (!Y || (cols > 0 && (!pieces || !X)))) return TSVD_ERR_INVALID_ARG;
    size_t need = 0;
    TSVD_TRY(tsvd_mm_bf16x6_workspace(rows, cols, w, &need));
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* status = static_cast<int*>(ws);
    TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    void* rest = static_cast<uint8_t*>(ws) + align256(sizeof(int) * kStCount);
    TSVD_TRY_CUDA(tc_mm(h, rows, cols, pieces, w, X, ldx, Y, ldy, rest, status, st));
    int hs[kStCount];
    TSVD_TRY(read_status(st, status, hs));
    return hs[kStTimeout] ? TSVD_ERR_TIMEOUT : TSVD_OK;
}

int tsvd_orth_workspace(int64_t q, int64_t s, int b, size_t* bytes) {
    if (!bytes || q < 0 || s < 0 || b < 1) return TSVD_ERR_INVALID_ARG;
    tsvd_handle hh{};
    hh.sm_count = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&hh.sm_count, cudaDevAttrMultiProcessorCount, dev);
    *bytes = align256(sizeof(int) * kStCount) + orth_ws(&hh, q, s, b) + align256(sizeof(double) * (size_t)(s + b) * b);
    return TSVD_OK;
}

extern "C++" {
template <typename T>
int orth_entry(tsvd_handle* h, int64_t q, int64_t s, int b, const T* P, int64_t ldp, T* Y,
                      int64_t ldy, double* H, double* R, uint64_t seed, int* replacements, int* breakdowns, void* ws,
                      size_t ws_bytes, void* stream) {
    if (!h || b < 1 || q < b || s < 0 || !Y || !R || ldy < b) return TSVD_ERR_INVALID_ARG;
    if (b > TSVD_MAX_BLOCK) return TSVD_ERR_UNSUPPORTED;
    if (s > 0 && (!P || ldp < s)) return TSVD_ERR_INVALID_ARG;
    if (s + b > q) return TSVD_ERR_INVALID_ARG;
    size_t need = 0;
    TSVD_TRY(tsvd_orth_workspace(q, s, b, &need));
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Arena ar{static_cast<char*>(ws), ws_bytes, 0};
    int* status = ar.take<int>(kStCount);
    TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    OrthCtx ctx;
    ctx.seed = seed;
    ctx.replacements = replacements ? *replacements : 0;
    TSVD_TRY_CUDA(cudaMemsetAsync(R, 0, sizeof(double) * (size_t)b * b, st));
    int rc = cgs_cqr2<T>(h, q, s, b, P, ldp, Y, ldy, H, R, b, false, ctx, ar, status, st);
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    if (replacements) *replacements = ctx.replacements;
    if (breakdowns) *breakdowns += ctx.fallbacks;
    return rc;
}
}  // extern "C++"

int tsvd_cholqr2(tsvd_handle* h, int64_t q, int b, double* Y, int64_t ldy, double* R, uint64_t seed,
                 int* replacements, int* breakdowns, void* ws, size_t ws_bytes, void* stream) {
    return orth_entry(h, q, 0, b, (const double*)nullptr, 0, Y, ldy, nullptr, R, seed, replacements, breakdowns, ws,
                      ws_bytes, stream);
}

int tsvd_cgs_cqr2(tsvd_handle* h, int64_t q, int64_t s, int b, const double* P, int64_t ldp, double* Y, int64_t ldy,
                  double* H, double* R, uint64_t seed, int* replacements, int* breakdowns, void* ws,
                  size_t ws_bytes, void* stream) {
    return orth_entry(h, q, s, b, P, ldp, Y, ldy, H, R, seed, replacements, breakdowns, ws, ws_bytes, stream);
}

int tsvd_cgs_cqr2_f32(tsvd_handle* h, int64_t q, int64_t s, int b, const float* P, int64_t ldp, float* Y,
                      int64_t ldy, double* H, double* R, uint64_t seed, int* replacements, int* breakdowns, void* ws,
                      size_t ws_bytes, void* stream) {
    return orth_entry(h, q, s, b, P, ldp, Y, ldy, H, R, seed, replacements, breakdowns, ws, ws_bytes, stream);
}

int tsvd_update_gram_f32_workspace(int64_t q, int b, size_t* bytes) {
    if (!bytes || q < 0 || b < 1) return TSVD_ERR_INVALID_ARG;
    if (b > 128) return TSVD_ERR_UNSUPPORTED;
    *bytes = update_gram_ws(q, b);
    return TSVD_OK;
}

int tsvd_update_gram_f32(tsvd_handle* h, int64_t q, int64_t s, int b, double alpha, const float* X, int64_t ldx,
                         const double* M, int64_t ldm, double beta, float* Y, int64_t ldy, int upper, double* W,
                         void* ws, size_t ws_bytes, void* stream) {
    if (!h || q < 0 || s < 1 || b < 1 || !X || !M || !Y || !W || ldx < s || ldm < b || ldy < b)
        return TSVD_ERR_INVALID_ARG;
    if (b > 128) return TSVD_ERR_UNSUPPORTED;
    if ((const void*)X == (const void*)Y && (s != b || ldx != ldy)) return TSVD_ERR_INVALID_ARG;
    size_t need = 0;
    TSVD_TRY(tsvd_update_gram_f32_workspace(q, b, &need));
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TSVD_TRY_CUDA(update_gram(h, q, s, b, alpha, X, ldx, M, ldm, beta, Y, ldy, upper != 0, W,
                              static_cast<double*>(ws), st));
    return TSVD_OK;
}

int tsvd_cgs_qr(tsvd_handle* h, int64_t q, int r, int b, double* Y, int64_t ldy, double* R, uint64_t seed,
                int* replacements, int* breakdowns, void* ws, size_t ws_bytes, void* stream) {
    if (!h || r < 1 || b < 1 || q < r || !Y || !R || ldy < r) return TSVD_ERR_INVALID_ARG;
    if (b > TSVD_MAX_BLOCK) return TSVD_ERR_UNSUPPORTED;
    const int bw = b < r ? b : r;
    size_t need = 0;
    TSVD_TRY(tsvd_orth_workspace(q, r - bw, bw, &need));
    need += align256(sizeof(double) * (size_t)r * bw);
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Arena ar{static_cast<char*>(ws), ws_bytes, 0};
    int* status = ar.take<int>(kStCount);
    TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    OrthCtx ctx;
    ctx.seed = seed;
    ctx.replacements = replacements ? *replacements : 0;
    int rc = cgs_qr<double>(h, q, r, bw, Y, ldy, R, ctx, ar, status, st);
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    if (replacements) *replacements = ctx.replacements;
    if (breakdowns) *breakdowns += ctx.fallbacks;
    return rc;
}

int tsvd_small_svd_workspace(int n, size_t* bytes) {
    if (!bytes || n < 1) return TSVD_ERR_INVALID_ARG;
    if (n > TSVD_MAX_SMALL_SVD) return TSVD_ERR_UNSUPPORTED;
    *bytes = align256(sizeof(int) * kStCount) + small_svd_ws(n);
    return TSVD_OK;
}

int tsvd_small_svd(tsvd_handle* h, int n, const double* B, int64_t ldb, int nv, double* Ubar, double* sigma,
                   double* Vbar, int* sweeps, void* ws, size_t ws_bytes, void* stream) {
    if (!h || n < 1 || !B || ldb < n || !Ubar || !sigma || !Vbar || nv < 0 || nv > n) return TSVD_ERR_INVALID_ARG;
    if (n > TSVD_MAX_SMALL_SVD) return TSVD_ERR_UNSUPPORTED;
    size_t need = 0;
    TSVD_TRY(tsvd_small_svd_workspace(n, &need));
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Arena ar{static_cast<char*>(ws), ws_bytes, 0};
    int* status = ar.take<int>(kStCount);
    TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    TSVD_TRY(small_svd(h, n, B, ldb, Ubar, sigma, Vbar, nv, ar, status, st));
    int hs[kStCount];
    TSVD_TRY(read_status(st, status, hs));
    if (sweeps) *sweeps = hs[kStSweeps];
    if (hs[kStTimeout]) return TSVD_ERR_TIMEOUT;
    if (hs[kStNonfinite]) return TSVD_ERR_NONFINITE;
    return TSVD_OK;
}

}  // extern "C"
