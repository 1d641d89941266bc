// C ABI (include/tsvd.h): handle, workspace sizing, the RandSVD and LancSVD
// drivers (Alg. 1, Alg. 2) and the building-block entry points.
//
// The drivers keep every step on the device; the host only sequences kernels
// and reads back a few status words (Cholesky breakdown flags, the Lanczos
// residual estimate, the explicit residual).  A is never modified.  When
// m < n both methods run on A^T and swap U and V on return (Sec. 2).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "tsvd_internal.cuh"

namespace tsvd {
int jacobi_coop_capacity(int device, int sm_count);
}

using namespace tsvd;

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

// op(A) as seen by the methods: m >= n after the optional transpose.
struct Op {
    bool sparse = false, transposed = false;
    int64_t m = 0, n = 0;            // dimensions of op(A)
    int64_t M = 0, N = 0;            // dimensions of A
    const int32_t *rp = nullptr, *ci = nullptr;  // CSR(A)
    const double* va = nullptr;
    int32_t *trp = nullptr, *tci = nullptr;      // CSR(A^T)
    double* tva = nullptr;
    int64_t nnz = 0;
    const double* dA = nullptr;      // dense A
    int64_t lda = 0;
    double* partial = nullptr;       // dense A^T X split-K scratch
};

// Y (op.m x w) = op(A) X (op.n x w)
int op_mul(tsvd_handle* h, Op& op, int w, const double* X, int64_t ldx, double* Y, int64_t ldy, int* status,
           cudaStream_t st) {
    if (op.sparse) {
        if (!op.transposed)
            TSVD_TRY_CUDA(launch_spmm(h, op.M, op.N, op.nnz, op.rp, op.ci, op.va, w, X, ldx, Y, ldy, status, st));
        else
            TSVD_TRY_CUDA(launch_spmm(h, op.N, op.M, op.nnz, op.trp, op.tci, op.tva, w, X, ldx, Y, ldy, status, st));
    } else {
        if (!op.transposed)
            TSVD_TRY_CUDA(gemm_nn(h, op.M, op.N, w, 1.0, op.dA, op.lda, X, ldx, 0.0, Y, ldy, false, st));
        else
            TSVD_TRY_CUDA(gemm_tn(h, op.M, op.N, w, op.dA, op.lda, X, ldx, Y, ldy, false, op.partial, st));
    }
    return TSVD_OK;
}

// Y (op.n x w) = op(A)^T X (op.m x w)
int op_tmul(tsvd_handle* h, Op& op, int w, const double* X, int64_t ldx, double* Y, int64_t ldy, int* status,
            cudaStream_t st) {
    if (op.sparse) {
        if (!op.transposed)
            TSVD_TRY_CUDA(launch_spmm(h, op.N, op.M, op.nnz, op.trp, op.tci, op.tva, w, X, ldx, Y, ldy, status, st));
        else
            TSVD_TRY_CUDA(launch_spmm(h, op.M, op.N, op.nnz, op.rp, op.ci, op.va, w, X, ldx, Y, ldy, status, st));
    } else {
        if (!op.transposed)
            TSVD_TRY_CUDA(gemm_tn(h, op.M, op.N, w, op.dA, op.lda, X, ldx, Y, ldy, false, op.partial, st));
        else
            TSVD_TRY_CUDA(gemm_nn(h, op.M, op.N, w, 1.0, op.dA, op.lda, X, ldx, 0.0, Y, ldy, false, st));
    }
    return TSVD_OK;
}

int validate_matrix(const tsvd_matrix* A) {
    if (A == nullptr) return TSVD_ERR_INVALID_ARG;
    if (A->m < 1 || A->n < 1) return TSVD_ERR_INVALID_ARG;
    if (A->dtype != TSVD_F64) return TSVD_ERR_UNSUPPORTED;
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

// Carves the operator's storage: staged host input, CSR(A^T), dense split-K scratch.
int setup_op(tsvd_handle* h, const tsvd_matrix* A, int wmax, Arena& ar, Op& op, int* status, cudaStream_t st,
             bool do_work, float* ms_transpose) {
    op.M = A->m;
    op.N = A->n;
    op.transposed = A->m < A->n;
    op.m = op.transposed ? A->n : A->m;
    op.n = op.transposed ? A->m : A->n;
    op.sparse = A->format == TSVD_CSR;
    if (op.sparse) {
        op.nnz = A->nnz;
        if (A->location == TSVD_HOST) {
            int32_t* rp = ar.take<int32_t>(A->m + 1);
            int32_t* ci = ar.take<int32_t>(A->nnz);
            double* va = ar.take<double>(A->nnz);
            if (do_work) {
                if (!ar.fits()) return TSVD_ERR_WORKSPACE;
                TSVD_TRY_CUDA(cudaMemcpyAsync(rp, A->row_ptr, sizeof(int32_t) * (A->m + 1), cudaMemcpyHostToDevice, st));
                TSVD_TRY_CUDA(cudaMemcpyAsync(ci, A->col_idx, sizeof(int32_t) * A->nnz, cudaMemcpyHostToDevice, st));
                TSVD_TRY_CUDA(cudaMemcpyAsync(va, A->val, sizeof(double) * A->nnz, cudaMemcpyHostToDevice, st));
            }
            op.rp = rp;
            op.ci = ci;
            op.va = va;
        } else {
            op.rp = A->row_ptr;
            op.ci = A->col_idx;
            op.va = static_cast<const double*>(A->val);
        }
        op.trp = ar.take<int32_t>(A->n + 1);
        op.tci = ar.take<int32_t>(A->nnz);
        op.tva = ar.take<double>(A->nnz);
        if (do_work) {
            Arena tmp = ar;
            tmp.take<char>(0);
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (ms_transpose) {
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                cudaEventRecord(e0, st);
            }
            int rc = csr_transpose(h, A->m, A->n, A->nnz, op.rp, op.ci, op.va, op.trp, op.tci, op.tva, tmp, status, st);
            if (ms_transpose) {
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(ms_transpose, e0, e1);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
            }
            if (rc < 0) return rc;
        } else {
            ar.take<char>(csr_transpose_ws(A->m, A->n, A->nnz));
            return TSVD_OK;
        }
        // the transpose scratch is dead after the build: later carving may reuse it
    } else {
        if (A->location == TSVD_HOST) {
            double* d = ar.take<double>((size_t)A->m * A->n);
            if (do_work) {
                if (!ar.fits()) return TSVD_ERR_WORKSPACE;
                TSVD_TRY_CUDA(cudaMemcpy2DAsync(d, sizeof(double) * A->n, A->val, sizeof(double) * A->ld,
                                                sizeof(double) * A->n, A->m, cudaMemcpyHostToDevice, st));
            }
            op.dA = d;
            op.lda = A->n;
        } else {
            op.dA = static_cast<const double*>(A->val);
            op.lda = A->ld;
        }
        size_t pb = 0;
        for (int w = 1; w <= wmax; ++w) {
            const size_t v = gemm_tn_ws(h, A->m, A->n, w, false);
            if (v > pb) pb = v;
        }
        op.partial = ar.take<double>(pb / sizeof(double) + 1);
    }
    return TSVD_OK;
}

struct Timer {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st;
    explicit Timer(cudaStream_t s) : st(s) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    double stop() {
        float ms = 0.f;
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    }
    ~Timer() {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
};

struct Outputs {
    double *sigma, *U, *V;  // device buffers the drivers write (op orientation)
};

// Explicit residual max_j ||op(A) v_j - s_j u_j|| / s_1 on the returned triplets.
int explicit_residual(tsvd_handle* h, Op& op, int k, const double* U, const double* V, const double* sigma,
                      double* Ytmp, double* res, double* partial, int* status, cudaStream_t st, double* out) {
    TSVD_TRY(op_mul(h, op, k, V, k, Ytmp, k, status, st));
    TSVD_TRY_CUDA(col_residual_sq(h, op.m, k, Ytmp, k, U, k, sigma, res, partial, st));
    std::vector<double> hres(k), hs(1);
    TSVD_TRY_CUDA(cudaMemcpyAsync(hres.data(), res, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    TSVD_TRY_CUDA(cudaMemcpyAsync(hs.data(), sigma, sizeof(double), cudaMemcpyDeviceToHost, st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    double mx = 0.0;
    for (int j = 0; j < k; ++j) mx = std::fmax(mx, std::sqrt(hres[j]));
    *out = hs[0] > 0.0 ? mx / hs[0] : NAN;
    return TSVD_OK;
}

int finish_outputs(tsvd_handle* h, const tsvd_opts* o, Op& op, int k, const Outputs& dev, double* sigma, double* U,
                   double* V, void* signws, cudaStream_t st) {
    // U is op.m x k, V is op.n x k in op orientation
    TSVD_TRY_CUDA(sign_fix(h, op.n, op.m, k, dev.V, k, dev.U, k, signws, st));
    double* userU = op.transposed ? V : U;  // op's U has op.m = A->n rows when transposed
    double* userV = op.transposed ? U : V;
    const cudaMemcpyKind kind = (o->output_location == TSVD_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (o->output_location == TSVD_HOST || dev.sigma != sigma) {
        TSVD_TRY_CUDA(cudaMemcpyAsync(sigma, dev.sigma, sizeof(double) * k, kind, st));
        TSVD_TRY_CUDA(cudaMemcpyAsync(userU, dev.U, sizeof(double) * op.m * k, kind, st));
        TSVD_TRY_CUDA(cudaMemcpyAsync(userV, dev.V, sizeof(double) * op.n * k, kind, st));
    }
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}

// ---------------------------------------------------------------------------
// Workspace plans (same carving code for sizing and for the run).
// ---------------------------------------------------------------------------
struct RsvdBufs {
    int* status;
    double *Qn, *Qm, *R, *Ub, *Vb, *sig, *Ytmp, *res, *cpart;
    double *oU, *oV, *osig;
    void* signws;
};

struct LancBufs {
    int* status;
    double *P, *Pbar, *Qnext, *B, *Ub, *Vb, *sig, *Rr, *rho, *Ytmp, *res, *cpart;
    double *oU, *oV, *osig;
    void* signws;
};

void carve_outputs(Arena& ar, const tsvd_opts* o, int64_t m, int64_t n, int k, double*& oU, double*& oV,
                   double*& osig) {
    if (o->output_location == TSVD_HOST) {
        oU = ar.take<double>((size_t)m * k);
        oV = ar.take<double>((size_t)n * k);
        osig = ar.take<double>(k);
    } else {
        oU = oV = osig = nullptr;
    }
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

// ---------------------------------------------------------------------------
static int plan_rsvd(tsvd_handle* h, const tsvd_matrix* A, int k, int p, int q, const tsvd_opts* o, Arena& ar,
                     Op& op, RsvdBufs& b, bool run, cudaStream_t st, float* ms_t) {
    b.status = ar.take<int>(kStCount);
    if (run) {
        if (!ar.fits()) return TSVD_ERR_WORKSPACE;
        TSVD_TRY_CUDA(cudaMemsetAsync(b.status, 0, sizeof(int) * kStCount, st));
    }
    const int ell = k + p;
    TSVD_TRY(setup_op(h, A, ell, ar, op, b.status, st, run, ms_t));
    const int64_t m = op.m, n = op.n;
    b.Qn = ar.take<double>((size_t)n * ell);
    b.Qm = ar.take<double>((size_t)m * ell);
    b.R = ar.take<double>((size_t)ell * ell);
    b.Ub = ar.take<double>((size_t)ell * ell);
    b.Vb = ar.take<double>((size_t)ell * ell);
    b.sig = ar.take<double>(ell);
    b.Ytmp = ar.take<double>((size_t)m * k);
    b.res = ar.take<double>(k);
    b.cpart = ar.take<double>(colres_ws(m, k) / sizeof(double) + 1);
    b.signws = ar.take<char>(sign_fix_ws(m > n ? m : n, k));
    carve_outputs(ar, o, m, n, k, b.oU, b.oV, b.osig);
    (void)q;
    return TSVD_OK;
}

static size_t rsvd_tail_ws(tsvd_handle* h, int64_t m, int64_t n, int ell, int bq) {
    const int64_t qmax = m > n ? m : n;
    size_t a = orth_ws(h, qmax, ell > bq ? ell - bq : 0, bq) + align256(sizeof(double) * (size_t)ell * bq);
    size_t s = small_svd_ws(ell);
    return a > s ? a : s;
}

static size_t lanc_tail_ws(tsvd_handle* h, int64_t m, int64_t n, int b, int r) {
    const int rb = r * b;
    size_t a = orth_ws(h, m, rb, b);
    size_t a2 = orth_ws(h, n, rb, b);
    if (a2 > a) a = a2;
    size_t s = small_svd_ws(rb);
    return a > s ? a : s;
}

static int check_rsvd_args(const tsvd_matrix* A, int k, int p, int q, const tsvd_opts* o) {
    TSVD_TRY(validate_matrix(A));
    const int64_t mn = A->m < A->n ? A->m : A->n;
    if (k < 1 || p < 0 || q < 0 || (int64_t)k + p > mn) return TSVD_ERR_INVALID_ARG;
    if (k + p > TSVD_MAX_SMALL_SVD) return TSVD_ERR_UNSUPPORTED;
    if (o && o->qr_block < 0) return TSVD_ERR_INVALID_ARG;
    return TSVD_OK;
}

static int check_lanc_args(const tsvd_matrix* A, int k, int b, int r, const tsvd_opts* o) {
    TSVD_TRY(validate_matrix(A));
    const int64_t mn = A->m < A->n ? A->m : A->n;
    if (b < 1 || r < 1 || k < 1) return TSVD_ERR_INVALID_ARG;
    if (b > TSVD_MAX_BLOCK) return TSVD_ERR_UNSUPPORTED;
    if ((int64_t)r * b > mn || k > r * b) return TSVD_ERR_INVALID_ARG;
    if (r * b > TSVD_MAX_SMALL_SVD) return TSVD_ERR_UNSUPPORTED;
    if (o && (o->max_restarts < 0 || !(o->tol >= 0.0))) return TSVD_ERR_INVALID_ARG;
    return TSVD_OK;
}

static int qr_block_of(const tsvd_opts* o, int ell) {
    int bq = (o && o->qr_block > 0) ? o->qr_block : ell;
    if (bq > ell) bq = ell;
    if (bq > TSVD_MAX_BLOCK) bq = TSVD_MAX_BLOCK;
    return bq;
}

static int plan_lanc(tsvd_handle* h, const tsvd_matrix* A, int k, int b, int r, const tsvd_opts* o, Arena& ar, Op& op,
                     LancBufs& L, bool run, cudaStream_t st, float* ms_t) {
    L.status = ar.take<int>(kStCount);
    if (run) {
        if (!ar.fits()) return TSVD_ERR_WORKSPACE;
        TSVD_TRY_CUDA(cudaMemsetAsync(L.status, 0, sizeof(int) * kStCount, st));
    }
    TSVD_TRY(setup_op(h, A, b > k ? b : k, ar, op, L.status, st, run, ms_t));
    const int64_t m = op.m, n = op.n;
    const int rb = r * b;
    L.P = ar.take<double>((size_t)n * rb);
    L.Pbar = ar.take<double>((size_t)m * rb);
    L.Qnext = ar.take<double>((size_t)m * b);
    L.B = ar.take<double>((size_t)rb * rb);
    L.Ub = ar.take<double>((size_t)rb * rb);
    L.Vb = ar.take<double>((size_t)rb * rb);
    L.sig = ar.take<double>(rb);
    L.Rr = ar.take<double>((size_t)b * b);
    L.rho = ar.take<double>(k);
    L.Ytmp = ar.take<double>((size_t)m * k);
    L.res = ar.take<double>(k);
    L.cpart = ar.take<double>(colres_ws(m, k) / sizeof(double) + 1);
    L.signws = ar.take<char>(sign_fix_ws(m > n ? m : n, k));
    carve_outputs(ar, o, m, n, k, L.oU, L.oV, L.osig);
    return TSVD_OK;
}

int tsvd_workspace_size(const tsvd_matrix* A, int method, int k, int a, int c, const tsvd_opts* opts, size_t* bytes) {
    if (!bytes) return TSVD_ERR_INVALID_ARG;
    tsvd_opts o;
    tsvd_default_opts(&o);
    if (opts) o = *opts;
    tsvd_handle hh{};
    hh.sm_count = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        int sm = 0;
        if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sm > 0) hh.sm_count = sm;
    }
    Arena ar;
    Op op;
    if (method == TSVD_METHOD_RSVD) {
        TSVD_TRY(check_rsvd_args(A, k, a, c, &o));
        RsvdBufs b{};
        TSVD_TRY(plan_rsvd(&hh, A, k, a, c, &o, ar, op, b, false, nullptr, nullptr));
        const int ell = k + a;
        ar.take<char>(rsvd_tail_ws(&hh, op.m, op.n, ell, qr_block_of(&o, ell)));
    } else if (method == TSVD_METHOD_BLANCZOS) {
        TSVD_TRY(check_lanc_args(A, k, a, c, &o));
        LancBufs L{};
        TSVD_TRY(plan_lanc(&hh, A, k, a, c, &o, ar, op, L, false, nullptr, nullptr));
        ar.take<char>(lanc_tail_ws(&hh, op.m, op.n, a, c));
    } else {
        return TSVD_ERR_INVALID_ARG;
    }
    *bytes = ar.off + 256;
    return TSVD_OK;
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
    TSVD_TRY_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = static_cast<cudaStream_t>(o.stream);
    const int64_t l0 = h->launches;
    ProfileGuard pg(h, (o.flags & TSVD_FLAG_PROFILE) != 0);
    Timer total(st);
    Arena ar{static_cast<char*>(ws), ws_bytes, 0};
    Op op;
    RsvdBufs b{};
    float ms_t = 0.f;
    TSVD_TRY(plan_rsvd(h, A, k, p, q, &o, ar, op, b, true, st, op.sparse || A->format == TSVD_CSR ? &ms_t : nullptr));
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    const int ell = k + p;
    const int bq = qr_block_of(&o, ell);
    const int64_t m = op.m, n = op.n;
    OrthCtx ctx;
    ctx.seed = seed;
    // Q_0 (n x l): raw Gaussian block (Alg. 1)
    if (o.start_block)
        TSVD_TRY_CUDA(copy_block(o.start_block, ell, b.Qn, ell, n, ell, st));
    else
        TSVD_TRY_CUDA(gaussian(h, n, ell, seed, 1u, b.Qn, ell, st));
    int iters = 0;
    for (int it = 0; it <= q; ++it) {
        TSVD_TRY(op_mul(h, op, ell, b.Qn, ell, b.Qm, ell, b.status, st));                      // S1
        TSVD_TRY(cgs_qr(h, m, ell, bq, b.Qm, ell, b.R, ctx, ar, b.status, st));                 // S2
        TSVD_TRY(op_tmul(h, op, ell, b.Qm, ell, b.Qn, ell, b.status, st));                     // S3
        TSVD_TRY(cgs_qr(h, n, ell, bq, b.Qn, ell, b.R, ctx, ar, b.status, st));                 // S4
        ++iters;
    }
    int hs[kStCount];
    {
        Arena sv = ar;
        TSVD_TRY(small_svd(h, ell, b.R, ell, b.Ub, b.sig, b.Vb, sv, b.status, st));             // S5
    }
    Outputs dev{b.osig ? b.osig : sigma, b.oU ? b.oU : (op.transposed ? V : U), b.oV ? b.oV : (op.transposed ? U : V)};
    TSVD_TRY_CUDA(gemm_nn(h, m, ell, k, 1.0, b.Qm, ell, b.Vb, ell, 0.0, dev.U, k, false, st));  // S6
    TSVD_TRY_CUDA(gemm_nn(h, n, ell, k, 1.0, b.Qn, ell, b.Ub, ell, 0.0, dev.V, k, false, st));  // S7
    TSVD_TRY_CUDA(cudaMemcpyAsync(dev.sigma, b.sig, sizeof(double) * k, cudaMemcpyDeviceToDevice, st));
    TSVD_TRY(read_status(st, b.status, hs));
    if (hs[kStTimeout]) return TSVD_ERR_TIMEOUT;
    if (hs[kStNonfinite]) return TSVD_ERR_NONFINITE;
    if (hs[kStBadCsr]) return TSVD_ERR_INVALID_ARG;
    const int sweeps = hs[kStSweeps];
    TSVD_TRY(finish_outputs(h, &o, op, k, dev, sigma, U, V, b.signws, st));
    const double ms_total = total.stop();
    double resid = NAN;
    TSVD_TRY(explicit_residual(h, op, k, dev.U, dev.V, dev.sigma, b.Ytmp, b.res, b.cpart, b.status, st, &resid));
    if (o.output_location == TSVD_HOST) {
        TSVD_TRY_CUDA(cudaMemcpyAsync(sigma, dev.sigma, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->iterations = iters;
        info->breakdowns = ctx.fallbacks;
        info->converged = 1;
        info->transposed = op.transposed ? 1 : 0;
        info->svd_sweeps = sweeps;
        info->resid_max = resid;
        info->rho_last = NAN;
        info->ms_total = ms_total;
        info->ms_transpose = ms_t;
        info->kernel_launches = h->launches - l0;
        prof_collect(h, info);
    }
    return TSVD_OK;
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
    TSVD_TRY_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = static_cast<cudaStream_t>(o.stream);
    const int64_t l0 = h->launches;
    ProfileGuard pg(h, (o.flags & TSVD_FLAG_PROFILE) != 0);
    Timer total(st);
    Arena ar{static_cast<char*>(ws), ws_bytes, 0};
    Op op;
    LancBufs L{};
    float ms_t = 0.f;
    TSVD_TRY(plan_lanc(h, A, k, b, r, &o, ar, op, L, true, st, A->format == TSVD_CSR ? &ms_t : nullptr));
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    const int rb = r * b;
    const int64_t m = op.m, n = op.n;
    OrthCtx ctx;
    ctx.seed = seed;
    Outputs dev{L.osig ? L.osig : sigma, L.oU ? L.oU : (op.transposed ? V : U), L.oV ? L.oV : (op.transposed ? U : V)};
    // S1: random orthonormal Qbar_1 (m x b) in the first block column of Pbar
    if (o.start_block)
        TSVD_TRY_CUDA(copy_block(o.start_block, b, L.Pbar, rb, m, b, st));
    else
        TSVD_TRY_CUDA(gaussian(h, m, b, seed, 2u, L.Pbar, rb, st));
    TSVD_TRY(cgs_cqr2(h, m, 0, b, nullptr, 0, L.Pbar, rb, nullptr, L.Rr, b, false, ctx, ar, L.status, st));
    int cycles = 0, restarts = 0, sweeps = 0, converged = 0;
    double rho_last = NAN, resid = NAN;
    std::vector<double> hrho(k), hsig(1);
    int hs[kStCount];
    for (;;) {
        TSVD_TRY_CUDA(cudaMemsetAsync(L.B, 0, sizeof(double) * (size_t)rb * rb, st));
        for (int i = 0; i < r; ++i) {
            const int c0 = i * b;
            double* Qi = L.P + c0;
            TSVD_TRY(op_tmul(h, op, b, L.Pbar + c0, rb, Qi, rb, L.status, st));                   // S2
            double* Lii = L.B + (int64_t)c0 * rb + c0;
            TSVD_TRY(cgs_cqr2(h, n, c0, b, L.P, rb, Qi, rb, nullptr, Lii, rb, true, ctx, ar, L.status, st));  // S3
            const bool last = (i + 1 == r);
            double* dst = last ? L.Qnext : L.Pbar + c0 + b;
            const int64_t ldd = last ? b : rb;
            TSVD_TRY(op_mul(h, op, b, Qi, rb, dst, ldd, L.status, st));                             // S4
            double* Ri = last ? L.Rr : L.B + (int64_t)(c0 + b) * rb + c0;
            TSVD_TRY(cgs_cqr2(h, m, c0 + b, b, L.Pbar, rb, dst, ldd, nullptr, Ri, last ? b : rb, false, ctx, ar,
                              L.status, st));                                                      // S5
        }
        ++cycles;
        {
            Arena sv = ar;
            TSVD_TRY(small_svd(h, rb, L.B, rb, L.Ub, L.sig, L.Vb, sv, L.status, st));               // S6
        }
        TSVD_TRY_CUDA(lanczos_rho(h, b, k, L.Rr, L.Vb + (int64_t)(rb - b) * rb, rb, L.rho, st));
        TSVD_TRY_CUDA(cudaMemcpyAsync(hrho.data(), L.rho, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        TSVD_TRY_CUDA(cudaMemcpyAsync(hsig.data(), L.sig, sizeof(double), cudaMemcpyDeviceToHost, st));
        TSVD_TRY(read_status(st, L.status, hs));
        if (hs[kStTimeout]) return TSVD_ERR_TIMEOUT;
        if (hs[kStNonfinite]) return TSVD_ERR_NONFINITE;
        if (hs[kStBadCsr]) return TSVD_ERR_INVALID_ARG;
        sweeps = hs[kStSweeps];
        double rmax = 0.0;
        for (int j = 0; j < k; ++j) rmax = std::fmax(rmax, hrho[j]);
        rho_last = hsig[0] > 0.0 ? rmax / hsig[0] : NAN;
        const bool done = rho_last <= o.tol;
        if (done || restarts >= o.max_restarts) {
            TSVD_TRY_CUDA(gemm_nn(h, m, rb, k, 1.0, L.Pbar, rb, L.Ub, rb, 0.0, dev.U, k, false, st));  // S9
            TSVD_TRY_CUDA(gemm_nn(h, n, rb, k, 1.0, L.P, rb, L.Vb, rb, 0.0, dev.V, k, false, st));     // S8
            TSVD_TRY_CUDA(cudaMemcpyAsync(dev.sigma, L.sig, sizeof(double) * k, cudaMemcpyDeviceToDevice, st));
            TSVD_TRY(explicit_residual(h, op, k, dev.U, dev.V, dev.sigma, L.Ytmp, L.res, L.cpart, L.status, st,
                                       &resid));
            if ((done && resid <= o.tol) || restarts >= o.max_restarts) {
                converged = resid <= o.tol ? 1 : 0;
                break;
            }
        }
        ++restarts;
        // S7: Qbar_1 = Pbar Ubar_1, re-orthonormalised by CholeskyQR2
        TSVD_TRY_CUDA(gemm_nn(h, m, rb, b, 1.0, L.Pbar, rb, L.Ub, rb, 0.0, L.Qnext, b, false, st));
        TSVD_TRY_CUDA(copy_block(L.Qnext, b, L.Pbar, rb, m, b, st));
        TSVD_TRY(cgs_cqr2(h, m, 0, b, nullptr, 0, L.Pbar, rb, nullptr, L.Rr, b, false, ctx, ar, L.status, st));
    }
    TSVD_TRY(finish_outputs(h, &o, op, k, dev, sigma, U, V, L.signws, st));
    const double ms_total = total.stop();
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->iterations = cycles;
        info->restarts = restarts;
        info->breakdowns = ctx.fallbacks;
        info->converged = converged;
        info->transposed = op.transposed ? 1 : 0;
        info->svd_sweeps = sweeps;
        info->resid_max = resid;
        info->rho_last = rho_last;
        info->ms_total = ms_total;
        info->ms_transpose = ms_t;
        info->kernel_launches = h->launches - l0;
        prof_collect(h, info);
    }
    return converged ? TSVD_OK : TSVD_NOT_CONVERGED;
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
    TSVD_TRY(csr_transpose(h, m, n, nnz, row_ptr, col_idx, val, t_row_ptr, t_col_idx, t_val, ar, status, st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}

int tsvd_spmm(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
              const double* val, int w, const double* X, int64_t ldx, double* Y, int64_t ldy, void* ws,
              size_t ws_bytes, void* stream) {
    if (!h || m < 0 || n < 0 || nnz < 0 || w < 0 || ldx < w || ldy < w || !row_ptr) return TSVD_ERR_INVALID_ARG;
    if (m * (int64_t)w > 0 && (!X || !Y)) return TSVD_ERR_INVALID_ARG;
    TSVD_TRY(check_ws(ws, ws_bytes, TSVD_SPMM_WORKSPACE));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* status = static_cast<int*>(ws);
    TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    TSVD_TRY_CUDA(launch_spmm(h, m, n, nnz, row_ptr, col_idx, val, w, X, ldx, Y, ldy, status, st));
    int hs[kStCount];
    TSVD_TRY(read_status(st, status, hs));
    return hs[kStBadCsr] ? TSVD_ERR_INVALID_ARG : TSVD_OK;
}

int tsvd_dense_mm_workspace(int trans, int64_t m, int64_t n, int w, size_t* bytes) {
    if (!bytes || m < 0 || n < 0 || w < 0) return TSVD_ERR_INVALID_ARG;
    tsvd_handle hh{};
    hh.sm_count = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&hh.sm_count, cudaDevAttrMultiProcessorCount, dev);
    *bytes = trans ? gemm_tn_ws(&hh, m, n, w, false) : 0;
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
        TSVD_TRY_CUDA(gemm_tn(h, m, n, w, A, lda, X, ldx, Y, ldy, false, static_cast<double*>(ws), st));
    else
        TSVD_TRY_CUDA(gemm_nn(h, m, n, w, 1.0, A, lda, X, ldx, 0.0, Y, ldy, false, st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
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

static int orth_entry(tsvd_handle* h, int64_t q, int64_t s, int b, const double* P, int64_t ldp, double* Y,
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
    int rc = cgs_cqr2(h, q, s, b, P, ldp, Y, ldy, H, R, b, false, ctx, ar, status, st);
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    if (replacements) *replacements = ctx.replacements;
    if (breakdowns) *breakdowns += ctx.fallbacks;
    return rc;
}

int tsvd_cholqr2(tsvd_handle* h, int64_t q, int b, double* Y, int64_t ldy, double* R, uint64_t seed,
                 int* replacements, int* breakdowns, void* ws, size_t ws_bytes, void* stream) {
    return orth_entry(h, q, 0, b, nullptr, 0, Y, ldy, nullptr, R, seed, replacements, breakdowns, ws, ws_bytes,
                      stream);
}

int tsvd_cgs_cqr2(tsvd_handle* h, int64_t q, int64_t s, int b, const double* P, int64_t ldp, double* Y, int64_t ldy,
                  double* H, double* R, uint64_t seed, int* replacements, int* breakdowns, void* ws,
                  size_t ws_bytes, void* stream) {
    return orth_entry(h, q, s, b, P, ldp, Y, ldy, H, R, seed, replacements, breakdowns, ws, ws_bytes, stream);
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
    int rc = cgs_qr(h, q, r, bw, Y, ldy, R, ctx, ar, status, st);
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

int tsvd_small_svd(tsvd_handle* h, int n, const double* B, int64_t ldb, double* Ubar, double* sigma, double* Vbar,
                   int* sweeps, void* ws, size_t ws_bytes, void* stream) {
    if (!h || n < 1 || !B || ldb < n || !Ubar || !sigma || !Vbar) return TSVD_ERR_INVALID_ARG;
    if (n > TSVD_MAX_SMALL_SVD) return TSVD_ERR_UNSUPPORTED;
    size_t need = 0;
    TSVD_TRY(tsvd_small_svd_workspace(n, &need));
    TSVD_TRY(check_ws(ws, ws_bytes, need));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Arena ar{static_cast<char*>(ws), ws_bytes, 0};
    int* status = ar.take<int>(kStCount);
    TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    TSVD_TRY(small_svd(h, n, B, ldb, Ubar, sigma, Vbar, ar, status, st));
    int hs[kStCount];
    TSVD_TRY(read_status(st, status, hs));
    if (sweeps) *sweeps = hs[kStSweeps];
    if (hs[kStTimeout]) return TSVD_ERR_TIMEOUT;
    if (hs[kStNonfinite]) return TSVD_ERR_NONFINITE;
    return TSVD_OK;
}

}  // extern "C"
