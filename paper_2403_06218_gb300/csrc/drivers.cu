// RandSVD (Alg. 1) and LancSVD (Alg. 2) on the device, for both precisions:
//   T = double: the FP64 method of the paper;
//   T = float : the mixed-precision form.  A and every tall block (Q, Qbar, the
//               Lanczos bases) are FP32 and the products accumulate in FP32
//               (dense A: split-BF16 tensor-core products of FP32 accuracy),
//               while every Gram matrix, Cholesky factor, R, B and the small SVD
//               stay FP64.  The returned triplets come from an FP64 Rayleigh-Ritz
//               step: the Ritz vectors are re-orthonormalised in FP64, the k x k
//               projection U^T A V is formed with the FP64 A and its SVD rotates
//               them; the residual test uses the FP64 A.
//
// LancSVD restarts either as the paper does (from the b leading left Ritz
// vectors) or thick: the s leading Ritz pairs are kept, B starts with diag(S_s)
// and the coupling block of the residual block, and the recurrence continues
// from that block (the improved restart the paper leaves to future work, Sec. 5).
// In the mixed form the kept vectors have FP64 master copies and the bases hold
// their FP32 rounding.  The gradient of a loss on the triplets (svd_backward_run)
// also lives here, next to the operator it applies.
//
// The host only sequences kernels and reads back a few status words (Cholesky
// breakdown flags after each orthogonalisation, the Lanczos estimate once per
// cycle, the explicit residual).  When m < n both methods run on A^T and swap U
// and V on return (Sec. 2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

template <typename TI, typename TO>
__global__ void convert2d_kernel(int64_t rows, int64_t cols, const TI* __restrict__ x, int64_t ldx,
                                 TO* __restrict__ y, int64_t ldy) {
    const int64_t tot = rows * cols;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / cols, c = i % cols;
        y[r * ldy + c] = (TO)x[r * ldx + c];
    }
}

template <typename TI, typename TO>
cudaError_t convert2d(tsvd_handle* h, int64_t rows, int64_t cols, const TI* x, int64_t ldx, TO* y, int64_t ldy,
                      cudaStream_t st) {
    const int64_t tot = rows * cols;
    if (tot == 0) return cudaSuccess;
    int64_t blocks = (tot + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    ProfScope prof(h, TSVD_K_OTHER, 0.0, (double)(sizeof(TI) + sizeof(TO)) * tot, st);
    h->launches++;
    convert2d_kernel<TI, TO><<<(unsigned)blocks, 256, 0, st>>>(rows, cols, x, ldx, y, ldy);
    return cudaGetLastError();
}

// op(A) as the methods see it (m >= n after the optional transpose), with the
// values in the working precision T and in FP64 (the same arrays when T = double).
template <typename T>
struct Op {
    bool sparse = false, transposed = false;
    int64_t m = 0, n = 0;  // op(A)
    int64_t M = 0, N = 0;  // A
    int64_t nnz = 0;
    const int32_t *rp = nullptr, *ci = nullptr;  // CSR(A)
    int32_t *trp = nullptr, *tci = nullptr;      // CSR(A^T)
    const T* va = nullptr;
    const T* tva = nullptr;
    const double* va64 = nullptr;
    const double* tva64 = nullptr;
    const T* dA = nullptr;  // dense A (row-major)
    int64_t lda = 0;
    const double* dA64 = nullptr;
    int64_t lda64 = 0;
    double* partial = nullptr;  // split-K scratch of dense A^T X
    // mixed form, dense A: BF16 pieces of A and of A^T for the tensor-core products
    SpmmPlan plan_a, plan_at;  // long-row split plans of CSR(A) and CSR(A^T)
    bool tc = false;
    const void* pA = nullptr;
    const void* pAt = nullptr;
    void* tcws = nullptr;
    // FP64 method, dense A: digit planes of A (rows layout, for A X) and of A^T (cols
    // layout, for A^T X), sliced once per solve for the tensor-core products
    bool oz = false;
    OzCache ozA[2];
};

// Y (op.m x w) = op(A) X ; in precision TV with values V (sparse) or D (dense).
template <typename TV>
int apply(tsvd_handle* h, bool sparse, bool trans_of_A, int64_t M, int64_t N, int64_t nnz, const int32_t* rp,
          const int32_t* ci, const TV* va, const int32_t* trp, const int32_t* tci, const TV* tva,
          const SpmmPlan* pa, const SpmmPlan* pat, const TV* dA, int64_t lda, double* partial, int w, const TV* X,
          int64_t ldx, TV* Y, int64_t ldy, int* status, cudaStream_t st) {
    if (sparse) {
        if (!trans_of_A)
            TSVD_TRY_CUDA(launch_spmm<TV>(h, M, N, nnz, rp, ci, va, w, X, ldx, Y, ldy, status, st, pa));
        else
            TSVD_TRY_CUDA(launch_spmm<TV>(h, N, M, nnz, trp, tci, tva, w, X, ldx, Y, ldy, status, st, pat));
    } else {
        ProfClass pc(h, TSVD_K_APROD);
        if (!trans_of_A)
            TSVD_TRY_CUDA((gemm_nn<TV, TV, TV>(h, M, N, w, 1.0, dA, lda, X, ldx, 0.0, Y, ldy, false, st)));
        else
            TSVD_TRY_CUDA((gemm_tn<TV, TV>(h, M, N, w, dA, lda, X, ldx, Y, ldy, false, partial, st)));
    }
    return TSVD_OK;
}

// op(A) X and op(A)^T X in the working precision.
template <typename T>
int op_mul(tsvd_handle* h, Op<T>& op, int w, const T* X, int64_t ldx, T* Y, int64_t ldy, int* status,
           cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        if (op.tc) {
            TSVD_TRY_CUDA(op.transposed ? tc_mm(h, op.N, op.M, op.pAt, w, X, ldx, Y, ldy, op.tcws, status, st)
                                        : tc_mm(h, op.M, op.N, op.pA, w, X, ldx, Y, ldy, op.tcws, status, st));
            return TSVD_OK;
        }
    }
    return apply<T>(h, op.sparse, op.transposed, op.M, op.N, op.nnz, op.rp, op.ci, op.va, op.trp, op.tci, op.tva,
                    &op.plan_a, &op.plan_at, op.dA, op.lda, op.partial, w, X, ldx, Y, ldy, status, st);
}
template <typename T>
int op_tmul(tsvd_handle* h, Op<T>& op, int w, const T* X, int64_t ldx, T* Y, int64_t ldy, int* status,
            cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        if (op.tc) {
            TSVD_TRY_CUDA(op.transposed ? tc_mm(h, op.M, op.N, op.pA, w, X, ldx, Y, ldy, op.tcws, status, st)
                                        : tc_mm(h, op.N, op.M, op.pAt, w, X, ldx, Y, ldy, op.tcws, status, st));
            return TSVD_OK;
        }
    }
    return apply<T>(h, op.sparse, !op.transposed, op.M, op.N, op.nnz, op.rp, op.ci, op.va, op.trp, op.tci, op.tva,
                    &op.plan_a, &op.plan_at, op.dA, op.lda, op.partial, w, X, ldx, Y, ldy, status, st);
}
// op(A) X and op(A)^T X with the FP64 values (final Rayleigh-Ritz step and residuals).
template <typename T>
int op_mul64(tsvd_handle* h, Op<T>& op, int w, const double* X, int64_t ldx, double* Y, int64_t ldy, int* status,
             cudaStream_t st) {
    return apply<double>(h, op.sparse, op.transposed, op.M, op.N, op.nnz, op.rp, op.ci, op.va64, op.trp, op.tci,
                         op.tva64, &op.plan_a, &op.plan_at, op.dA64, op.lda64, op.partial, w, X, ldx, Y, ldy, status,
                         st);
}
template <typename T>
int op_tmul64(tsvd_handle* h, Op<T>& op, int w, const double* X, int64_t ldx, double* Y, int64_t ldy, int* status,
              cudaStream_t st) {
    return apply<double>(h, op.sparse, !op.transposed, op.M, op.N, op.nnz, op.rp, op.ci, op.va64, op.trp, op.tci,
                         op.tva64, &op.plan_a, &op.plan_at, op.dA64, op.lda64, op.partial, w, X, ldx, Y, ldy, status,
                         st);
}

size_t tn_partial_max(tsvd_handle* h, int64_t q, int64_t s, int wmax) {
    size_t pb = 0;
    for (int w = 1; w <= wmax; ++w) {
        for (int eb : {4, 8}) {
            const size_t v = gemm_tn_ws(h, q, s, w, false, eb);
            if (v > pb) pb = v;
        }
    }
    return pb;
}

// Carves and (when run) fills the operator: staged host input, CSR(A^T),
// value conversions between FP64 and FP32, dense split-K scratch.
template <typename T>
int setup_op(tsvd_handle* h, const tsvd_matrix* A, int wmax, Arena& ar, Op<T>& op, int* status, cudaStream_t st,
             bool run, float* ms_transpose, bool oz_planes = false, bool no_transpose = false) {
    constexpr bool kF64 = sizeof(T) == sizeof(double);
    const bool in64 = A->dtype == TSVD_F64;
    const bool host = A->location == TSVD_HOST;
    op.M = A->m;
    op.N = A->n;
    op.transposed = !no_transpose && A->m < A->n;
    op.m = op.transposed ? A->n : A->m;
    op.n = op.transposed ? A->m : A->n;
    op.sparse = A->format == TSVD_CSR;
    const int64_t M = A->m, N = A->n;
    if (op.sparse) {
        const int64_t nnz = A->nnz;
        op.nnz = nnz;
        const int32_t* rp = A->row_ptr;
        const int32_t* ci = A->col_idx;
        const void* va = A->val;
        if (host) {
            int32_t* drp = ar.take<int32_t>(M + 1);
            int32_t* dci = ar.take<int32_t>(nnz);
            void* dva = in64 ? (void*)ar.take<double>(nnz) : (void*)ar.take<float>(nnz);
            if (run) {
                if (!ar.fits()) return TSVD_ERR_WORKSPACE;
                TSVD_TRY_CUDA(cudaMemcpyAsync(drp, rp, sizeof(int32_t) * (M + 1), cudaMemcpyHostToDevice, st));
                TSVD_TRY_CUDA(cudaMemcpyAsync(dci, ci, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
                TSVD_TRY_CUDA(cudaMemcpyAsync(dva, va, (in64 ? 8 : 4) * nnz, cudaMemcpyHostToDevice, st));
            }
            rp = drp;
            ci = dci;
            va = dva;
        }
        op.rp = rp;
        op.ci = ci;
        op.trp = ar.take<int32_t>(N + 1);
        op.tci = ar.take<int32_t>(nnz);
        void* tva_in = in64 ? (void*)ar.take<double>(nnz) : (void*)ar.take<float>(nnz);
        if (run) {
            if (!ar.fits()) return TSVD_ERR_WORKSPACE;
            Arena tmp = ar;  // transpose scratch, dead after the build
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (ms_transpose) {
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                cudaEventRecord(e0, st);
            }
            const int rc = in64 ? csr_transpose<double>(h, M, N, nnz, rp, ci, (const double*)va, op.trp, op.tci,
                                                        (double*)tva_in, tmp, status, st)
                                : csr_transpose<float>(h, M, N, nnz, rp, ci, (const float*)va, op.trp, op.tci,
                                                       (float*)tva_in, tmp, status, st);
            if (ms_transpose) {
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(ms_transpose, e0, e1);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
            }
            if (rc < 0) return rc;
        } else {
            Arena tmp = ar;
            tmp.take<char>(csr_transpose_ws(M, N, nnz));
            ar.off = tmp.off;  // size the scratch (the run reuses it later)
        }
        // values in both precisions
        if (in64) {
            op.va64 = (const double*)va;
            op.tva64 = (const double*)tva_in;
        } else {
            double* v64 = ar.take<double>(nnz);
            double* tv64 = ar.take<double>(nnz);
            if (run) {
                if (!ar.fits()) return TSVD_ERR_WORKSPACE;
                TSVD_TRY_CUDA((convert2d<float, double>(h, 1, nnz, (const float*)va, nnz, v64, nnz, st)));
                TSVD_TRY_CUDA((convert2d<float, double>(h, 1, nnz, (const float*)tva_in, nnz, tv64, nnz, st)));
            }
            op.va64 = v64;
            op.tva64 = tv64;
        }
        if (kF64) {
            op.va = (const T*)op.va64;
            op.tva = (const T*)op.tva64;
        } else if (!in64) {
            op.va = (const T*)va;
            op.tva = (const T*)tva_in;
        } else {
            T* v = ar.take<T>(nnz);
            T* tv = ar.take<T>(nnz);
            if (run) {
                if (!ar.fits()) return TSVD_ERR_WORKSPACE;
                TSVD_TRY_CUDA((convert2d<double, T>(h, 1, nnz, op.va64, nnz, v, nnz, st)));
                TSVD_TRY_CUDA((convert2d<double, T>(h, 1, nnz, op.tva64, nnz, tv, nnz, st)));
            }
            op.va = v;
            op.tva = tv;
        }
        // long-row split plans (partials sized for FP64, which covers FP32)
        if (run) {
            TSVD_TRY(spmm_plan(h, M, nnz, op.rp, wmax, sizeof(double), ar, &op.plan_a, st));
            TSVD_TRY(spmm_plan(h, N, nnz, op.trp, wmax, sizeof(double), ar, &op.plan_at, st));
        } else {
            ar.take<char>(spmm_plan_ws(M, nnz, wmax, sizeof(double)));
            ar.take<char>(spmm_plan_ws(N, nnz, wmax, sizeof(double)));
        }
    } else {
        const void* a = A->val;
        int64_t lda = A->ld;
        if (host) {
            void* d = in64 ? (void*)ar.take<double>((size_t)M * N) : (void*)ar.take<float>((size_t)M * N);
            if (run) {
                if (!ar.fits()) return TSVD_ERR_WORKSPACE;
                const size_t es = in64 ? 8 : 4;
                TSVD_TRY_CUDA(cudaMemcpy2DAsync(d, es * N, a, es * lda, es * N, M, cudaMemcpyHostToDevice, st));
            }
            a = d;
            lda = N;
        }
        if (in64) {
            op.dA64 = (const double*)a;
            op.lda64 = lda;
        } else {
            double* d64 = ar.take<double>((size_t)M * N);
            if (run) {
                if (!ar.fits()) return TSVD_ERR_WORKSPACE;
                TSVD_TRY_CUDA((convert2d<float, double>(h, M, N, (const float*)a, lda, d64, N, st)));
            }
            op.dA64 = d64;
            op.lda64 = N;
        }
        if (kF64) {
            op.dA = (const T*)op.dA64;
            op.lda = op.lda64;
        } else {
            // mixed form: the products run on the tensor cores from BF16 pieces of A and
            // A^T (24 significant bits, as many as the FP32 values carry)
            op.tc = true;
            void* pa = ar.take<char>(bf16x3_bytes(M, N));
            void* pat = ar.take<char>(bf16x3_bytes(N, M));
            op.tcws = ar.take<char>(std::max(tc_mm_ws(M, N, wmax), tc_mm_ws(N, M, wmax)));
            if (run) {
                if (!ar.fits()) return TSVD_ERR_WORKSPACE;
                if (in64) {
                    TSVD_TRY_CUDA(bf16x3_split<double>(h, M, N, (const double*)a, lda, false, pa, st));
                    TSVD_TRY_CUDA(bf16x3_split<double>(h, M, N, (const double*)a, lda, true, pat, st));
                } else {
                    TSVD_TRY_CUDA(bf16x3_split<float>(h, M, N, (const float*)a, lda, false, pa, st));
                    TSVD_TRY_CUDA(bf16x3_split<float>(h, M, N, (const float*)a, lda, true, pat, st));
                }
            }
            op.pA = pa;
            op.pAt = pat;
        }
        op.partial = ar.take<double>(tn_partial_max(h, M, N, wmax) / sizeof(double) + 1);
        if (oz_planes) {
            op.oz = true;
            oz_cache_carve(op.ozA[0], ar, op.dA64, op.lda64, M, N, false, kOzNoFixedExp);
            oz_cache_carve(op.ozA[1], ar, op.dA64, op.lda64, M, N, true, kOzNoFixedExp);
            if (run) {
                if (!ar.fits()) return TSVD_ERR_WORKSPACE;
                TSVD_TRY(oz_cache_slice(h, op.ozA[0], 0, N, st));
                TSVD_TRY(oz_cache_slice(h, op.ozA[1], 0, N, st));
            }
        }
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

// Buffers of the final step and the outputs (FP64), shared by both methods.
struct Final {
    double *U64, *V64, *AV, *Mkk, *Uk, *Vk, *sk, *res, *cpart;
    double *oU, *oV, *osig;  // device outputs when the caller wants host outputs
    void* signws;
};

void carve_final(Arena& ar, const tsvd_opts* o, int64_t m, int64_t n, int k, bool mixed, Final& f) {
    f = Final{};
    if (mixed) {
        f.U64 = ar.take<double>((size_t)m * k);
        f.V64 = ar.take<double>((size_t)n * k);
        f.Mkk = ar.take<double>((size_t)k * k);
        f.Uk = ar.take<double>((size_t)k * k);
        f.Vk = ar.take<double>((size_t)k * k);
        f.sk = ar.take<double>(k);
    }
    f.AV = ar.take<double>((size_t)(m > n ? m : n) * k);
    f.res = ar.take<double>(2 * (size_t)k);
    f.cpart = ar.take<double>(colres_ws(m > n ? m : n, k) / sizeof(double) + 1);
    f.signws = ar.take<char>(sign_fix_ws(m > n ? m : n, k));
    if (o->output_location == TSVD_HOST) {
        f.oU = ar.take<double>((size_t)m * k);
        f.oV = ar.take<double>((size_t)n * k);
        f.osig = ar.take<double>(k);
    }
}

size_t final_tail_ws(tsvd_handle* h, int64_t m, int64_t n, int k, bool mixed) {
    if (!mixed) return 0;
    size_t a = orth_ws(h, m, 0, k), b = orth_ws(h, n, 0, k), c = small_svd_ws(k);
    size_t p = tn_partial_max(h, m, k, k);
    size_t r = a > b ? a : b;
    if (c > r) r = c;
    return r + p + 256;
}

// The returned triplets from the last small SVD: sigma, U = Bm Wm[:, :k],
// V = Bn Wn[:, :k] (FP64 path), or the same followed by the FP64 Rayleigh-Ritz
// step (mixed path).  Writes dev.{U,V,sigma} in op orientation.
// In the mixed form the first s0 basis columns may have FP64 master copies (Mm, Mn:
// the kept Ritz vectors of a thick restart); their share of U and V is then formed
// from the masters in FP64.
template <typename T>
int final_triplets(tsvd_handle* h, Op<T>& op, int k, const T* Bm, int64_t ldbm, const double* Wm, int64_t ldwm,
                   const T* Bn, int64_t ldbn, const double* Wn, int64_t ldwn, int wdim, const double* sig,
                   Final& f, double* dU, double* dV, double* dsig, OrthCtx& ctx, Arena tail, int* status,
                   cudaStream_t st, int* sweeps, const double* Mm = nullptr, int64_t ldmm = 0,
                   const double* Mn = nullptr, int64_t ldmn = 0, int s0 = 0) {
    constexpr bool kF64 = sizeof(T) == sizeof(double);
    const int64_t m = op.m, n = op.n;
    if (kF64) {
        OzFreshRows fresh(h);  // the returned vectors to full FP64 accuracy
        TSVD_TRY_CUDA((gemm_nn<T, double, double>(h, m, wdim, k, 1.0, Bm, ldbm, Wm, ldwm, 0.0, dU, k, false, st)));
        TSVD_TRY_CUDA((gemm_nn<T, double, double>(h, n, wdim, k, 1.0, Bn, ldbn, Wn, ldwn, 0.0, dV, k, false, st)));
        TSVD_TRY_CUDA(cudaMemcpyAsync(dsig, sig, sizeof(double) * k, cudaMemcpyDeviceToDevice, st));
        return TSVD_OK;
    }
    // FP64 Rayleigh-Ritz on span(U), span(V)
    if (s0 > 0 && Mm && Mn) {
        // the FP32 columns first, then the FP64 masters added by the FP64 kernel
        TSVD_TRY_CUDA((gemm_nn<T, double, double>(h, m, wdim - s0, k, 1.0, Bm + s0, ldbm, Wm + (int64_t)s0 * ldwm,
                                                  ldwm, 0.0, f.U64, k, false, st)));
        TSVD_TRY_CUDA((gemm_nn<double, double, double>(h, m, s0, k, 1.0, Mm, ldmm, Wm, ldwm, 1.0, f.U64, k, false,
                                                       st)));
        TSVD_TRY_CUDA((gemm_nn<T, double, double>(h, n, wdim - s0, k, 1.0, Bn + s0, ldbn, Wn + (int64_t)s0 * ldwn,
                                                  ldwn, 0.0, f.V64, k, false, st)));
        TSVD_TRY_CUDA((gemm_nn<double, double, double>(h, n, s0, k, 1.0, Mn, ldmn, Wn, ldwn, 1.0, f.V64, k, false,
                                                       st)));
    } else {
        TSVD_TRY_CUDA((gemm_nn<T, double, double>(h, m, wdim, k, 1.0, Bm, ldbm, Wm, ldwm, 0.0, f.U64, k, false, st)));
        TSVD_TRY_CUDA((gemm_nn<T, double, double>(h, n, wdim, k, 1.0, Bn, ldbn, Wn, ldwn, 0.0, f.V64, k, false, st)));
    }
    TSVD_TRY(cgs_cqr2<double>(h, m, 0, k, nullptr, 0, f.U64, k, nullptr, f.Mkk, k, false, ctx, tail, status, st));
    TSVD_TRY(cgs_cqr2<double>(h, n, 0, k, nullptr, 0, f.V64, k, nullptr, f.Mkk, k, false, ctx, tail, status, st));
    TSVD_TRY(op_mul64(h, op, k, f.V64, k, f.AV, k, status, st));
    Arena t2 = tail;
    double* part = t2.take<double>(tn_partial_max(h, m, k, k) / sizeof(double) + 1);
    if (!t2.fits()) return TSVD_ERR_WORKSPACE;
    TSVD_TRY_CUDA((gemm_tn<double, double>(h, m, k, k, f.U64, k, f.AV, k, f.Mkk, k, false, part, st)));
    TSVD_TRY(small_svd(h, k, f.Mkk, k, f.Uk, f.sk, f.Vk, k, t2, status, st));
    TSVD_TRY_CUDA((gemm_nn<double, double, double>(h, m, k, k, 1.0, f.U64, k, f.Uk, k, 0.0, dU, k, false, st)));
    TSVD_TRY_CUDA((gemm_nn<double, double, double>(h, n, k, k, 1.0, f.V64, k, f.Vk, k, 0.0, dV, k, false, st)));
    TSVD_TRY_CUDA(cudaMemcpyAsync(dsig, f.sk, sizeof(double) * k, cudaMemcpyDeviceToDevice, st));
    (void)sweeps;
    return TSVD_OK;
}

// max_j max(||op(A) v_j - s_j u_j||, ||op(A)^T u_j - s_j v_j||) / s_1 with the FP64 A
// (both one-sided residuals: the second vanishes by construction in the FP64
// method, not after the mixed form's two-sided Rayleigh-Ritz step).
template <typename T>
int explicit_residual(tsvd_handle* h, Op<T>& op, int k, const double* U, const double* V, const double* sigma,
                      Final& f, int* status, cudaStream_t st, double* out, bool part = false) {
    TSVD_TRY(op_mul64(h, op, k, V, k, f.AV, k, status, st));
    TSVD_TRY_CUDA(col_residual_sq(h, op.m, k, f.AV, k, U, k, sigma, f.res, f.cpart, st));
    if (part) TSVD_TRY(part_sum(h, f.res, 1, k, k, st));  // this process's rows of A V - U S
    TSVD_TRY(op_tmul64(h, op, k, U, k, f.AV, k, status, st));
    if (part) TSVD_TRY(part_sum(h, f.AV, op.n, k, k, st));  // A^T U over all rows
    TSVD_TRY_CUDA(col_residual_sq(h, op.n, k, f.AV, k, V, k, sigma, f.res + k, f.cpart, st));
    std::vector<double> hres(2 * k), hs(1);
    TSVD_TRY_CUDA(cudaMemcpyAsync(hres.data(), f.res, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, st));
    TSVD_TRY_CUDA(cudaMemcpyAsync(hs.data(), sigma, sizeof(double), cudaMemcpyDeviceToHost, st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    double mx = 0.0;
    for (int j = 0; j < 2 * k; ++j) mx = std::fmax(mx, std::sqrt(hres[j]));
    *out = hs[0] > 0.0 ? mx / hs[0] : NAN;
    return TSVD_OK;
}

// Sign convention, copies to the caller (host or device), U/V swap when transposed.
template <typename T>
int finish_outputs(tsvd_handle* h, const tsvd_opts* o, Op<T>& op, int k, double* dU, double* dV, double* dsig,
                   Final& f, double* sigma, double* U, double* V, cudaStream_t st) {
    TSVD_TRY_CUDA(sign_fix(h, op.n, op.m, k, dV, k, dU, k, f.signws, st));
    if (o->output_location == TSVD_HOST) {
        double* userU = op.transposed ? V : U;
        double* userV = op.transposed ? U : V;
        TSVD_TRY_CUDA(cudaMemcpyAsync(sigma, dsig, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        TSVD_TRY_CUDA(cudaMemcpyAsync(userU, dU, sizeof(double) * op.m * k, cudaMemcpyDeviceToHost, st));
        TSVD_TRY_CUDA(cudaMemcpyAsync(userV, dV, sizeof(double) * op.n * k, cudaMemcpyDeviceToHost, st));
    }
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}

int status_code(const int* hs) {
    if (hs[kStTimeout]) return TSVD_ERR_TIMEOUT;
    if (hs[kStNonfinite]) return TSVD_ERR_NONFINITE;
    if (hs[kStBadCsr]) return TSVD_ERR_INVALID_ARG;
    return TSVD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// RandSVD
// ---------------------------------------------------------------------------
template <typename T>
int rsvd_run(tsvd_handle* h, const tsvd_matrix* A, int k, int p, int q, int bq, uint64_t seed, const tsvd_opts* o,
             char* ws, size_t ws_bytes, size_t* sizing, double* sigma, double* U, double* V, tsvd_info* info) {
    constexpr bool kMixed = sizeof(T) != sizeof(double);
    const bool run = sizing == nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(o->stream);
    Arena ar{run ? ws : nullptr, ws_bytes, 0};
    int* status = ar.take<int>(kStCount);
    if (run) {
        if (!ar.fits()) return TSVD_ERR_WORKSPACE;
        TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    }
    const int ell = k + p;
    const int64_t l0 = h->launches;
    Timer* total = run ? new Timer(st) : nullptr;
    struct Del {
        Timer* t;
        ~Del() { delete t; }
    } del{total};
    Op<T> op;
    float ms_t = 0.f;
    if ((o->flags & TSVD_FLAG_ROW_PARTITION) || (run && h->part_fn)) return TSVD_ERR_UNSUPPORTED;
    TSVD_TRY(setup_op<T>(h, A, ell > k ? ell : k, ar, op, status, st, run, A->format == TSVD_CSR ? &ms_t : nullptr,
                         true));
    OzCacheScope ocs(h);
    if (op.oz && run) {
        ocs.add(&op.ozA[0]);
        ocs.add(&op.ozA[1]);
    }
    const int64_t m = op.m, n = op.n;
    T* Qn = ar.take<T>((size_t)n * ell);
    T* Qm = ar.take<T>((size_t)m * ell);
    double* R = ar.take<double>((size_t)ell * ell);
    double* Ub = ar.take<double>((size_t)ell * ell);
    double* Vb = ar.take<double>((size_t)ell * ell);
    double* sig = ar.take<double>(ell);
    double* g64 = kMixed ? ar.take<double>((size_t)n * ell) : nullptr;
    T* Qsave = ar.take<T>((size_t)n * ell);
    Final f;
    carve_final(ar, o, m, n, k, kMixed, f);
    // scratch of the FP64-accurate tensor-core products (the mixed form's FP64 final
    // Rayleigh-Ritz step and residual use them too)
    const size_t ozb = oz_ws_bound(std::max(m, n), kMixed ? k : ell, kMixed ? k : ell);
    void* ozws = ar.take<char>(ozb);
    if (!run) {
        const int64_t qmax = m > n ? m : n;
        size_t t1 = orth_ws(h, qmax, ell > bq ? ell - bq : 0, bq) + align256(sizeof(double) * (size_t)ell * bq);
        const size_t t2 = small_svd_ws(ell), t3 = final_tail_ws(h, m, n, k, kMixed);
        if (t2 > t1) t1 = t2;
        if (t3 > t1) t1 = t3;
        *sizing = ar.off + t1 + 256;
        return TSVD_OK;
    }
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    OzScope oz(h, ozws, ozb, status);
    OrthCtx ctx;
    ctx.seed = seed;
    // Q_0 (n x l): raw Gaussian block (Alg. 1)
    if (o->start_block) {
        TSVD_TRY_CUDA((convert2d<double, T>(h, n, ell, o->start_block, ell, Qn, ell, st)));
    } else if (kMixed) {
        TSVD_TRY_CUDA(gaussian(h, n, ell, seed, 1u, g64, ell, st));
        TSVD_TRY_CUDA((convert2d<double, T>(h, n, ell, g64, ell, Qn, ell, st)));
    } else {
        TSVD_TRY_CUDA(gaussian(h, n, ell, seed, 1u, reinterpret_cast<double*>(Qn), ell, st));
    }
    int iters = 0;
    int hs[kStCount];
    for (int it = 0; it <= q; ++it) {
        // unchecked trip first; if a Cholesky broke down, restore Q and redo the trip checked
        TSVD_TRY_CUDA(copy_block<T>(Qn, ell, Qsave, ell, n, ell, st));
        for (int pass = 0; pass < 2; ++pass) {
            ctx.deferred = (pass == 0);
            TSVD_TRY(op_mul<T>(h, op, ell, Qn, ell, Qm, ell, status, st));               // S1
            TSVD_TRY(cgs_qr<T>(h, m, ell, bq, Qm, ell, R, ctx, ar, status, st));        // S2
            TSVD_TRY(op_tmul<T>(h, op, ell, Qm, ell, Qn, ell, status, st));              // S3
            TSVD_TRY(cgs_qr<T>(h, n, ell, bq, Qn, ell, R, ctx, ar, status, st));        // S4
            ctx.deferred = false;
            if (pass == 1) break;
            TSVD_TRY(read_status(st, status, hs));
            if (!hs[kStBreakdown]) {
                TSVD_TRY(status_code(hs));
                break;
            }
            TSVD_TRY_CUDA(cudaMemsetAsync(status + kStBreakdown, 0, 2 * sizeof(int), st));
            TSVD_TRY_CUDA(copy_block<T>(Qsave, ell, Qn, ell, n, ell, st));
        }
        ++iters;
    }
    {
        Arena sv = ar;
        TSVD_TRY(small_svd(h, ell, R, ell, Ub, sig, Vb, k, sv, status, st));           // S5
    }
    double* dU = f.oU ? f.oU : (op.transposed ? V : U);
    double* dV = f.oV ? f.oV : (op.transposed ? U : V);
    double* dsig = f.osig ? f.osig : sigma;
    // S6 U = Qbar Vbar, S7 V = Q Ubar (then the FP64 Rayleigh-Ritz step in the mixed form)
    TSVD_TRY(final_triplets<T>(h, op, k, Qm, ell, Vb, ell, Qn, ell, Ub, ell, ell, sig, f, dU, dV, dsig, ctx, ar,
                               status, st, nullptr));
    TSVD_TRY(read_status(st, status, hs));
    TSVD_TRY(status_code(hs));
    const int sweeps = hs[kStSweeps];
    prof_set_last_flops(h, TSVD_K_SVD, jacobi_flops(ell, k, sweeps));
    TSVD_TRY(finish_outputs<T>(h, o, op, k, dU, dV, dsig, f, sigma, U, V, st));
    const double ms_total = total->stop();
    double resid = NAN;
    TSVD_TRY(explicit_residual<T>(h, op, k, dU, dV, dsig, f, status, st, &resid));
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

// ---------------------------------------------------------------------------
// LancSVD
// ---------------------------------------------------------------------------
template <typename T>
int blanczos_run(tsvd_handle* h, const tsvd_matrix* A, int k, int b, int r, uint64_t seed, const tsvd_opts* o,
                 char* ws, size_t ws_bytes, size_t* sizing, double* sigma, double* U, double* V, tsvd_info* info) {
    constexpr bool kMixed = sizeof(T) != sizeof(double);
    const bool run = sizing == nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(o->stream);
    Arena ar{run ? ws : nullptr, ws_bytes, 0};
    int* status = ar.take<int>(kStCount);
    if (run) {
        if (!ar.fits()) return TSVD_ERR_WORKSPACE;
        TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    }
    const int rb = r * b;
    const int64_t l0 = h->launches;
    Timer* total = run ? new Timer(st) : nullptr;
    struct Del {
        Timer* t;
        ~Del() { delete t; }
    } del{total};
    Op<T> op;
    float ms_t = 0.f;
    // row partition: this process's rows of A and of the left basis; sums over the
    // rows (Gram matrices, projections, A^T Qbar, residual norms) are summed over the
    // processes, everything n-side and small is replicated
    const bool part = (o->flags & TSVD_FLAG_ROW_PARTITION) != 0;
    if (part && (kMixed || (run && !h->part_fn))) return kMixed ? TSVD_ERR_UNSUPPORTED : TSVD_ERR_INVALID_ARG;
    if (!part && run && h->part_fn) return TSVD_ERR_INVALID_ARG;
    TSVD_TRY(setup_op<T>(h, A, b > k ? b : k, ar, op, status, st, run, A->format == TSVD_CSR ? &ms_t : nullptr,
                         true, part));
    OzCacheScope ocs(h);
    if (op.oz && run) {
        ocs.add(&op.ozA[0]);
        ocs.add(&op.ozA[1]);
    }
    const int64_t m = op.m, n = op.n;
    const int keep = o->restart_keep;                   // thick restart when > 0
    const int nv = std::max(std::max(k, b), keep);      // right vectors the small SVD must return
    T* P = ar.take<T>((size_t)n * rb);
    T* Pbar = ar.take<T>((size_t)m * rb);
    T* Qnext = ar.take<T>((size_t)m * b);
    T* Pk = keep ? ar.take<T>((size_t)n * keep) : nullptr;    // P Vbar_s, Pbar Ubar_s
    T* Pbk = keep ? ar.take<T>((size_t)m * keep) : nullptr;
    // mixed form: FP64 master copies of the kept Ritz vectors (two generations each); the
    // bases hold their FP32 rounding for the orthogonalisations
    const bool masters = kMixed && keep > 0;
    double* Pk64[2] = {nullptr, nullptr};
    double* Pbk64[2] = {nullptr, nullptr};
    if (masters)
        for (int g = 0; g < 2; ++g) {
            Pk64[g] = ar.take<double>((size_t)n * keep);
            Pbk64[g] = ar.take<double>((size_t)m * keep);
        }
    int cur = 0;
    double* Hk = keep ? ar.take<double>((size_t)keep * b) : nullptr;  // coefficients of A^T Qbar on P Vbar_s
    double* B = ar.take<double>((size_t)rb * rb);
    double* Ub = ar.take<double>((size_t)rb * rb);
    double* Vb = ar.take<double>((size_t)rb * rb);
    double* sig = ar.take<double>(rb);
    double* Rr = ar.take<double>((size_t)b * b);
    double* Bsave = ar.take<double>((size_t)rb * rb);  // B at the start of a cycle (redo after a breakdown)
    double* rho = ar.take<double>(k);
    double* g64 = kMixed ? ar.take<double>((size_t)m * b) : nullptr;
    Final f;
    carve_final(ar, o, m, n, k, kMixed, f);
    // FP64 method: scratch of the FP64-accurate tensor-core products, and the digit
    // planes of both bases, kept up to date block by block: cols layout (per-column
    // exponents) for P^T Y, rows layout (the fixed exponent 1 of an orthonormal basis,
    // |entries| < 2) for P H and the Ritz products
    const size_t ozb = kMixed ? oz_ws_bound(std::max(m, n), std::max(k, keep), std::max(k, keep))
                              : oz_ws_bound(std::max(m, n), rb, std::max(std::max(b, k), keep));
    void* ozws = ar.take<char>(ozb);
    OzCache cP[2], cPb[2];
    if (!kMixed) {
        for (int l = 0; l < 2; ++l) {
            oz_cache_carve(cP[l], ar, reinterpret_cast<const double*>(P), rb, n, rb, l == 0, l == 0 ? kOzNoFixedExp : 1);
            oz_cache_carve(cPb[l], ar, reinterpret_cast<const double*>(Pbar), rb, m, rb, l == 0,
                           l == 0 ? kOzNoFixedExp : 1);
        }
        if (run)
            for (int l = 0; l < 2; ++l) {
                ocs.add(&cP[l]);
                ocs.add(&cPb[l]);
            }
    }
    // columns [c0, c1) of a basis were written: slice them (c0 <= the current prefix)
    auto slice_cols = [&](OzCache* c, int64_t c0, int64_t c1) -> int {
        if (kMixed) return TSVD_OK;
        for (int l = 0; l < 2; ++l) TSVD_TRY(oz_cache_slice(h, c[l], c0, c1, st));
        return TSVD_OK;
    };
    // columns from v on are about to be rewritten: the caches no longer cover them
    auto keep_cols = [&](OzCache* c, int64_t v) -> int {
        if (kMixed) return TSVD_OK;
        for (int l = 0; l < 2; ++l) TSVD_TRY(oz_cache_truncate(h, c[l], v, st));
        return TSVD_OK;
    };
    if (!run) {
        size_t t1 = orth_ws(h, m, rb, b);
        const size_t t2 = orth_ws(h, n, rb, b), t3 = small_svd_ws(rb), t4 = final_tail_ws(h, m, n, k, kMixed);
        if (t2 > t1) t1 = t2;
        if (t3 > t1) t1 = t3;
        if (t4 > t1) t1 = t4;
        *sizing = ar.off + t1 + 256;
        return TSVD_OK;
    }
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    OzScope oz(h, ozws, ozb, status);
    OrthCtx ctx;  // n-side blocks (replicated)
    ctx.seed = seed;
    OrthCtx mctx;  // m-side blocks (this process's rows when partitioned)
    mctx.seed = seed;
    mctx.reduce = part;
    mctx.row0 = part ? h->part_row0 : 0;
    double* dU = f.oU ? f.oU : (op.transposed ? V : U);
    double* dV = f.oV ? f.oV : (op.transposed ? U : V);
    double* dsig = f.osig ? f.osig : sigma;
    // S1: random orthonormal Qbar_1 (m x b) in the first block column of Pbar
    if (o->start_block) {
        TSVD_TRY_CUDA((convert2d<double, T>(h, m, b, o->start_block, b, Pbar, rb, st)));
    } else if (kMixed) {
        TSVD_TRY_CUDA(gaussian(h, m, b, seed, 2u, g64, b, st));
        TSVD_TRY_CUDA((convert2d<double, T>(h, m, b, g64, b, Pbar, rb, st)));
    } else {
        TSVD_TRY_CUDA(gaussian(h, m, b, seed, 2u, reinterpret_cast<double*>(Pbar), rb, st, mctx.row0));
    }
    TSVD_TRY(cgs_cqr2<T>(h, m, 0, b, nullptr, 0, Pbar, rb, nullptr, Rr, b, false, mctx, ar, status, st));
    TSVD_TRY(slice_cols(cPb, 0, b));
    int cycles = 0, restarts = 0, sweeps = 0, converged = 0;
    double rho_last = NAN, resid = NAN;
    std::vector<double> hrho(k), hsig(1);
    int hs[kStCount];
    // A cycle first runs deferred: its orthogonalisations are not synchronised, a
    // Cholesky breakdown only sets the sticky status word, and the word is read once,
    // with the Lanczos estimate, after the cycle.  If it is set, the cycle is redone
    // from its saved start (the bases' leading columns and the start block are not
    // written by the cycle; B is restored) with every orthogonalisation checked, so
    // that the fallback runs where it is needed; later cycles then stay checked (with
    // basic restart, the first S5 after a restart breaks down in most cycles near
    // convergence: converged Ritz vectors deflate the new block).
    // s0 = Ritz pairs carried into the current cycle (thick restart), d = its dimension:
    // basis [P~ (s0), Q_1 .. Q_nblk], [Pbar~ (s0), Qbar_1 .. Qbar_nblk], B d x d with
    // diag(S_s0) and the coupling block G below it (see the thick-restart reading)
    int s0 = 0;
    bool defer = true;
    for (;;) {
        const int nblk = s0 == 0 ? r : (rb - s0) / b;
        const int d = s0 + nblk * b;
        if (s0 == 0) TSVD_TRY_CUDA(cudaMemsetAsync(B, 0, sizeof(double) * (size_t)rb * rb, st));
        if (defer)
            TSVD_TRY_CUDA(cudaMemcpyAsync(Bsave, B, sizeof(double) * (size_t)rb * rb, cudaMemcpyDeviceToDevice, st));
        for (int pass = 0; pass < 2; ++pass) {
            ctx.deferred = defer && pass == 0;
            mctx.deferred = ctx.deferred;
            TSVD_TRY(keep_cols(cP, s0));
            TSVD_TRY(keep_cols(cPb, s0 + b));
            for (int i = 0; i < nblk; ++i) {
                const int c0 = s0 + i * b;
                T* Qi = P + c0;
                TSVD_TRY(op_tmul<T>(h, op, b, Pbar + c0, rb, Qi, rb, status, st));                    // S2
                if (part) TSVD_TRY(part_sum(h, reinterpret_cast<double*>(Qi), n, b, rb, st));
                double* Lii = B + (int64_t)c0 * rb + c0;
                const bool couple = (i == 0 && s0 > 0);
                TSVD_TRY(cgs_cqr2<T>(h, n, c0, b, P, rb, Qi, rb, couple ? Hk : nullptr, Lii, rb, true, ctx, ar, status,
                                     st));                                                                // S3
                if (couple) TSVD_TRY_CUDA(put_transposed(h, s0, b, Hk, b, B + (int64_t)c0 * rb, rb, st));  // G
                TSVD_TRY(slice_cols(cP, c0, c0 + b));
                const bool last = (i + 1 == nblk);
                T* dst = last ? Qnext : Pbar + c0 + b;
                const int64_t ldd = last ? b : rb;
                TSVD_TRY(op_mul<T>(h, op, b, Qi, rb, dst, ldd, status, st));                             // S4
                double* Ri = last ? Rr : B + (int64_t)(c0 + b) * rb + c0;
                TSVD_TRY(cgs_cqr2<T>(h, m, c0 + b, b, Pbar, rb, dst, ldd, nullptr, Ri, last ? b : rb, false, mctx,
                                     ar, status, st));                                                   // S5
                if (!last) TSVD_TRY(slice_cols(cPb, c0 + b, c0 + 2 * b));
            }
            {
                Arena sv = ar;
                TSVD_TRY(small_svd(h, d, B, rb, Ub, sig, Vb, nv, sv, status, st, ctx.deferred, o->tol));  // S6
            }
            TSVD_TRY_CUDA(lanczos_rho(h, b, k, Rr, Vb + (int64_t)(d - b) * d, d, rho, st));
            TSVD_TRY_CUDA(cudaMemcpyAsync(hrho.data(), rho, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
            TSVD_TRY_CUDA(cudaMemcpyAsync(hsig.data(), sig, sizeof(double), cudaMemcpyDeviceToHost, st));
            TSVD_TRY(read_status(st, status, hs));
            if (!(ctx.deferred && hs[kStBreakdown])) break;
            // a deferred cycle met a breakdown: redo it checked
            TSVD_TRY_CUDA(cudaMemsetAsync(status + kStBreakdown, 0, 2 * sizeof(int), st));
            TSVD_TRY_CUDA(cudaMemcpyAsync(B, Bsave, sizeof(double) * (size_t)rb * rb, cudaMemcpyDeviceToDevice, st));
            defer = false;
        }
        ctx.deferred = false;
        mctx.deferred = false;
        ++cycles;
        TSVD_TRY(status_code(hs));
        sweeps = hs[kStSweeps];
        prof_set_last_flops(h, TSVD_K_SVD, jacobi_flops(d, nv, sweeps));
        double rmax = 0.0;
        for (int j = 0; j < k; ++j) rmax = std::fmax(rmax, hrho[j]);
        rho_last = hsig[0] > 0.0 ? rmax / hsig[0] : NAN;
        const bool done = rho_last <= o->tol;
        if (done || restarts >= o->max_restarts) {
            // S8/S9 (and the FP64 Rayleigh-Ritz step in the mixed form)
            const bool with_masters = masters && s0 > 0;
            TSVD_TRY(final_triplets<T>(h, op, k, Pbar, rb, Ub, d, P, rb, Vb, d, d, sig, f, dU, dV, dsig, ctx, ar,
                                       status, st, nullptr, with_masters ? Pbk64[cur] : nullptr, keep,
                                       with_masters ? Pk64[cur] : nullptr, keep, with_masters ? s0 : 0));
            TSVD_TRY(explicit_residual<T>(h, op, k, dU, dV, dsig, f, status, st, &resid, part));
            if ((done && resid <= o->tol) || restarts >= o->max_restarts) {
                converged = resid <= o->tol ? 1 : 0;
                break;
            }
        }
        ++restarts;
        if (keep > 0) {
            // thick restart: P~ = P Vbar_s, Pbar~ = Pbar Ubar_s, B = diag(S_s) on them, and the
            // residual block Qbar_{r+1} continues the recurrence as the next left block
            if (masters) {
                // new FP64 masters from the FP32 columns and the old masters, then their
                // FP32 rounding into the bases
                double* nPk = Pk64[1 - cur];
                double* nPbk = Pbk64[1 - cur];
                TSVD_TRY_CUDA((gemm_nn<T, double, double>(h, n, d - s0, keep, 1.0, P + s0, rb, Vb + (int64_t)s0 * d,
                                                          d, 0.0, nPk, keep, false, st)));
                TSVD_TRY_CUDA((gemm_nn<T, double, double>(h, m, d - s0, keep, 1.0, Pbar + s0, rb,
                                                          Ub + (int64_t)s0 * d, d, 0.0, nPbk, keep, false, st)));
                if (s0 > 0) {
                    TSVD_TRY_CUDA((gemm_nn<double, double, double>(h, n, s0, keep, 1.0, Pk64[cur], keep, Vb, d, 1.0,
                                                                   nPk, keep, false, st)));
                    TSVD_TRY_CUDA((gemm_nn<double, double, double>(h, m, s0, keep, 1.0, Pbk64[cur], keep, Ub, d, 1.0,
                                                                   nPbk, keep, false, st)));
                }
                cur = 1 - cur;
                TSVD_TRY_CUDA((convert2d<double, T>(h, n, keep, Pk64[cur], keep, P, rb, st)));
                TSVD_TRY_CUDA((convert2d<double, T>(h, m, keep, Pbk64[cur], keep, Pbar, rb, st)));
            } else {
                OzFreshRows fresh(h);  // the kept Ritz vectors to full FP64 accuracy
                TSVD_TRY_CUDA((gemm_nn<T, double, T>(h, n, d, keep, 1.0, P, rb, Vb, d, 0.0, Pk, keep, false, st)));
                TSVD_TRY_CUDA((gemm_nn<T, double, T>(h, m, d, keep, 1.0, Pbar, rb, Ub, d, 0.0, Pbk, keep, false, st)));
                TSVD_TRY(keep_cols(cP, 0));
                TSVD_TRY(keep_cols(cPb, 0));
                TSVD_TRY_CUDA(copy_block<T>(Pk, keep, P, rb, n, keep, st));
                TSVD_TRY_CUDA(copy_block<T>(Pbk, keep, Pbar, rb, m, keep, st));
            }
            TSVD_TRY(keep_cols(cPb, keep));
            TSVD_TRY_CUDA(copy_block<T>(Qnext, b, Pbar + keep, rb, m, b, st));
            TSVD_TRY(slice_cols(cP, 0, keep));
            TSVD_TRY(slice_cols(cPb, 0, keep + b));
            TSVD_TRY_CUDA(cudaMemsetAsync(B, 0, sizeof(double) * (size_t)rb * rb, st));
            TSVD_TRY_CUDA(put_diagonal(h, keep, sig, B, rb, st));
            s0 = keep;
        } else {
            // S7: Qbar_1 = Pbar Ubar_1, re-orthonormalised by CholeskyQR2
            {
                OzFreshRows fresh(h);
                TSVD_TRY_CUDA((gemm_nn<T, double, T>(h, m, rb, b, 1.0, Pbar, rb, Ub, rb, 0.0, Qnext, b, false, st)));
            }
            TSVD_TRY(keep_cols(cP, 0));
            TSVD_TRY(keep_cols(cPb, 0));
            TSVD_TRY_CUDA(copy_block<T>(Qnext, b, Pbar, rb, m, b, st));
            TSVD_TRY(cgs_cqr2<T>(h, m, 0, b, nullptr, 0, Pbar, rb, nullptr, Rr, b, false, mctx, ar, status, st));
            TSVD_TRY(slice_cols(cPb, 0, b));
        }
    }
    TSVD_TRY(read_status(st, status, hs));
    TSVD_TRY(status_code(hs));
    TSVD_TRY(finish_outputs<T>(h, o, op, k, dU, dV, dsig, f, sigma, U, V, st));
    const double ms_total = total->stop();
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->iterations = cycles;
        info->restarts = restarts;
        info->breakdowns = ctx.fallbacks + mctx.fallbacks;
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
// Gradient of a loss on the k leading triplets (see backward.cu for the formula).
namespace {

// One side's complement solves by CG: columns x_j of X (rows x k) with
// (s_j^2 I - G) x_j = (I - Q Q^T) rhs_j on the complement of span(Q), where
// G = op2(op1(.)) is A A^T (op1 = A^T, op2 = A) or A^T A.  Every operator
// application is projected back onto the complement.
struct CgBufs {
    double *R, *P, *AP, *T, *H, *rr, *rr_new, *pap, *bb, *alpha, *beta, *part, *cpart;
};

template <typename F1, typename F2>
int cg_side(tsvd_handle* h, int64_t rows, int k, const double* Q, const double* rhs, const double* s, F1 op1, F2 op2,
            double* X, const tsvd_backward_opts* o, CgBufs& b, cudaStream_t st, int* iters, double* resid) {
    const size_t bytes = sizeof(double) * (size_t)rows * k;
    auto project = [&](double* Z) -> int {
        TSVD_TRY_CUDA((gemm_tn<double, double>(h, rows, k, k, Q, k, Z, k, b.H, k, false, b.part, st)));
        TSVD_TRY_CUDA((gemm_nn<double, double, double>(h, rows, k, k, -1.0, Q, k, b.H, k, 1.0, Z, k, false, st)));
        return TSVD_OK;
    };
    TSVD_TRY_CUDA(cudaMemcpyAsync(b.R, rhs, bytes, cudaMemcpyDeviceToDevice, st));
    TSVD_TRY(project(b.R));
    TSVD_TRY_CUDA(cudaMemsetAsync(X, 0, bytes, st));
    TSVD_TRY_CUDA(cudaMemcpyAsync(b.P, b.R, bytes, cudaMemcpyDeviceToDevice, st));
    TSVD_TRY_CUDA(coldot(h, rows, k, b.R, k, b.R, k, b.bb, b.cpart, st));
    TSVD_TRY_CUDA(cudaMemcpyAsync(b.rr, b.bb, sizeof(double) * k, cudaMemcpyDeviceToDevice, st));
    const double tol2 = o->cg_tol * o->cg_tol;
    std::vector<double> hrr(k), hbb(k);
    int it = 0;
    double worst = 0.0;
    for (;;) {
        const bool check = (it % std::max(1, o->check_every) == 0) || it >= o->cg_max_iter;
        if (check) {
            TSVD_TRY_CUDA(cudaMemcpyAsync(hrr.data(), b.rr, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
            TSVD_TRY_CUDA(cudaMemcpyAsync(hbb.data(), b.bb, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
            TSVD_TRY_CUDA(cudaStreamSynchronize(st));
            bool done = true;
            worst = 0.0;
            for (int j = 0; j < k; ++j) {
                if (!std::isfinite(hrr[j])) return TSVD_ERR_NONFINITE;
                if (hbb[j] > 0.0) {
                    worst = std::fmax(worst, std::sqrt(hrr[j] / hbb[j]));
                    if (hrr[j] > tol2 * hbb[j]) done = false;
                }
            }
            if (done || it >= o->cg_max_iter) break;
        }
        TSVD_TRY(op1(b.P, b.T));                                                  // T = op1(P)
        TSVD_TRY(op2(b.T, b.AP));                                                 // AP = op2(T)
        TSVD_TRY_CUDA(shifted(h, rows, k, s, b.P, b.AP, b.AP, st));               // AP = s^2 P - G P
        TSVD_TRY(project(b.AP));
        TSVD_TRY_CUDA(coldot(h, rows, k, b.P, k, b.AP, k, b.pap, b.cpart, st));
        TSVD_TRY_CUDA(cg_alpha(h, k, b.rr, b.pap, b.bb, tol2, b.alpha, st));
        TSVD_TRY_CUDA(cg_xr(h, rows, k, b.alpha, b.P, b.AP, X, b.R, st));
        TSVD_TRY_CUDA(coldot(h, rows, k, b.R, k, b.R, k, b.rr_new, b.cpart, st));
        TSVD_TRY_CUDA(cg_beta(h, k, b.rr, b.rr_new, b.alpha, b.beta, st));
        TSVD_TRY_CUDA(cg_p(h, rows, k, b.alpha, b.beta, b.R, b.P, st));
        ++it;
    }
    TSVD_TRY(project(X));
    *iters = it;
    *resid = worst;
    return worst <= o->cg_tol ? TSVD_OK : TSVD_NOT_CONVERGED;
}

}  // namespace

int svd_backward_run(tsvd_handle* h, const tsvd_matrix* A, int k, const double* sigma, const double* U,
                     const double* V, const double* sb, const double* Ub, const double* Vb, double* grad,
                     const tsvd_backward_opts* o, char* ws, size_t ws_bytes, size_t* sizing,
                     tsvd_backward_info* info) {
    const bool run = sizing == nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(o->stream);
    Arena ar{run ? ws : nullptr, ws_bytes, 0};
    int* status = ar.take<int>(kStCount);
    if (run) {
        if (!ar.fits()) return TSVD_ERR_WORKSPACE;
        TSVD_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * kStCount, st));
    }
    Timer* total = run ? new Timer(st) : nullptr;
    struct Del {
        Timer* t;
        ~Del() { delete t; }
    } del{total};
    Op<double> op;
    TSVD_TRY(setup_op<double>(h, A, k, ar, op, status, st, run, nullptr));
    const int64_t m = A->m, n = A->n, mx = std::max(m, n);
    const int kk = 2 * k;
    double* J = ar.take<double>((size_t)k * k);
    double* K = ar.take<double>((size_t)k * k);
    double* C = ar.take<double>((size_t)k * k);
    double* Y = ar.take<double>((size_t)m * k);
    double* Z = ar.take<double>((size_t)n * k);
    double* Lf = ar.take<double>((size_t)m * kk);
    double* Rf = ar.take<double>((size_t)n * kk);
    double* RfT = A->format == TSVD_CSR ? nullptr : ar.take<double>((size_t)n * kk);
    CgBufs b{};
    b.R = ar.take<double>((size_t)mx * k);
    b.P = ar.take<double>((size_t)mx * k);
    b.AP = ar.take<double>((size_t)mx * k);
    b.T = ar.take<double>((size_t)mx * k);
    b.H = ar.take<double>((size_t)k * k);
    for (double** v : {&b.rr, &b.rr_new, &b.pap, &b.bb, &b.alpha, &b.beta}) *v = ar.take<double>(k);
    b.part = ar.take<double>(tn_partial_max(h, mx, k, k) / sizeof(double) + 1);
    b.cpart = ar.take<double>(coldot_ws(mx, k) / sizeof(double) + 1);
    if (!run) {
        *sizing = ar.off + 256;
        return TSVD_OK;
    }
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    // products with A and A^T in the caller's orientation (op(A) may be A^T)
    auto amul = [&](const double* X, double* Yo, int64_t ldy) {
        return op.transposed ? op_tmul64(h, op, k, X, k, Yo, ldy, status, st) : op_mul64(h, op, k, X, k, Yo, ldy, status, st);
    };
    auto atmul = [&](const double* X, double* Yo, int64_t ldy) {
        return op.transposed ? op_mul64(h, op, k, X, k, Yo, ldy, status, st) : op_tmul64(h, op, k, X, k, Yo, ldy, status, st);
    };
    // inside span(U), span(V): C
    if (Ub) TSVD_TRY_CUDA((gemm_tn<double, double>(h, m, k, k, U, k, Ub, k, J, k, false, b.part, st)));
    if (Vb) TSVD_TRY_CUDA((gemm_tn<double, double>(h, n, k, k, V, k, Vb, k, K, k, false, b.part, st)));
    TSVD_TRY_CUDA(coupling(h, k, sigma, sb, Ub ? J : nullptr, Vb ? K : nullptr, C, st));
    // outside: complement solves
    int it_u = 0, it_v = 0;
    double res_u = 0.0, res_v = 0.0;
    int rc_u = TSVD_OK, rc_v = TSVD_OK;
    if (Ub) {
        rc_u = cg_side(h, m, k, U, Ub, sigma, [&](const double* X, double* T) { return atmul(X, T, k); },
                       [&](const double* X, double* T) { return amul(X, T, k); }, Y, o, b, st, &it_u, &res_u);
        TSVD_TRY(rc_u);
    } else {
        TSVD_TRY_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)m * k, st));
    }
    if (Vb) {
        rc_v = cg_side(h, n, k, V, Vb, sigma, [&](const double* X, double* T) { return amul(X, T, k); },
                       [&](const double* X, double* T) { return atmul(X, T, k); }, Z, o, b, st, &it_v, &res_v);
        TSVD_TRY(rc_v);
    } else {
        TSVD_TRY_CUDA(cudaMemsetAsync(Z, 0, sizeof(double) * (size_t)n * k, st));
    }
    // Lf = [A Z + U C + Y S, U],  Rf = [V, A^T Y + Z S]
    TSVD_TRY(amul(Z, Lf, kk));
    TSVD_TRY_CUDA((gemm_nn<double, double, double>(h, m, k, k, 1.0, U, k, C, k, 1.0, Lf, kk, false, st)));
    TSVD_TRY_CUDA(add_scaled_cols(h, m, k, Y, sigma, Lf, kk, st));
    TSVD_TRY_CUDA(copy_block<double>(U, k, Lf + k, kk, m, k, st));
    TSVD_TRY_CUDA(copy_block<double>(V, k, Rf, kk, n, k, st));
    TSVD_TRY(atmul(Y, Rf + k, kk));
    TSVD_TRY_CUDA(add_scaled_cols(h, n, k, Z, sigma, Rf + k, kk, st));
    if (A->format == TSVD_CSR) {
        TSVD_TRY_CUDA(sddmm(h, m, A->nnz, op.rp, op.ci, kk, Lf, kk, Rf, kk, grad, st));
    } else {
        TSVD_TRY_CUDA(put_transposed(h, (int)n, kk, Rf, kk, RfT, n, st));
        ProfClass pc(h, TSVD_K_APROD);
        TSVD_TRY_CUDA((gemm_nn<double, double, double>(h, m, kk, n, 1.0, Lf, kk, RfT, n, 0.0, grad, n, false, st)));
    }
    int hs[kStCount];
    TSVD_TRY(read_status(st, status, hs));
    TSVD_TRY(status_code(hs));
    const double ms = total->stop();
    if (info) {
        info->cg_iters_u = it_u;
        info->cg_iters_v = it_v;
        info->cg_resid_u = res_u;
        info->cg_resid_v = res_v;
        info->ms_total = ms;
    }
    return (rc_u == TSVD_OK && rc_v == TSVD_OK) ? TSVD_OK : TSVD_NOT_CONVERGED;
}

template int rsvd_run<double>(tsvd_handle*, const tsvd_matrix*, int, int, int, int, uint64_t, const tsvd_opts*,
                              char*, size_t, size_t*, double*, double*, double*, tsvd_info*);
template int rsvd_run<float>(tsvd_handle*, const tsvd_matrix*, int, int, int, int, uint64_t, const tsvd_opts*,
                             char*, size_t, size_t*, double*, double*, double*, tsvd_info*);
template int blanczos_run<double>(tsvd_handle*, const tsvd_matrix*, int, int, int, uint64_t, const tsvd_opts*,
                                  char*, size_t, size_t*, double*, double*, double*, tsvd_info*);
template int blanczos_run<float>(tsvd_handle*, const tsvd_matrix*, int, int, int, uint64_t, const tsvd_opts*,
                                 char*, size_t, size_t*, double*, double*, double*, tsvd_info*);

}  // namespace tsvd
