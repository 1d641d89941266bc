// Orthogonalisation building blocks on the device, ordered as in the paper:
//   CholeskyQR2 (Alg. 4, Sec. 3.2), CGS-CQR2 (Alg. 5, Sec. 3.3), CGS-QR (Alg. 3,
//   Sec. 3.1), and the fallback Sec. 3.2 prescribes when a Cholesky factorisation
//   breaks down: column-wise classical Gram-Schmidt with re-orthogonalisation.
//
// Differences from the paper's hybrid realisation (Table 1): POTRF, TRMM and the
// matrix addition run on the GPU (no host round trips for W, L, R), and the
// triangular solve Q L^{-T} is applied as a product with the explicitly inverted
// factor (same DFMA count, a product kernel instead of a solve).  The outputs
// follow the exact algebra: R = Lbar^T L^T and H = H + Hbar L^T.
//
// The routines are templated on the storage type T of the tall blocks: double for
// the FP64 method, float for the mixed-precision form, where the products read
// FP32 blocks but every Gram matrix, projection coefficient, Cholesky factor and R
// stays FP64 (split-K partial sums are reduced in FP64).  With FP32 blocks each
// update runs as one pass with the Gram matrix of its result (fused_cgs_cqr2_f32).
#include <cmath>
#include <type_traits>
#include <vector>

#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

__global__ void axpy_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}

// v[i*ld] = v[i*ld] / d[0]
template <typename T>
__global__ void scale_col_kernel(int64_t q, T* __restrict__ v, int64_t ld, const double* __restrict__ d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < q) v[i * ld] = (T)((double)v[i * ld] / d[0]);
}

template <typename T>
__global__ void d2t_kernel(int64_t n, const double* __restrict__ x, T* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (T)x[i];
}

__global__ void sqrt_kernel(double* __restrict__ x) { x[0] = sqrt(x[0]); }

// Writes column j of R (or of R^T when trans): R[i][j] = c[i] (i < j), R[j][j] = d.
__global__ void put_rcol_kernel(int j, const double* __restrict__ c, double d, double* __restrict__ R,
                                int64_t ldr, int trans) {
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double v = (i < j) ? c[i] : d;
        if (trans)
            R[(int64_t)j * ldr + i] = v;
        else
            R[(int64_t)i * ldr + j] = v;
    }
}

// Writes column j of H (s x b, ldh) from h[s].
__global__ void put_hcol_kernel(int64_t s, int j, const double* __restrict__ hcol, double* __restrict__ H,
                                int64_t ldh) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += (int64_t)gridDim.x * blockDim.x)
        H[i * ldh + j] = hcol[i];
}

template <typename T>
struct OrthWs {
    double *W, *Lt1, *Mt1, *Lt2, *Mt2, *H1, *H2, *partial;
    T *save, *fcol;
    double *fcol64, *fh, *fhacc, *fc, *fcacc, *fnrm;
};

template <typename T>
OrthWs<T> carve(tsvd_handle* h, Arena& ar, int64_t q, int64_t s, int b) {
    OrthWs<T> w{};
    const size_t bb = (size_t)b * b;
    w.W = ar.take<double>(bb);
    w.Lt1 = ar.take<double>(bb);
    w.Mt1 = ar.take<double>(bb);
    w.Lt2 = ar.take<double>(bb);
    w.Mt2 = ar.take<double>(bb);
    const size_t sb = (size_t)(s > 0 ? s : 1) * b;
    w.H1 = ar.take<double>(sb);
    w.H2 = ar.take<double>(sb);
    // split-K partial sums for every product shape used below (incl. the fallback's widths)
    const int eb = (int)sizeof(T);
    size_t pbytes = gemm_tn_ws(h, q, b, b, true, eb);
    auto upd = [&](size_t v) { if (v > pbytes) pbytes = v; };
    if (s > 0) {
        upd(gemm_tn_ws(h, q, s, b, false, eb));
        upd(gemm_tn_ws(h, q, s, 1, false, eb));
    }
    for (int j = 1; j <= b; ++j) upd(gemm_tn_ws(h, q, j, 1, false, eb));
    upd(gemm_tn_ws(h, q, 1, 1, true, eb));
    if (eb == 4) upd(update_gram_ws(q, b));
    w.partial = ar.take<double>(pbytes / sizeof(double) + 1);
    w.save = ar.take<T>((size_t)q * b);
    w.fcol = ar.take<T>((size_t)q);
    w.fcol64 = ar.take<double>((size_t)q);
    w.fh = ar.take<double>((size_t)(s > 0 ? s : 1));
    w.fhacc = ar.take<double>((size_t)(s > 0 ? s : 1));
    w.fc = ar.take<double>((size_t)b);
    w.fcacc = ar.take<double>((size_t)b);
    w.fnrm = ar.take<double>(2);
    return w;
}

// One CholeskyQR step (Alg. 4 S1-S3): W = Y^T Y, W = L L^T, Y <- Y L^{-T}.  With a
// row partition, W is the sum of the processes' Gram matrices (the communication-
// avoiding property of Sec. 3.2: one b x b reduction per step).
template <typename T>
int cholqr_step(tsvd_handle* h, int64_t q, int b, T* Y, int64_t ldy, double* W, double* Lt, double* Mt,
                double* partial, int* status, const OrthCtx& ctx, cudaStream_t st) {
    TSVD_TRY_CUDA(gemm_tn(h, q, b, b, Y, ldy, Y, ldy, W, b, true, partial, st));
    if (ctx.reduce) TSVD_TRY(part_sum(h, W, b, b, b, st));
    TSVD_TRY_CUDA(chol_inv(h, b, W, Lt, Mt, status, st));
    TSVD_TRY_CUDA(gemm_nn(h, q, b, b, 1.0, Y, ldy, Mt, b, 0.0, Y, ldy, true, st));
    return TSVD_OK;
}

// CGS-CQR2 (Alg. 5) on FP32 blocks with the fused update + Gram pass: per CGS
// pass, the projection H = P^T Y is its own pass (split-K over the rows), then one
// pass forms Y - P H and the Gram matrix of the result, whose Cholesky factor
// normalises the block.  Without P (s = 0: CholeskyQR2, Alg. 4) the first step's
// Y L^{-T} is fused with the second step's Gram matrix instead.
//
// The second projection is not folded into the first pass (P^T of the unnormalised
// Y - P H, then multiplied by L^{-T}): that product misses the rounding committed
// when Y L^{-T} is formed, which is of order eps cond(Y - P H), so the result would be
// orthogonal to P only to that level instead of to eps.  Alg. 5 projects the
// normalised block, and so does this sequence.
template <typename T>
int fused_cgs_cqr2_f32(tsvd_handle* h, int64_t q, int64_t s, int b, const T* P, int64_t ldp, T* Y, int64_t ldy,
                       OrthWs<T>& w, int* status, const OrthCtx& ctx, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        if (s > 0) {
            TSVD_TRY_CUDA(gemm_tn(h, q, s, b, P, ldp, Y, ldy, w.H1, b, false, w.partial, st));        // S1
            if (ctx.reduce) TSVD_TRY(part_sum(h, w.H1, s, b, b, st));
            TSVD_TRY_CUDA(update_gram(h, q, s, b, -1.0, P, ldp, w.H1, b, 1.0, Y, ldy, false, w.W, w.partial,
                                      st));                                                             // S2, S3
            if (ctx.reduce) TSVD_TRY(part_sum(h, w.W, b, b, b, st));
            TSVD_TRY_CUDA(chol_inv(h, b, w.W, w.Lt1, w.Mt1, status, st));                              // S4
            TSVD_TRY_CUDA(gemm_nn(h, q, b, b, 1.0, Y, ldy, w.Mt1, b, 0.0, Y, ldy, true, st));          // S5
            TSVD_TRY_CUDA(gemm_tn(h, q, s, b, P, ldp, Y, ldy, w.H2, b, false, w.partial, st));        // S6
            if (ctx.reduce) TSVD_TRY(part_sum(h, w.H2, s, b, b, st));
            TSVD_TRY_CUDA(update_gram(h, q, s, b, -1.0, P, ldp, w.H2, b, 1.0, Y, ldy, false, w.W, w.partial,
                                      st));                                                             // S7, S8
        } else {
            TSVD_TRY_CUDA(gemm_tn(h, q, b, b, Y, ldy, Y, ldy, w.W, b, true, w.partial, st));          // S3
            if (ctx.reduce) TSVD_TRY(part_sum(h, w.W, b, b, b, st));
            TSVD_TRY_CUDA(chol_inv(h, b, w.W, w.Lt1, w.Mt1, status, st));                              // S4
            TSVD_TRY_CUDA(update_gram(h, q, b, b, 1.0, Y, ldy, w.Mt1, b, 0.0, Y, ldy, true, w.W, w.partial,
                                      st));                                                             // S5, S8
        }
        if (ctx.reduce) TSVD_TRY(part_sum(h, w.W, b, b, b, st));
        TSVD_TRY_CUDA(chol_inv(h, b, w.W, w.Lt2, w.Mt2, status, st));                                  // S9
        TSVD_TRY_CUDA(gemm_nn(h, q, b, b, 1.0, Y, ldy, w.Mt2, b, 0.0, Y, ldy, true, st));              // S10
        return TSVD_OK;
    } else {
        return TSVD_ERR_UNSUPPORTED;
    }
}

// v -= [P, Yprev] ([P, Yprev]^T v), twice; accumulating coefficients when asked.
template <typename T>
int project_twice(tsvd_handle* h, int64_t q, int64_t s, const T* P, int64_t ldp, int j, const T* Yprev,
                  int64_t ldy, T* v, int64_t ldv, OrthWs<T>& w, bool accumulate, const OrthCtx& ctx,
                  cudaStream_t st) {
    for (int pass = 0; pass < 2; ++pass) {
        if (s > 0) {
            TSVD_TRY_CUDA(gemm_tn(h, q, s, 1, P, ldp, v, ldv, w.fh, 1, false, w.partial, st));
            if (ctx.reduce) TSVD_TRY(part_sum(h, w.fh, s, 1, 1, st));
            TSVD_TRY_CUDA(gemm_nn(h, q, s, 1, -1.0, P, ldp, w.fh, 1, 1.0, v, ldv, false, st));
            if (accumulate) {
                h->launches++;
                axpy_kernel<<<(unsigned)((s + 255) / 256), 256, 0, st>>>(s, w.fh, w.fhacc);
            }
        }
        if (j > 0) {
            TSVD_TRY_CUDA(gemm_tn(h, q, j, 1, Yprev, ldy, v, ldv, w.fc, 1, false, w.partial, st));
            if (ctx.reduce) TSVD_TRY(part_sum(h, w.fc, j, 1, 1, st));
            TSVD_TRY_CUDA(gemm_nn(h, q, j, 1, -1.0, Yprev, ldy, w.fc, 1, 1.0, v, ldv, false, st));
            if (accumulate) {
                h->launches++;
                axpy_kernel<<<1, 256, 0, st>>>(j, w.fc, w.fcacc);
            }
        }
        TSVD_TRY_CUDA(cudaGetLastError());
    }
    return TSVD_OK;
}

template <typename T>
int read_norm(tsvd_handle* h, int64_t q, const T* v, int64_t ldv, OrthWs<T>& w, double* out, const OrthCtx& ctx,
              cudaStream_t st) {
    TSVD_TRY_CUDA(gemm_tn(h, q, 1, 1, v, ldv, v, ldv, w.fnrm, 1, true, w.partial, st));
    if (ctx.reduce) TSVD_TRY(part_sum(h, w.fnrm, 1, 1, 1, st));
    h->launches++;
    sqrt_kernel<<<1, 1, 0, st>>>(w.fnrm);
    TSVD_TRY_CUDA(cudaGetLastError());
    TSVD_TRY_CUDA(cudaMemcpyAsync(out, w.fnrm, sizeof(double), cudaMemcpyDeviceToHost, st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}

// Column-wise CGS with re-orthogonalisation (fallback of Sec. 3.2):
// Y_in = P H + Q R, P^T Q = 0, Q^T Q = I; numerically dependent columns get Philox replacements.
template <typename T>
int cgs2_columns(tsvd_handle* h, int64_t q, int64_t s, int b, const T* P, int64_t ldp, T* Y, int64_t ldy,
                 double* H, int64_t ldh, double* R, int64_t ldr, bool r_trans, OrthCtx& ctx, OrthWs<T>& w,
                 cudaStream_t st) {
    for (int j = 0; j < b; ++j) {
        T* v = Y + j;
        double nrm0 = 0.0, nrm = 0.0;
        TSVD_TRY(read_norm(h, q, v, ldy, w, &nrm0, ctx, st));
        if (s > 0) TSVD_TRY_CUDA(cudaMemsetAsync(w.fhacc, 0, sizeof(double) * s, st));
        TSVD_TRY_CUDA(cudaMemsetAsync(w.fcacc, 0, sizeof(double) * b, st));
        TSVD_TRY(project_twice(h, q, s, P, ldp, j, Y, ldy, v, ldy, w, true, ctx, st));
        TSVD_TRY(read_norm(h, q, v, ldy, w, &nrm, ctx, st));
        if (!std::isfinite(nrm0) || !std::isfinite(nrm)) return TSVD_ERR_NONFINITE;
        h->launches++;
        put_rcol_kernel<<<1, 128, 0, st>>>(j, w.fcacc, nrm, R, ldr, r_trans ? 1 : 0);
        if (H != nullptr && s > 0) {
            h->launches++;
            put_hcol_kernel<<<(unsigned)((s + 255) / 256 < 1024 ? (s + 255) / 256 : 1024), 256, 0, st>>>(
                s, j, w.fhacc, H, ldh);
        }
        TSVD_TRY_CUDA(cudaGetLastError());
        if (!(nrm > 1e-10 * nrm0) || nrm0 == 0.0) {
            // dependent column: replace its direction by a Philox N(0,1) column
            TSVD_TRY_CUDA(gaussian(h, q, 1, ctx.seed, 0x100u + (uint32_t)ctx.replacements, w.fcol64, 1, st, ctx.row0));
            ctx.replacements++;
            h->launches++;
            d2t_kernel<T><<<(unsigned)((q + 255) / 256), 256, 0, st>>>(q, w.fcol64, w.fcol);
            TSVD_TRY(project_twice(h, q, s, P, ldp, j, Y, ldy, w.fcol, 1, w, false, ctx, st));
            double zn = 0.0;
            TSVD_TRY(read_norm(h, q, w.fcol, 1, w, &zn, ctx, st));
            if (!(zn > 0.0) || !std::isfinite(zn)) return TSVD_ERR_NONFINITE;
            TSVD_TRY_CUDA(copy_block(w.fcol, 1, v, ldy, q, 1, st));
        }
        h->launches++;
        scale_col_kernel<T><<<(unsigned)((q + 255) / 256), 256, 0, st>>>(q, v, ldy, w.fnrm);
        TSVD_TRY_CUDA(cudaGetLastError());
    }
    return TSVD_OK;
}

}  // namespace

int read_status(cudaStream_t st, const int* d_status, int* h_status) {
    TSVD_TRY_CUDA(cudaMemcpyAsync(h_status, d_status, sizeof(int) * kStCount, cudaMemcpyDeviceToHost, st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}

// Covers both block types: FP32 blocks take half the copies but a wider split-K
// plan and the fused update + Gram partials.
size_t orth_ws(tsvd_handle* h, int64_t q, int64_t s, int b) {
    Arena a64, a32;
    carve<double>(h, a64, q, s, b);
    carve<float>(h, a32, q, s, b);
    return a64.off > a32.off ? a64.off : a32.off;
}

template <typename T>
int cgs_cqr2(tsvd_handle* h, int64_t q, int64_t s, int b, const T* P, int64_t ldp, T* Y, int64_t ldy,
             double* H, double* R, int64_t ldr, bool r_trans, OrthCtx& ctx, Arena ar, int* status,
             cudaStream_t st) {
    if (b < 1 || b > TSVD_MAX_BLOCK || q < b) return TSVD_ERR_INVALID_ARG;
    OrthWs<T> w = carve<T>(h, ar, q, s, b);
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    TSVD_TRY_CUDA(copy_block(Y, ldy, w.save, b, q, b, st));
    if constexpr (std::is_same<T, float>::value) {
        // FP32 blocks: each update is fused with the Gram matrix of its result (one
        // pass over the rows; update_gram).  The projections stay separate passes: the
        // second one must see the normalised block (see fused_cgs_cqr2_f32).
        TSVD_TRY(fused_cgs_cqr2_f32(h, q, s, b, P, ldp, Y, ldy, w, status, ctx, st));
    } else {
        if (s > 0) {
            TSVD_TRY_CUDA(gemm_tn(h, q, s, b, P, ldp, Y, ldy, w.H1, b, false, w.partial, st));       // S1
            if (ctx.reduce) TSVD_TRY(part_sum(h, w.H1, s, b, b, st));
            TSVD_TRY_CUDA(gemm_nn(h, q, s, b, -1.0, P, ldp, w.H1, b, 1.0, Y, ldy, false, st));       // S2
        }
        TSVD_TRY(cholqr_step(h, q, b, Y, ldy, w.W, w.Lt1, w.Mt1, w.partial, status, ctx, st));  // S3-S5
        if (s > 0) {
            TSVD_TRY_CUDA(gemm_tn(h, q, s, b, P, ldp, Y, ldy, w.H2, b, false, w.partial, st));       // S6
            if (ctx.reduce) TSVD_TRY(part_sum(h, w.H2, s, b, b, st));
            TSVD_TRY_CUDA(gemm_nn(h, q, s, b, -1.0, P, ldp, w.H2, b, 1.0, Y, ldy, false, st));       // S7
        }
        TSVD_TRY(cholqr_step(h, q, b, Y, ldy, w.W, w.Lt2, w.Mt2, w.partial, status, ctx, st));  // S8-S10
    }
    TSVD_TRY_CUDA(trmm_upper(h, b, w.Lt2, w.Lt1, R, ldr, r_trans, st));                         // S11
    if (H != nullptr && s > 0) {                                                                 // S12
        TSVD_TRY_CUDA(copy_block(w.H1, b, H, b, s, b, st));
        TSVD_TRY_CUDA(gemm_nn(h, s, b, b, 1.0, w.H2, b, w.Lt1, b, 1.0, H, b, true, st));
    }
    if (ctx.deferred) return TSVD_OK;
    int hs[kStCount];
    TSVD_TRY(read_status(st, status, hs));
    if (hs[kStNonfinite]) return TSVD_ERR_NONFINITE;
    if (hs[kStBreakdown]) {
        TSVD_TRY_CUDA(cudaMemsetAsync(status + kStBreakdown, 0, sizeof(int), st));
        TSVD_TRY_CUDA(copy_block(w.save, b, Y, ldy, q, b, st));
        ctx.fallbacks++;
        for (int64_t i = 0; i < b; ++i) TSVD_TRY_CUDA(cudaMemsetAsync(R + i * ldr, 0, sizeof(double) * b, st));
        TSVD_TRY(cgs2_columns(h, q, s, b, P, ldp, Y, ldy, H, b, R, ldr, r_trans, ctx, w, st));
    }
    return TSVD_OK;
}

template <typename T>
int cgs_qr(tsvd_handle* h, int64_t q, int r, int b, T* Y, int64_t ldy, double* R, OrthCtx& ctx, Arena ar,
           int* status, cudaStream_t st) {
    if (b < 1) return TSVD_ERR_INVALID_ARG;
    if (b > r) b = r;
    TSVD_TRY_CUDA(cudaMemsetAsync(R, 0, sizeof(double) * (size_t)r * r, st));
    // S1: first block by CholeskyQR2; its R goes to R[0:b, 0:b]
    TSVD_TRY(cgs_cqr2<T>(h, q, 0, b, nullptr, 0, Y, ldy, nullptr, R, r, false, ctx, ar, status, st));
    for (int c0 = b; c0 < r; c0 += b) {  // S2: later blocks against the earlier ones
        const int c1 = c0 + b < r ? c0 + b : r;
        const int bw = c1 - c0;
        // H_j lands in R[0:c0, c0:c1]; it is produced in a packed s x bw buffer first.
        Arena sub = ar;
        double* Hp = sub.take<double>((size_t)c0 * bw);
        if (!sub.fits()) return TSVD_ERR_WORKSPACE;
        TSVD_TRY(cgs_cqr2<T>(h, q, c0, bw, Y, ldy, Y + c0, ldy, Hp, R + (int64_t)c0 * r + c0, r, false, ctx, sub,
                             status, st));
        TSVD_TRY_CUDA(copy_block(Hp, bw, R + c0, r, c0, bw, st));
    }
    return TSVD_OK;
}

template int cgs_cqr2<double>(tsvd_handle*, int64_t, int64_t, int, const double*, int64_t, double*, int64_t,
                              double*, double*, int64_t, bool, OrthCtx&, Arena, int*, cudaStream_t);
template int cgs_cqr2<float>(tsvd_handle*, int64_t, int64_t, int, const float*, int64_t, float*, int64_t, double*,
                             double*, int64_t, bool, OrthCtx&, Arena, int*, cudaStream_t);
template int cgs_qr<double>(tsvd_handle*, int64_t, int, int, double*, int64_t, double*, OrthCtx&, Arena, int*,
                            cudaStream_t);
template int cgs_qr<float>(tsvd_handle*, int64_t, int, int, float*, int64_t, double*, OrthCtx&, Arena, int*,
                           cudaStream_t);

}  // namespace tsvd
