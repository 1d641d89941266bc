// Kernels of the gradient of a loss on the k leading singular triplets with
// respect to A (the differentiation pattern built on the paper's methods; the
// paper has no backward pass):
//   dL/dA = Lf Rf^T,  Lf = [U C + Y S + A Z, U],  Rf = [V, A^T Y + Z S],
// with C the k x k coupling inside span(U), span(V), and Y, Z the solutions of
// the shifted systems (s_i^2 I - A A^T) y_i = (I - U U^T) u_bar_i and
// (s_i^2 I - A^T A) z_i = (I - V V^T) v_bar_i on the complements, found by
// conjugate gradients with one right-hand side (and shift) per column.
//
// Column-wise reductions are two-stage with a fixed order (deterministic).  For
// sparse A the gradient is needed on A's pattern only: an SDDMM forms
// grad_e = Lf[row(e), :] . Rf[col(e), :] for every stored entry.
#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

constexpr int kColRows = 256;  // rows per partial sum of a column reduction

// partial[g][j] = sum over rows [g R, (g+1) R) of X[i][j] * Y[i][j]
__global__ void coldot_partial_kernel(int64_t rows, int k, const double* __restrict__ X, int64_t ldx,
                                      const double* __restrict__ Y, int64_t ldy, double* __restrict__ partial) {
    const int64_t r0 = (int64_t)blockIdx.x * kColRows;
    const int64_t r1 = min(rows, r0 + kColRows);
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double acc = 0.0;
        for (int64_t i = r0; i < r1; ++i) acc = fma(X[i * ldx + j], Y[i * ldy + j], acc);
        partial[(int64_t)blockIdx.x * k + j] = acc;
    }
}

__global__ void coldot_reduce_kernel(int k, int64_t groups, const double* __restrict__ partial,
                                     double* __restrict__ out) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double acc = 0.0;
        for (int64_t g = 0; g < groups; ++g) acc += partial[g * k + j];
        out[j] = acc;
    }
}

// Per-column CG scalars.  A column is frozen once rr <= tol^2 bb (or when its
// denominator vanishes): alpha = beta = 0 leave its iterate unchanged.
__global__ void cg_alpha_kernel(int k, const double* __restrict__ rr, const double* __restrict__ pap,
                                const double* __restrict__ bb, double tol2, double* __restrict__ alpha) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    const bool live = rr[j] > tol2 * bb[j] && pap[j] > 0.0;
    alpha[j] = live ? rr[j] / pap[j] : 0.0;
}

__global__ void cg_beta_kernel(int k, double* __restrict__ rr, const double* __restrict__ rr_new,
                               const double* __restrict__ alpha, double* __restrict__ beta) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    beta[j] = (alpha[j] != 0.0 && rr[j] > 0.0) ? rr_new[j] / rr[j] : 0.0;
    if (alpha[j] != 0.0) rr[j] = rr_new[j];
}

// x += alpha_j p, r -= alpha_j Ap
__global__ void cg_xr_kernel(int64_t rows, int k, const double* __restrict__ alpha, const double* __restrict__ p,
                             const double* __restrict__ Ap, double* __restrict__ x, double* __restrict__ r) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    const double a = alpha[idx % k];
    if (a == 0.0) return;
    x[idx] = fma(a, p[idx], x[idx]);
    r[idx] = fma(-a, Ap[idx], r[idx]);
}

// p = r + beta_j p (frozen columns keep p)
__global__ void cg_p_kernel(int64_t rows, int k, const double* __restrict__ alpha, const double* __restrict__ beta,
                            const double* __restrict__ r, double* __restrict__ p) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    if (alpha[idx % k] == 0.0) return;
    p[idx] = fma(beta[idx % k], p[idx], r[idx]);
}

// out = s_j^2 p - q
__global__ void shifted_kernel(int64_t rows, int k, const double* __restrict__ s, const double* __restrict__ p,
                               const double* __restrict__ q, double* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    const double sj = s[idx % k];
    out[idx] = fma(sj * sj, p[idx], -q[idx]);
}

// out[i][j] (ld ldo) += Y[i][j] s_j
__global__ void add_scaled_cols_kernel(int64_t rows, int k, const double* __restrict__ Y, const double* __restrict__ s,
                                       double* __restrict__ out, int64_t ldo) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    const int64_t i = idx / k;
    const int j = (int)(idx % k);
    out[i * ldo + j] = fma(Y[idx], s[j], out[i * ldo + j]);
}

// C = (F o (J - J^T)) S + diag(sb) + S (F o (K - K^T)),  F_ij = 1 / (s_j^2 - s_i^2), i != j
__global__ void coupling_kernel(int k, const double* __restrict__ s, const double* __restrict__ sb,
                                const double* __restrict__ J, const double* __restrict__ K, double* __restrict__ C) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= k * k) return;
    const int i = idx / k, j = idx % k;
    double c = 0.0;
    if (i == j) {
        c = sb ? sb[i] : 0.0;
    } else {
        const double f = 1.0 / (s[j] * s[j] - s[i] * s[i]);
        const double jj = J ? (J[i * k + j] - J[j * k + i]) : 0.0;
        const double kk = K ? (K[i * k + j] - K[j * k + i]) : 0.0;
        c = f * jj * s[j] + s[i] * f * kk;
    }
    C[idx] = c;
}

// grad_e = sum_t Lf[row][t] Rf[col(e)][t] for every stored entry; warp per row,
// each lane sums a strided share of the t terms, a shuffle tree adds the lanes.
__global__ void __launch_bounds__(256) sddmm_kernel(int64_t m, const int32_t* __restrict__ rp,
                                                    const int32_t* __restrict__ ci, int kk,
                                                    const double* __restrict__ Lf, int64_t ldl,
                                                    const double* __restrict__ Rf, int64_t ldr,
                                                    double* __restrict__ grad) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    constexpr int kMaxPerLane = 8;  // kk <= 256
    double l[kMaxPerLane];
#pragma unroll
    for (int q = 0; q < kMaxPerLane; ++q) {
        const int t = lane + 32 * q;
        l[q] = t < kk ? Lf[row * ldl + t] : 0.0;
    }
    const int64_t beg = rp[row], end = rp[row + 1];
    for (int64_t e = beg; e < end; ++e) {
        const double* rr = Rf + (int64_t)ci[e] * ldr;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < kMaxPerLane; ++q) {
            const int t = lane + 32 * q;
            if (t < kk) acc = fma(l[q], rr[t], acc);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) grad[e] = acc;
    }
}

}  // namespace

size_t coldot_ws(int64_t rows, int k) { return align256(sizeof(double) * (size_t)((rows + kColRows - 1) / kColRows + 1) * k); }

cudaError_t coldot(tsvd_handle* h, int64_t rows, int k, const double* X, int64_t ldx, const double* Y, int64_t ldy,
                   double* out, double* partial, cudaStream_t st) {
    const int64_t groups = rows > 0 ? (rows + kColRows - 1) / kColRows : 1;
    h->launches += 2;
    if (rows > 0) {
        coldot_partial_kernel<<<(unsigned)groups, 64, 0, st>>>(rows, k, X, ldx, Y, ldy, partial);
    } else {
        cudaError_t e = cudaMemsetAsync(partial, 0, sizeof(double) * k, st);
        if (e != cudaSuccess) return e;
    }
    coldot_reduce_kernel<<<1, 128, 0, st>>>(k, groups, partial, out);
    return cudaGetLastError();
}

cudaError_t cg_alpha(tsvd_handle* h, int k, const double* rr, const double* pap, const double* bb, double tol2,
                     double* alpha, cudaStream_t st) {
    h->launches++;
    cg_alpha_kernel<<<(k + 127) / 128, 128, 0, st>>>(k, rr, pap, bb, tol2, alpha);
    return cudaGetLastError();
}

cudaError_t cg_beta(tsvd_handle* h, int k, double* rr, const double* rr_new, const double* alpha, double* beta,
                    cudaStream_t st) {
    h->launches++;
    cg_beta_kernel<<<(k + 127) / 128, 128, 0, st>>>(k, rr, rr_new, alpha, beta);
    return cudaGetLastError();
}

static unsigned grid_of(int64_t n) { return (unsigned)((n + 255) / 256); }

cudaError_t cg_xr(tsvd_handle* h, int64_t rows, int k, const double* alpha, const double* p, const double* Ap,
                  double* x, double* r, cudaStream_t st) {
    if (rows * k == 0) return cudaSuccess;
    h->launches++;
    cg_xr_kernel<<<grid_of(rows * k), 256, 0, st>>>(rows, k, alpha, p, Ap, x, r);
    return cudaGetLastError();
}

cudaError_t cg_p(tsvd_handle* h, int64_t rows, int k, const double* alpha, const double* beta, const double* r,
                 double* p, cudaStream_t st) {
    if (rows * k == 0) return cudaSuccess;
    h->launches++;
    cg_p_kernel<<<grid_of(rows * k), 256, 0, st>>>(rows, k, alpha, beta, r, p);
    return cudaGetLastError();
}

cudaError_t shifted(tsvd_handle* h, int64_t rows, int k, const double* s, const double* p, const double* q,
                    double* out, cudaStream_t st) {
    if (rows * k == 0) return cudaSuccess;
    h->launches++;
    shifted_kernel<<<grid_of(rows * k), 256, 0, st>>>(rows, k, s, p, q, out);
    return cudaGetLastError();
}

cudaError_t add_scaled_cols(tsvd_handle* h, int64_t rows, int k, const double* Y, const double* s, double* out,
                            int64_t ldo, cudaStream_t st) {
    if (rows * k == 0) return cudaSuccess;
    h->launches++;
    add_scaled_cols_kernel<<<grid_of(rows * k), 256, 0, st>>>(rows, k, Y, s, out, ldo);
    return cudaGetLastError();
}

cudaError_t coupling(tsvd_handle* h, int k, const double* s, const double* sb, const double* J, const double* K,
                     double* C, cudaStream_t st) {
    h->launches++;
    coupling_kernel<<<(k * k + 127) / 128, 128, 0, st>>>(k, s, sb, J, K, C);
    return cudaGetLastError();
}

cudaError_t sddmm(tsvd_handle* h, int64_t m, int64_t nnz, const int32_t* rp, const int32_t* ci, int kk,
                  const double* Lf, int64_t ldl, const double* Rf, int64_t ldr, double* grad, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    if (kk > 256) return cudaErrorInvalidValue;
    h->launches++;
    // compulsory traffic: the pattern, Lf and the gradient once, one Rf row gathered per entry
    ProfScope prof(h, TSVD_K_APROD, 2.0 * kk * (double)nnz,
                   12.0 * nnz + 4.0 * (m + 1) + 8.0 * kk * (double)m + 8.0 * kk * (double)nnz, st);
    sddmm_kernel<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(m, rp, ci, kk, Lf, ldl, Rf, ldr, grad);
    return cudaGetLastError();
}

}  // namespace tsvd
