// Dense FP64 kernels of the orthogonalisation building blocks (Table 1):
//   gemm_tn   C = X^T Z        Gram W = Q^T Q (Alg. 4 S1/S4, Alg. 5 S3/S8),
//                              projection H = P^T Q (Alg. 5 S1/S6), A^T X for dense A;
//   gemm_nn   Y = b Y + a X M  update Q - P H (Alg. 5 S2/S7), TRSM applied as the
//                              product with L^{-T} (Alg. 4 S3/S6, Alg. 5 S5/S10),
//                              Ritz/restart products (Alg. 1 S6/S7, Alg. 2 S7-S9), A X;
//   chol_inv  W = L L^T and L^{-T} of the b x b Gram matrix (POTRF of Table 1; one
//             CTA, or a cluster of 8 CTAs for b >= 64);
//   trmm      R = Lbar^T L^T (Alg. 4 S7, Alg. 5 S11);
// plus the Philox/Box-Muller start block, residual column norms, the Lanczos
// residual estimate and the output sign convention.
//
// On GB300 the FP64 pipe issues 2 DFMA/clk/SM (about 1.2 TFLOP/s for the chip),
// which puts every one of these products far above the FP64 ridge point: the
// design goal is the minimum number of DFMAs spread over all SMs, not memory
// traffic.  Symmetric Gram matrices compute only their upper half, triangular
// factors skip their zero half at warp granularity, and split-K partial sums
// are reduced in a fixed order so results are bitwise reproducible.
#include <cooperative_groups.h>

#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

// ---------------------------------------------------------------------------
// gemm_tn: CTA = 4 warps computes a 32 x 32 region of C over one row slab.
// Warp (wr, wc) owns a 16 x 16 sub-tile; lane owns C[i][jg .. jg+7].
// ---------------------------------------------------------------------------
constexpr int kTnR = 32;
constexpr int kTnKc = 32;

__device__ inline void decode_upper(int lin, int nr, int& ri, int& rj) {
    int r = 0;
    while (lin >= nr - r) {
        lin -= nr - r;
        ++r;
    }
    ri = r;
    rj = r + lin;
}

// TI: input element type (also the accumulation type within a slab); TW: type written.
template <typename TI, typename TW>
__global__ void __launch_bounds__(128) gemm_tn_kernel(int64_t q, int64_t s, int64_t b,
                                                      const TI* __restrict__ X, int64_t ldx,
                                                      const TI* __restrict__ Z, int64_t ldz,
                                                      TW* __restrict__ out, int64_t ldo,
                                                      int64_t slab_stride, int64_t slab_rows, int symmetric,
                                                      int nreg_s, int nreg_b) {
    __shared__ TI Xs[kTnKc][kTnR];
    __shared__ TI Zs[kTnKc][kTnR];
    int ri, rj;
    if (symmetric) {
        decode_upper((int)blockIdx.x, nreg_s, ri, rj);
    } else {
        ri = (int)blockIdx.x / nreg_b;
        rj = (int)blockIdx.x % nreg_b;
    }
    const int64_t r0 = (int64_t)blockIdx.y * slab_rows;
    const int64_t r1 = min(q, r0 + slab_rows);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wr = warp >> 1, wc = warp & 1;
    const int i = lane >> 1, jg = (lane & 1) * 8;
    const bool active = !(symmetric && ri == rj && wr > wc);
    TI acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = TI(0);
    const int64_t xc0 = (int64_t)ri * kTnR, zc0 = (int64_t)rj * kTnR;
    for (int64_t k0 = r0; k0 < r1; k0 += kTnKc) {
        for (int idx = tid; idx < kTnKc * kTnR; idx += 128) {
            const int rr = idx / kTnR, cc = idx % kTnR;
            const int64_t row = k0 + rr;
            const bool rin = row < r1;
            Xs[rr][cc] = (rin && xc0 + cc < s) ? X[row * ldx + xc0 + cc] : TI(0);
            Zs[rr][cc] = (rin && zc0 + cc < b) ? Z[row * ldz + zc0 + cc] : TI(0);
        }
        __syncthreads();
        if (active) {
#pragma unroll 4
            for (int kk = 0; kk < kTnKc; ++kk) {
                const TI x = Xs[kk][wr * 16 + i];
                const TI* zr = &Zs[kk][wc * 16 + jg];
#pragma unroll
                for (int t = 0; t < 8; ++t) acc[t] = fma(x, zr[t], acc[t]);
            }
        }
        __syncthreads();
    }
    if (!active) return;
    const int64_t orow = xc0 + wr * 16 + i;
    if (orow >= s) return;
    TW* o = out + (int64_t)blockIdx.y * slab_stride + orow * ldo + zc0 + wc * 16 + jg;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        if (zc0 + wc * 16 + jg + t < b) o[t] = (TW)acc[t];
    }
}

// C[i][j] = sum over slabs of partial[slab][i][j] in a fixed order: thread
// (x, y) of a 32 x 8 block sums slabs y, y + 8, ... of element x, then the 8
// partial sums are added in y order.  Symmetric reads the upper element for both
// halves.
template <typename TC>
__global__ void __launch_bounds__(256) gemm_tn_reduce_kernel(int64_t s, int64_t b, int slabs,
                                                             const double* __restrict__ partial, int64_t slab_stride,
                                                             TC* __restrict__ C, int64_t ldc, int symmetric) {
    __shared__ double red[8][33];
    const int64_t idx = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const bool in = idx < s * b;
    int64_t i = 0, j = 0, src = 0;
    if (in) {
        i = idx / b;
        j = idx % b;
        const int64_t ii = (symmetric && i > j) ? j : i;
        const int64_t jj = (symmetric && i > j) ? i : j;
        src = ii * b + jj;
    }
    double acc = 0.0;
    if (in)
        for (int sl = threadIdx.y; sl < slabs; sl += 8) acc += partial[(int64_t)sl * slab_stride + src];
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && in) {
        double t = red[0][threadIdx.x];
#pragma unroll
        for (int y = 1; y < 8; ++y) t += red[y][threadIdx.x];
        C[i * ldc + j] = (TC)t;
    }
}

struct TnPlan {
    int nreg_s, nreg_b, regions, slabs;
    int64_t slab_rows;
};

// One full wave of the kernel on a 152-SM GB300: 7 resident CTAs per SM for the
// FP64 kernel (its 72 registers x 128 threads and 16 KB of shared memory allow 7),
// 16 for the 64-thread FP32 kernel (bounded to 64 registers, which it fits without
// spilling).  Splitting K so that regions x slabs fills
// exactly one wave keeps every SM equally busy; a fixed target (rather than the
// device's SM count) keeps the split, the workspace size and the summation order
// independent of the device.
constexpr int64_t kTnWave = 152 * 7;
constexpr int64_t kTnWaveF32 = 152 * 16;

TnPlan tn_plan(int64_t q, int64_t s, int64_t b, bool symmetric, int elem_bytes) {
    TnPlan p;
    p.nreg_s = (int)((s + kTnR - 1) / kTnR);
    p.nreg_b = (int)((b + kTnR - 1) / kTnR);
    p.regions = symmetric ? p.nreg_s * (p.nreg_s + 1) / 2 : p.nreg_s * p.nreg_b;
    int64_t slabs = (elem_bytes == 4 ? kTnWaveF32 : kTnWave) / p.regions;
    const int64_t max_slabs = (q + 255) / 256;
    if (slabs > max_slabs) slabs = max_slabs;
    if (slabs > 65535) slabs = 65535;
    if (slabs < 1) slabs = 1;
    int64_t rows = (q + slabs - 1) / slabs;
    rows = (rows + kTnKc - 1) / kTnKc * kTnKc;
    if (rows < kTnKc) rows = kTnKc;
    p.slab_rows = rows;
    p.slabs = (int)((q + rows - 1) / rows);
    if (p.slabs < 1) p.slabs = 1;
    return p;
}

// ---------------------------------------------------------------------------
// gemm_nn: CTA = 4 warps, 32 rows; lane = row, warp w owns CW columns of the
// current panel (4*CW columns).  X tile and M chunk staged in shared memory,
// output staged for coalesced stores.
// ---------------------------------------------------------------------------
// Accumulation in TX (the precision of the tall operand); M is converted to TX on load.
template <int CW, typename TX, typename TM, typename TY>
__global__ void __launch_bounds__(128) gemm_nn_kernel(int64_t q, int64_t s, int64_t b, double alpha,
                                                      const TX* __restrict__ X, int64_t ldx,
                                                      const TM* __restrict__ M, int64_t ldm, double beta,
                                                      TY* Y, int64_t ldy, int upper) {
    constexpr int PW = 4 * CW;
    __shared__ TX Xs[32][33];
    __shared__ TX Ms[32][PW + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    for (int64_t c0 = 0; c0 < b; c0 += PW) {
        TX acc[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) acc[c] = TX(0);
        const int64_t jw_hi = c0 + (int64_t)(warp + 1) * CW - 1;  // last column of this warp
        int64_t kmax = s;
        if (upper) kmax = min(s, c0 + PW);
        for (int64_t k0 = 0; k0 < kmax; k0 += 32) {
            for (int idx = tid; idx < 32 * 32; idx += 128) {
                const int rr = idx >> 5, kk = idx & 31;
                const int64_t row = r0 + rr, k = k0 + kk;
                Xs[rr][kk] = (row < q && k < s) ? X[row * ldx + k] : TX(0);
            }
            for (int idx = tid; idx < 32 * PW; idx += 128) {
                const int kk = idx / PW, cc = idx % PW;
                const int64_t k = k0 + kk, col = c0 + cc;
                const bool in = k < s && col < b && !(upper && k > col);
                Ms[kk][cc] = in ? (TX)M[k * ldm + col] : TX(0);
            }
            __syncthreads();
            if (!(upper && k0 > jw_hi)) {
#pragma unroll 4
                for (int kk = 0; kk < 32; ++kk) {
                    const TX x = Xs[lane][kk];
                    const TX* mr = &Ms[kk][warp * CW];
#pragma unroll
                    for (int c = 0; c < CW; ++c) acc[c] = fma(x, mr[c], acc[c]);
                }
            }
            __syncthreads();
        }
        // stage through shared memory (reusing Ms) for coalesced stores
#pragma unroll
        for (int c = 0; c < CW; ++c) Ms[lane][warp * CW + c] = acc[c];
        __syncthreads();
        for (int idx = tid; idx < 32 * PW; idx += 128) {
            const int rr = idx / PW, cc = idx % PW;
            const int64_t row = r0 + rr, col = c0 + cc;
            if (row < q && col < b) {
                TY* y = Y + row * ldy + col;
                const TX v = (TX)alpha * Ms[rr][cc];
                *y = (beta != 0.0) ? (TY)fma((TX)beta, (TX)*y, v) : (TY)v;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// chol_inv: one CTA of 256 threads.  Right-looking Cholesky of the lower triangle
// in shared memory (breakdown test d <= b*eps*max_i W_ii), then L^{-1} by
// right-looking forward substitution, stored transposed in the upper triangle of
// the same array (row k of L^{-1} is final once scaled; the rows below it take
// a rank-1 update).  GB300's FP64 pipe costs a warp instruction 16 cycles
// whatever its active lanes, so every FP64 phase is a flat loop over whole
// warps of independent elements (no per-thread chains of varying length), and
// the one scalar step per column (1/sqrt of the pivot) is an FP32 estimate with
// two FP64 Newton steps.
// ---------------------------------------------------------------------------
__device__ inline void tri_decode(int idx, int& ii, int& kk) {
    int r = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
    while (r * (r + 1) / 2 > idx) --r;
    while ((r + 1) * (r + 2) / 2 <= idx) ++r;
    ii = r;
    kk = idx - r * (r + 1) / 2;
}

// 1/sqrt(d) for finite d > 0: FP32 estimate of the scaled value, two Newton steps
// y <- y (3 - d y^2) / 2 in FP64 (24 -> 48 -> beyond 53 bits), rescaled.
__device__ inline double rsqrt_fp64(double d) {
    const int e = ilogb(d) & ~1;  // even exponent: d = dd 2^e, dd in [1, 4)
    const double dd = scalbn(d, -e);
    double y = (double)rsqrtf((float)dd);
    y = y * fma(-0.5 * dd, y * y, 1.5);
    y = y * fma(-0.5 * dd, y * y, 1.5);
    return scalbn(y, -e / 2);
}

__global__ void __launch_bounds__(256) chol_inv_kernel(int b, const double* __restrict__ W, double* __restrict__ Lt,
                                                       double* __restrict__ Mt, int* status) {
    extern __shared__ double sm[];
    const int ld = b + 1;
    double* A = sm;                    // lower: L; upper (transposed): L^{-1}
    double* dinv = sm + (size_t)b * ld; // 1 / L_jj
    __shared__ double s_thresh;
    __shared__ int s_bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int idx = tid; idx < b * b; idx += nt) {
        const int i = idx / b, j = idx % b;
        A[i * ld + j] = (j <= i) ? W[idx] : 0.0;  // the upper part starts as zero (L^{-1} = I - ...)
    }
    __syncthreads();
    if (tid == 0) {
        double wmax = 0.0;
        int bad = 0;
        for (int i = 0; i < b; ++i) {
            const double d = A[i * ld + i];
            if (!isfinite(d)) bad = 2;
            if (d > wmax) wmax = d;
        }
        if (bad == 0 && !(wmax > 0.0)) bad = 1;
        s_bad = bad;
        s_thresh = (double)b * kEps * wmax;
    }
    __syncthreads();
    for (int j = 0; j < b && s_bad == 0; ++j) {
        if (tid == 0) {
            const double d = A[j * ld + j];
            if (!isfinite(d) || !(d > s_thresh)) {
                s_bad = isfinite(d) ? 1 : 2;
            } else {
                const double y = rsqrt_fp64(d);
                A[j * ld + j] = d * y;  // L_jj
                dinv[j] = y;
            }
        }
        __syncthreads();
        if (s_bad) break;
        const double inv = dinv[j];
        for (int i = j + 1 + tid; i < b; i += nt) A[i * ld + j] *= inv;
        __syncthreads();
        const int nn = b - j - 1;
        const int cnt = nn * (nn + 1) / 2;
        for (int idx = tid; idx < cnt; idx += nt) {
            int ii, kk;
            tri_decode(idx, ii, kk);
            const int i = j + 1 + ii, k = j + 1 + kk;
            A[i * ld + k] = fma(-A[i * ld + j], A[k * ld + j], A[i * ld + k]);
        }
        __syncthreads();
    }
    if (s_bad) {
        if (tid == 0) atomicOr(&status[s_bad == 2 ? kStNonfinite : kStBreakdown], 1);
        for (int idx = tid; idx < b * b; idx += nt) {
            const double v = (idx / b == idx % b) ? 1.0 : 0.0;
            Lt[idx] = v;
            Mt[idx] = v;
        }
        return;
    }
    // X = L^{-1}: for k = 0..b-1, row k of X (columns c <= k) is scaled by 1/L_kk and
    // is then final; rows i > k take X[i][c] -= L[i][k] X[k][c].  X[i][c] (c < i) is
    // held at A[c][i]; the diagonal of X is dinv.
    for (int k = 0; k < b; ++k) {
        const double ik = dinv[k];
        for (int c = tid; c < k; c += nt) A[c * ld + k] *= ik;
        __syncthreads();
        const int rows = b - k - 1, cols = k + 1;
        for (int idx = tid; idx < rows * cols; idx += nt) {
            const int i = k + 1 + idx / cols, c = idx % cols;
            const double xkc = (c == k) ? ik : A[c * ld + k];
            A[c * ld + i] = fma(-A[i * ld + k], xkc, A[c * ld + i]);
        }
        __syncthreads();
    }
    // Lt = L^T and Mt = L^{-T} = X^T, both upper
    for (int idx = tid; idx < b * b; idx += nt) {
        const int i = idx / b, j = idx % b;
        Lt[idx] = (j >= i) ? A[j * ld + i] : 0.0;
        Mt[idx] = (j > i) ? A[i * ld + j] : (j == i ? dinv[i] : 0.0);
    }
}

// ---------------------------------------------------------------------------
// chol_inv on a cluster of kCholCluster CTAs (b >= kCholClusterMin): the same
// factorisation and inverse with the FP64 work spread over 8 SMs (one SM's FP64
// pipe, 2 DFMA/clk, bounds the single-CTA kernel above).  Every CTA keeps a full
// b x b copy in its shared memory; row i belongs to CTA i mod 8.  Per panel of 16
// columns:
//   1. every CTA factors the 16 x 16 diagonal block (warp 0; the same numbers and
//      code in every CTA, so every CTA takes the same breakdown decision);
//   2. each CTA solves its rows of the panel, L[i][P] = A[i][P] L11^{-T}, and writes
//      them into every CTA's copy (distributed shared memory); cluster barrier;
//   3. each CTA applies the rank-16 update A[i][k] -= L[i][P] L[k][P]^T to its rows
//      (k <= i), then writes its rows of the next diagonal block into every copy;
//      cluster barrier.
// Afterwards every copy holds all of L; the inverse is split by columns (column c of
// L^{-1} on CTA c mod 8, no exchange), and each CTA writes its rows of Lt and Mt.
// The trailing updates sum 16 products per panel before subtracting (the one-CTA
// kernel subtracts them one at a time), so results agree to rounding, not bits.
// ---------------------------------------------------------------------------
constexpr int kCholCluster = 8;
constexpr int kCholPanel = 16;
constexpr int kCholClusterMin = 64;

__global__ void __cluster_dims__(kCholCluster, 1, 1) __launch_bounds__(256)
    chol_inv_cluster_kernel(int b, const double* __restrict__ W, double* __restrict__ Lt, double* __restrict__ Mt,
                            int* status) {
    namespace cg = cooperative_groups;
    constexpr int C = kCholCluster;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    extern __shared__ double sm[];
    const int ld = b + 1;
    double* A = sm;                     // lower: L; upper (transposed): own columns of L^{-1}
    double* dinv = sm + (size_t)b * ld;  // 1 / L_jj
    __shared__ double s_thresh;
    __shared__ int s_bad;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    for (int idx = tid; idx < b * b; idx += nt) {
        const int i = idx / b, j = idx % b;
        A[i * ld + j] = (j <= i) ? W[idx] : 0.0;
    }
    __syncthreads();
    if (tid < 32) {  // max of the diagonal and a non-finite flag, over warp 0
        double wmax = 0.0;
        int bad = 0;
        for (int i = lane; i < b; i += 32) {
            const double d = A[i * ld + i];
            if (!isfinite(d)) bad = 2;
            if (d > wmax) wmax = d;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
            bad = max(bad, __shfl_xor_sync(0xffffffffu, bad, o));
        }
        if (lane == 0) {
            if (bad == 0 && !(wmax > 0.0)) bad = 1;
            s_bad = bad;
            s_thresh = (double)b * kEps * wmax;
        }
    }
    __syncthreads();
    cl.sync();  // every copy is loaded before any CTA writes into another's
    for (int p0 = 0; p0 < b; p0 += kCholPanel) {
        if (s_bad) break;  // the same in every CTA
        const int p1 = min(b, p0 + kCholPanel), pw = p1 - p0;
        // 1. the diagonal block
        if (tid < 32) {
            for (int j = p0; j < p1; ++j) {
                if (lane == 0) {
                    const double d = A[j * ld + j];
                    if (!isfinite(d) || !(d > s_thresh)) {
                        s_bad = isfinite(d) ? 1 : 2;
                    } else {
                        const double y = rsqrt_fp64(d);
                        A[j * ld + j] = d * y;
                        dinv[j] = y;
                    }
                }
                __syncwarp();
                if (s_bad) break;
                const double inv = dinv[j];
                for (int i = j + 1 + lane; i < p1; i += 32) A[i * ld + j] *= inv;
                __syncwarp();
                const int nn = p1 - j - 1;
                for (int idx = lane; idx < nn * (nn + 1) / 2; idx += 32) {
                    int ii, kk;
                    tri_decode(idx, ii, kk);
                    const int i = j + 1 + ii, k = j + 1 + kk;
                    A[i * ld + k] = fma(-A[i * ld + j], A[k * ld + j], A[i * ld + k]);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (s_bad) break;
        // 2. this CTA's rows below the block (one thread a row), then every CTA's
        //    copy of them (all threads, one remote store each)
        const int first = p1 + ((rank - p1 % C) % C + C) % C;
        const int nown = first < b ? (b - first + C - 1) / C : 0;
        for (int i = first + C * tid; i < b; i += C * nt) {
            double x[kCholPanel];
#pragma unroll
            for (int l = 0; l < kCholPanel; ++l) {
                if (l < pw) {
                    double a = A[i * ld + p0 + l];
#pragma unroll
                    for (int m = 0; m < l; ++m) a = fma(-x[m], A[(p0 + l) * ld + p0 + m], a);
                    x[l] = a * dinv[p0 + l];
                }
            }
#pragma unroll
            for (int l = 0; l < kCholPanel; ++l)
                if (l < pw) A[i * ld + p0 + l] = x[l];
        }
        __syncthreads();
        for (int idx = tid; idx < nown * pw * (C - 1); idx += nt) {
            const int r = (rank + 1 + idx % (C - 1)) % C, rest = idx / (C - 1);
            const int i = first + C * (rest / pw), col = p0 + rest % pw;
            cl.map_shared_rank(A, r)[i * ld + col] = A[i * ld + col];
        }
        cl.sync();
        // 3. rank-pw update of this CTA's rows i >= p1, columns p1 <= k <= i: 16
        //    threads a row, each over k = p1 + (tid % 16) + 16 m
        for (int t = tid / 16; t < nown; t += nt / 16) {
            const int i = first + C * t;
            double li[kCholPanel];
#pragma unroll
            for (int l = 0; l < kCholPanel; ++l) li[l] = l < pw ? A[i * ld + p0 + l] : 0.0;
            for (int k = p1 + (tid % 16); k <= i; k += 16) {
                double acc = 0.0;
#pragma unroll
                for (int l = 0; l < kCholPanel; ++l)
                    if (l < pw) acc = fma(li[l], A[k * ld + p0 + l], acc);
                A[i * ld + k] -= acc;
            }
        }
        __syncthreads();
        // this CTA's rows of the next diagonal block into every other copy, one remote
        // store per thread: (row t, column p1 + kk <= row, rank)
        const int p2 = min(b, p1 + kCholPanel);
        const int nnext = first < p2 ? (p2 - first + C - 1) / C : 0;
        for (int idx = tid; idx < nnext * kCholPanel * (C - 1); idx += nt) {
            const int r = (rank + 1 + idx % (C - 1)) % C, rest = idx / (C - 1);
            const int i = first + C * (rest / kCholPanel), k = p1 + rest % kCholPanel;
            if (k <= i) cl.map_shared_rank(A, r)[i * ld + k] = A[i * ld + k];
        }
        cl.sync();
    }
    if (s_bad) {
        if (rank == 0 && tid == 0) atomicOr(&status[s_bad == 2 ? kStNonfinite : kStBreakdown], 1);
        for (int idx = rank * nt + tid; idx < b * b; idx += C * nt) {
            const double v = (idx / b == idx % b) ? 1.0 : 0.0;
            Lt[idx] = v;
            Mt[idx] = v;
        }
        return;
    }
    // Lt = L^T (rows i = rank + C u)
    for (int row = rank; row < b; row += C)
        for (int j = tid; j < b; j += nt) Lt[(size_t)row * b + j] = (j >= row) ? A[j * ld + row] : 0.0;
    // X = L^{-1}, column c = rank + C u by one warp (no barriers): forward substitution
    // L x = e_c with the running sums of rows c + lane + 32 t in registers; x_k =
    // acc_k / L_kk comes from the lane holding row k, then rows i > k take
    // acc_i -= L[i][k] x_k.  Row c of Mt = L^{-T} is x (zero left of c).
    constexpr int kRowsPerLane = TSVD_MAX_BLOCK / 32;
    const int warp = tid >> 5, nwarps = nt >> 5;
    for (int c = rank + C * warp; c < b; c += C * nwarps) {
        double acc[kRowsPerLane];
#pragma unroll
        for (int t = 0; t < kRowsPerLane; ++t) acc[t] = (c + lane + 32 * t == c) ? 1.0 : 0.0;
        double* mrow = Mt + (size_t)c * b;
        for (int j = lane; j < c; j += 32) mrow[j] = 0.0;
#pragma unroll
        for (int tt = 0; tt < kRowsPerLane; ++tt) {
            for (int ll = 0; ll < 32; ++ll) {
                const int k = c + 32 * tt + ll;
                if (k >= b) break;  // uniform over the warp
                const double xk = __shfl_sync(0xffffffffu, acc[tt], ll) * dinv[k];
                if (lane == 0) mrow[k] = xk;
#pragma unroll
                for (int t = tt; t < kRowsPerLane; ++t) {
                    const int i = c + lane + 32 * t;
                    if (i > k && i < b) acc[t] = fma(-A[i * ld + k], xk, acc[t]);
                }
            }
        }
    }
}

// out = A U, A and U upper triangular b x b (ld b).  Block = one row i.
__global__ void trmm_upper_kernel(int b, const double* __restrict__ A, const double* __restrict__ U,
                                  double* __restrict__ out, int64_t ldo, int trans) {
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < b; j += blockDim.x) {
        double acc = 0.0;
        for (int k = i; k <= j; ++k) acc = fma(A[i * b + k], U[k * b + j], acc);
        if (trans)
            out[(int64_t)j * ldo + i] = acc;
        else
            out[(int64_t)i * ldo + j] = acc;
    }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and Box-Muller.
// ---------------------------------------------------------------------------
__device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__global__ void gaussian_kernel(int64_t rows, int64_t cols, uint32_t k0, uint32_t k1, uint32_t sid,
                                double* __restrict__ out, int64_t ld, int64_t e_off) {
    // elements e_off .. e_off + rows cols - 1 of the row-major global block: element e
    // is half of Philox counter e / 2, so a slice that starts at an odd element drops
    // the first half of its first pair
    const int64_t n_el = rows * cols;
    const int64_t t0 = e_off / 2, t1 = (e_off + n_el - 1) / 2;
    for (int64_t t = t0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= t1;
         t += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[4] = {(uint32_t)(t & 0xffffffffu), (uint32_t)((uint64_t)t >> 32), sid, 0u};
        philox4x32_10(c, k0, k1);
        const double two53 = 1.1102230246251565e-16;  // 2^-53
        const double u1 = (double)(((uint64_t)(c[0] >> 5) << 26) + (c[1] >> 6) + 1) * two53;
        const double u2 = (double)(((uint64_t)(c[2] >> 5) << 26) + (c[3] >> 6) + 1) * two53;
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        const int64_t e0 = 2 * t - e_off, e1 = e0 + 1;
        if (e0 >= 0 && e0 < n_el) out[(e0 / cols) * ld + (e0 % cols)] = rad * cs;
        if (e1 >= 0 && e1 < n_el) out[(e1 / cols) * ld + (e1 % cols)] = rad * sn;
    }
}

// ---------------------------------------------------------------------------
// Residual column sums of squares, Lanczos estimate, sign convention.
// ---------------------------------------------------------------------------
__global__ void colres_partial_kernel(int64_t q, int k, const double* __restrict__ Y, int64_t ldy,
                                      const double* __restrict__ U, int64_t ldu, const double* __restrict__ sigma,
                                      double* __restrict__ partial, int64_t rows_per) {
    const int64_t r0 = (int64_t)blockIdx.x * rows_per, r1 = min(q, r0 + rows_per);
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double sj = sigma[j];
        double acc = 0.0;
        for (int64_t i = r0; i < r1; ++i) {
            const double d = fma(-U[i * ldu + j], sj, Y[i * ldy + j]);
            acc = fma(d, d, acc);
        }
        partial[(int64_t)blockIdx.x * k + j] = acc;
    }
}

__global__ void colres_reduce_kernel(int k, int g, const double* __restrict__ partial, double* __restrict__ out) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double acc = 0.0;
        for (int t = 0; t < g; ++t) acc += partial[(int64_t)t * k + j];
        out[j] = acc;
    }
}

__global__ void lanczos_rho_kernel(int b, int k, const double* __restrict__ Rr, const double* __restrict__ V,
                                   int64_t ldv, double* __restrict__ rho) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < b; ++i) {
            double yi = 0.0;
            for (int l = i; l < b; ++l) yi = fma(Rr[i * b + l], V[(int64_t)l * ldv + j], yi);
            acc = fma(yi, yi, acc);
        }
        rho[j] = sqrt(acc);
    }
}

__global__ void argmax_partial_kernel(int64_t n, int k, const double* __restrict__ V, int64_t ldv,
                                      int64_t rows_per, double* __restrict__ pv, int64_t* __restrict__ pi) {
    const int64_t r0 = (int64_t)blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double best = -1.0;
        int64_t bi = 0;
        for (int64_t i = r0; i < r1; ++i) {
            const double a = fabs(V[i * ldv + j]);
            if (a > best) {
                best = a;
                bi = i;
            }
        }
        pv[(int64_t)blockIdx.x * k + j] = best;
        pi[(int64_t)blockIdx.x * k + j] = bi;
    }
}

__global__ void argmax_sign_kernel(int k, int g, const double* __restrict__ pv, const int64_t* __restrict__ pi,
                                   const double* __restrict__ V, int64_t ldv, double* __restrict__ sgn) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double best = -1.0;
        int64_t bi = 0;
        for (int t = 0; t < g; ++t) {
            const double a = pv[(int64_t)t * k + j];
            if (a > best) {
                best = a;
                bi = pi[(int64_t)t * k + j];
            }
        }
        sgn[j] = V[bi * ldv + j] < 0.0 ? -1.0 : 1.0;
    }
}

__global__ void apply_sign_kernel(int64_t rows, int k, double* __restrict__ A, int64_t lda,
                                  const double* __restrict__ sgn) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    const int64_t i = idx / k;
    const int j = (int)(idx % k);
    if (sgn[j] < 0.0) A[i * lda + j] = -A[i * lda + j];
}

__global__ void put_transposed_kernel(int rows, int cols, const double* __restrict__ H, int64_t ldh,
                                      double* __restrict__ D, int64_t ldd) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)rows * cols) return;
    const int i = (int)(idx / cols), j = (int)(idx % cols);
    D[(int64_t)j * ldd + i] = H[(int64_t)i * ldh + j];
}

__global__ void put_diagonal_kernel(int s, const double* __restrict__ sig, double* __restrict__ B, int64_t ldb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < s) B[(int64_t)i * ldb + i] = sig[i];
}

int colres_groups(int64_t q) {
    int64_t g = (q + 255) / 256;
    if (g > 512) g = 512;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------
size_t gemm_tn_ws(tsvd_handle* h, int64_t q, int64_t s, int64_t b, bool symmetric, int elem_bytes) {
    (void)h;
    const TnPlan p = tn_plan(q, s, b, symmetric, elem_bytes);
    if (p.slabs == 1 && !symmetric) return 0;
    return align256(sizeof(double) * (size_t)p.slabs * (size_t)s * (size_t)b);
}

template <typename TI, typename TC>
cudaError_t gemm_tn(tsvd_handle* h, int64_t q, int64_t s, int64_t b, const TI* X, int64_t ldx, const TI* Z,
                    int64_t ldz, TC* C, int64_t ldc, bool symmetric, double* partial, cudaStream_t st) {
    if (s == 0 || b == 0) return cudaSuccess;
    constexpr bool kF32 = std::is_same<TI, float>::value;
    const TnPlan p = tn_plan(q, s, b, symmetric, (int)sizeof(TI));
    if (q == 0) {
        for (int64_t i = 0; i < s; ++i) {
            cudaError_t e = cudaMemsetAsync(C + i * ldc, 0, sizeof(TC) * b, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const dim3 grid((unsigned)p.regions, (unsigned)p.slabs);
    // algorithmic work: 2qsb flops (the upper half, q b (b+1), for a Gram matrix);
    // compulsory traffic: X and Z read once, C written once
    ProfScope prof(h, TSVD_K_GEMM_TN, symmetric ? (double)q * b * (b + 1) : 2.0 * q * s * b,
                   (double)sizeof(TI) * (double)q * (symmetric ? b : s + b) + (double)sizeof(TC) * s * b, st);
    if constexpr (std::is_same<TI, double>::value && std::is_same<TC, double>::value) {
        const OzCache* xc = h->oz_ws ? oz_find_cache(h, X, ldx, q, s, true) : nullptr;
        if (h->oz_ws && oz_worth(s, b, q) && oz_tn_ws(q, s, b, symmetric, xc != nullptr) <= h->oz_bytes) {
            const int rc = oz_gemm_tn(h, q, s, b, X, ldx, Z, ldz, C, ldc, symmetric, h->oz_ws, h->oz_bytes,
                                      h->oz_status, st, xc);
            return rc == TSVD_OK ? cudaSuccess : cudaErrorUnknown;
        }
    }
    if (p.slabs == 1 && !symmetric) {
        h->launches++;
        if constexpr (kF32)
            return launch_gemm_tn_f32<TC>(grid, st, q, s, b, X, ldx, Z, ldz, C, ldc, 0, p.slab_rows, 0, p.nreg_s,
                                          p.nreg_b);
        gemm_tn_kernel<TI, TC><<<grid, 128, 0, st>>>(q, s, b, X, ldx, Z, ldz, C, ldc, 0, p.slab_rows, 0, p.nreg_s,
                                                     p.nreg_b);
        return cudaGetLastError();
    }
    const int64_t stride = s * b;
    h->launches += 2;
    if constexpr (kF32) {
        cudaError_t e = launch_gemm_tn_f32<double>(grid, st, q, s, b, X, ldx, Z, ldz, partial, b, stride, p.slab_rows,
                                                   symmetric ? 1 : 0, p.nreg_s, p.nreg_b);
        if (e != cudaSuccess) return e;
    } else {
        gemm_tn_kernel<TI, double><<<grid, 128, 0, st>>>(q, s, b, X, ldx, Z, ldz, partial, b, stride, p.slab_rows,
                                                         symmetric ? 1 : 0, p.nreg_s, p.nreg_b);
    }
    const int64_t tot = s * b;
    gemm_tn_reduce_kernel<TC><<<(unsigned)((tot + 31) / 32), dim3(32, 8), 0, st>>>(s, b, p.slabs, partial, stride, C,
                                                                                  ldc, symmetric ? 1 : 0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused update + Gram of FP32 blocks.  One CTA per slab of consecutive 64-row
// tiles; the split targets one wave of the kernel's resident 256-thread CTAs on
// 152 SMs: 4 per SM for b <= 64, 2 for b <= 128 (a fixed target, so the split, the
// workspace and the summation order do not depend on the device).
struct UgPlan {
    int slabs;
    int64_t slab_rows;
};

static UgPlan ug_plan(int64_t q, int64_t b) {
    UgPlan p;
    const int64_t wave = 152 * (b <= 64 ? 4 : 2);
    int64_t tiles = (q + 63) / 64;
    if (tiles < 1) tiles = 1;
    const int64_t slabs = tiles < wave ? tiles : wave;
    p.slab_rows = (tiles + slabs - 1) / slabs * 64;
    p.slabs = (int)((q + p.slab_rows - 1) / p.slab_rows);
    if (p.slabs < 1) p.slabs = 1;
    return p;
}

size_t update_gram_ws(int64_t q, int64_t b) {
    return align256(sizeof(double) * (size_t)ug_plan(q, b).slabs * (size_t)b * (size_t)b);
}

cudaError_t update_gram(tsvd_handle* h, int64_t q, int64_t s, int64_t b, double alpha, const float* X, int64_t ldx,
                        const double* M, int64_t ldm, double beta, float* Y, int64_t ldy, bool upper, double* W,
                        double* partial, cudaStream_t st) {
    if (b < 1 || b > 128 || s < 1) return cudaErrorInvalidValue;
    if (q == 0) return cudaMemsetAsync(W, 0, sizeof(double) * (size_t)b * b, st);
    const UgPlan p = ug_plan(q, b);
    // algorithmic work: the update (2qsb, or q b (b+1) for a triangular M) plus the
    // upper half of the Gram matrix, q b (b+1); compulsory traffic: X and M read,
    // Y read (beta != 0, unless it is X) and written, W written
    const bool alias = (const void*)X == (const void*)Y;
    const double upd = upper ? (double)q * b * (b + 1) : 2.0 * q * s * b;
    const double bytes = 4.0 * q * s + ((beta != 0.0 && !alias) ? 4.0 * q * b : 0.0) + 4.0 * q * b +
                         8.0 * s * b + 8.0 * b * b;
    ProfScope prof(h, TSVD_K_UPD_GRAM, upd + (double)q * b * (b + 1), bytes, st);
    h->launches += 2;
    cudaError_t e = launch_update_gram_f32<double>(st, p.slabs, p.slab_rows, q, s, b, alpha, X, ldx, M, ldm, beta, Y,
                                                   ldy, upper, partial);
    if (e != cudaSuccess) return e;
    gemm_tn_reduce_kernel<double><<<(unsigned)((b * b + 31) / 32), dim3(32, 8), 0, st>>>(b, b, p.slabs, partial,
                                                                                         b * b, W, b, 1);
    return cudaGetLastError();
}

template cudaError_t gemm_tn<double, double>(tsvd_handle*, int64_t, int64_t, int64_t, const double*, int64_t,
                                             const double*, int64_t, double*, int64_t, bool, double*, cudaStream_t);
template cudaError_t gemm_tn<float, double>(tsvd_handle*, int64_t, int64_t, int64_t, const float*, int64_t,
                                            const float*, int64_t, double*, int64_t, bool, double*, cudaStream_t);
template cudaError_t gemm_tn<float, float>(tsvd_handle*, int64_t, int64_t, int64_t, const float*, int64_t,
                                           const float*, int64_t, float*, int64_t, bool, double*, cudaStream_t);

template <typename TX, typename TM, typename TY>
cudaError_t gemm_nn(tsvd_handle* h, int64_t q, int64_t s, int64_t b, double alpha, const TX* X, int64_t ldx,
                    const TM* M, int64_t ldm, double beta, TY* Y, int64_t ldy, bool upper, cudaStream_t st) {
    if (q == 0 || b == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((q + 31) / 32);
    ProfScope prof(h, TSVD_K_GEMM_NN, upper ? (double)q * b * (b + 1) : 2.0 * q * s * b,
                   (double)sizeof(TX) * q * s + (double)sizeof(TM) * s * b +
                       (double)sizeof(TY) * q * b * (beta != 0.0 ? 2 : 1), st);
    if constexpr (std::is_same<TX, double>::value && std::is_same<TM, double>::value &&
                  std::is_same<TY, double>::value) {
        const OzCache* xc = (h->oz_ws && !h->oz_fresh_rows) ? oz_find_cache(h, X, ldx, q, s, false) : nullptr;
        if (h->oz_ws && s > 0 && oz_worth(q, b, s) && oz_nn_ws(q, s, b, xc != nullptr) <= h->oz_bytes) {
            const int rc = oz_gemm_nn(h, q, s, b, alpha, X, ldx, M, ldm, beta, Y, ldy, upper, h->oz_ws, h->oz_bytes,
                                      h->oz_status, st, xc);
            return rc == TSVD_OK ? cudaSuccess : cudaErrorUnknown;
        }
    }
    h->launches++;
    if constexpr (std::is_same<TX, float>::value) {
        if (b <= 128) return launch_gemm_nn_f32<TM, TY>(st, q, s, b, alpha, X, ldx, M, ldm, beta, Y, ldy, upper);
    }
    if (b <= 32) {
        gemm_nn_kernel<8, TX, TM, TY><<<grid, 128, 0, st>>>(q, s, b, alpha, X, ldx, M, ldm, beta, Y, ldy, upper ? 1 : 0);
    } else if (b <= 64) {
        gemm_nn_kernel<16, TX, TM, TY><<<grid, 128, 0, st>>>(q, s, b, alpha, X, ldx, M, ldm, beta, Y, ldy,
                                                             upper ? 1 : 0);
    } else {
        gemm_nn_kernel<32, TX, TM, TY><<<grid, 128, 0, st>>>(q, s, b, alpha, X, ldx, M, ldm, beta, Y, ldy,
                                                             upper ? 1 : 0);
    }
    return cudaGetLastError();
}

#define TSVD_INST_NN(TX, TM, TY)                                                                                  \
    template cudaError_t gemm_nn<TX, TM, TY>(tsvd_handle*, int64_t, int64_t, int64_t, double, const TX*, int64_t, \
                                             const TM*, int64_t, double, TY*, int64_t, bool, cudaStream_t);
TSVD_INST_NN(double, double, double)
TSVD_INST_NN(float, double, float)
TSVD_INST_NN(float, float, float)
TSVD_INST_NN(float, double, double)
#undef TSVD_INST_NN

static size_t chol_smem(int b) { return sizeof(double) * ((size_t)b * (b + 1) + b); }

cudaError_t chol_inv(tsvd_handle* h, int b, const double* W, double* Lt, double* Mt, int* status,
                     cudaStream_t st) {
    const size_t smem = chol_smem(b);
    static thread_local int configured_device = -1;
    if (configured_device != h->device) {
        cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)chol_smem(TSVD_MAX_BLOCK));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(chol_inv_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)chol_smem(TSVD_MAX_BLOCK));
        if (e != cudaSuccess) return e;
        configured_device = h->device;
    }
    ProfScope prof(h, TSVD_K_CHOL, 2.0 * b * b * (double)b / 3.0, 24.0 * b * b, st);
    h->launches++;
    if (b >= kCholClusterMin)
        chol_inv_cluster_kernel<<<kCholCluster, 256, smem, st>>>(b, W, Lt, Mt, status);
    else
        chol_inv_kernel<<<1, 256, smem, st>>>(b, W, Lt, Mt, status);
    return cudaGetLastError();
}

cudaError_t trmm_upper(tsvd_handle* h, int b, const double* A, const double* U, double* out, int64_t ldo,
                       bool trans, cudaStream_t st) {
    ProfScope prof(h, TSVD_K_OTHER, b * b * (double)b / 3.0, 24.0 * b * b, st);
    h->launches++;
    trmm_upper_kernel<<<b, 128, 0, st>>>(b, A, U, out, ldo, trans ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t gaussian(tsvd_handle* h, int64_t rows, int64_t cols, uint64_t seed, uint32_t stream_id, double* out,
                     int64_t ld, cudaStream_t st, int64_t row0) {
    if (rows * cols == 0) return cudaSuccess;
    const int64_t e_off = row0 * cols;
    const int64_t n_pairs = (e_off + rows * cols - 1) / 2 - e_off / 2 + 1;
    int64_t blocks = (n_pairs + 255) / 256;
    if (blocks > 8LL * h->sm_count * 8) blocks = 8LL * h->sm_count * 8;
    ProfScope prof(h, TSVD_K_OTHER, 0.0, 8.0 * rows * cols, st);
    h->launches++;
    gaussian_kernel<<<(unsigned)blocks, 256, 0, st>>>(rows, cols, (uint32_t)(seed & 0xffffffffu),
                                                      (uint32_t)(seed >> 32), stream_id, out, ld, e_off);
    return cudaGetLastError();
}

size_t colres_ws(int64_t q, int k) { return align256(sizeof(double) * (size_t)colres_groups(q) * (size_t)k); }

cudaError_t col_residual_sq(tsvd_handle* h, int64_t q, int k, const double* Y, int64_t ldy, const double* U,
                            int64_t ldu, const double* sigma, double* out, double* partial, cudaStream_t st) {
    const int g = colres_groups(q);
    const int64_t rows_per = (q + g - 1) / g;
    ProfScope prof(h, TSVD_K_OTHER, 0.0, 0.0, st);
    h->launches += 2;
    colres_partial_kernel<<<g, 128, 0, st>>>(q, k, Y, ldy, U, ldu, sigma, partial, rows_per);
    colres_reduce_kernel<<<1, 128, 0, st>>>(k, g, partial, out);
    return cudaGetLastError();
}

cudaError_t put_transposed(tsvd_handle* h, int rows, int cols, const double* H, int64_t ldh, double* D, int64_t ldd,
                           cudaStream_t st) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    const int64_t tot = (int64_t)rows * cols;
    h->launches++;
    put_transposed_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(rows, cols, H, ldh, D, ldd);
    return cudaGetLastError();
}

cudaError_t put_diagonal(tsvd_handle* h, int s, const double* sig, double* B, int64_t ldb, cudaStream_t st) {
    if (s == 0) return cudaSuccess;
    h->launches++;
    put_diagonal_kernel<<<(unsigned)((s + 255) / 256), 256, 0, st>>>(s, sig, B, ldb);
    return cudaGetLastError();
}

cudaError_t lanczos_rho(tsvd_handle* h, int b, int k, const double* Rr, const double* Vlast, int64_t ldv,
                        double* rho, cudaStream_t st) {
    ProfScope prof(h, TSVD_K_OTHER, 0.0, 0.0, st);
    h->launches++;
    lanczos_rho_kernel<<<1, 128, 0, st>>>(b, k, Rr, Vlast, ldv, rho);
    return cudaGetLastError();
}

size_t sign_fix_ws(int64_t n, int k) {
    const size_t g = (size_t)colres_groups(n);
    return align256(sizeof(double) * g * k) + align256(sizeof(int64_t) * g * k) + align256(sizeof(double) * k);
}

cudaError_t sign_fix(tsvd_handle* h, int64_t n, int64_t m, int k, double* V, int64_t ldv, double* U, int64_t ldu,
                     void* ws, cudaStream_t st) {
    const int g = colres_groups(n);
    char* p = static_cast<char*>(ws);
    double* pv = reinterpret_cast<double*>(p);
    p += align256(sizeof(double) * (size_t)g * k);
    int64_t* pi = reinterpret_cast<int64_t*>(p);
    p += align256(sizeof(int64_t) * (size_t)g * k);
    double* sgn = reinterpret_cast<double*>(p);
    const int64_t rows_per = (n + g - 1) / g;
    ProfScope prof(h, TSVD_K_OTHER, 0.0, 0.0, st);
    h->launches += 4;
    argmax_partial_kernel<<<g, 128, 0, st>>>(n, k, V, ldv, rows_per, pv, pi);
    argmax_sign_kernel<<<1, 128, 0, st>>>(k, g, pv, pi, V, ldv, sgn);
    if (n * k > 0) apply_sign_kernel<<<(unsigned)((n * k + 255) / 256), 256, 0, st>>>(n, k, V, ldv, sgn);
    if (m * k > 0) apply_sign_kernel<<<(unsigned)((m * k + 255) / 256), 256, 0, st>>>(m, k, U, ldu, sgn);
    return cudaGetLastError();
}

}  // namespace tsvd
