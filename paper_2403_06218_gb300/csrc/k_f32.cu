// Register-tiled FP32 products of the mixed-precision form (Sec. 3 building
// blocks with FP32 blocks): the FP32 pipe is 64 times wider than the FP64 one, so
// here the limit is feeding it, not issuing it.  Each thread owns a 4 x 4 (or
// 4 x 8) tile of outputs and does 16 (32) FMAs per pair of 16-byte shared-memory
// loads.
//   gemm_tn_f32: C (s x b) = X^T Z over one row slab per CTA (split-K partials in
//                FP64, the same plan and workspace as the FP64 kernel);
//   gemm_nn_f32: Y (q x b) = beta Y + alpha X M, M in FP64 or FP32 converted on load.
#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

constexpr int kR = 32;   // region edge (same regions as the FP64 kernel)
constexpr int kKc = 32;  // rows per shared-memory chunk

__device__ inline void decode_upper32(int lin, int nr, int& ri, int& rj) {
    int r = 0;
    while (lin >= nr - r) {
        lin -= nr - r;
        ++r;
    }
    ri = r;
    rj = r + lin;
}

// 64 threads: thread (ty, tx) in 8 x 8 owns rows 4ty..4ty+3, columns 4tx..4tx+3 of the region.
template <typename TW>
__global__ void __launch_bounds__(64) gemm_tn_f32_kernel(int64_t q, int64_t s, int64_t b,
                                                         const float* __restrict__ X, int64_t ldx,
                                                         const float* __restrict__ Z, int64_t ldz,
                                                         TW* __restrict__ out, int64_t ldo, int64_t slab_stride,
                                                         int64_t slab_rows, int symmetric, int nreg_s, int nreg_b) {
    __shared__ __align__(16) float Xs[kKc][kR];
    __shared__ __align__(16) float Zs[kKc][kR];
    int ri, rj;
    if (symmetric) {
        decode_upper32((int)blockIdx.x, nreg_s, ri, rj);
    } else {
        ri = (int)blockIdx.x / nreg_b;
        rj = (int)blockIdx.x % nreg_b;
    }
    const int64_t r0 = (int64_t)blockIdx.y * slab_rows;
    const int64_t r1 = min(q, r0 + slab_rows);
    const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
    const int64_t xc0 = (int64_t)ri * kR, zc0 = (int64_t)rj * kR;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int64_t k0 = r0; k0 < r1; k0 += kKc) {
        for (int idx = tid; idx < kKc * kR; idx += 64) {
            const int rr = idx / kR, cc = idx % kR;
            const int64_t row = k0 + rr;
            const bool rin = row < r1;
            Xs[rr][cc] = (rin && xc0 + cc < s) ? X[row * ldx + xc0 + cc] : 0.f;
            Zs[rr][cc] = (rin && zc0 + cc < b) ? Z[row * ldz + zc0 + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kKc; ++kk) {
            const float4 xv = *reinterpret_cast<const float4*>(&Xs[kk][4 * ty]);
            const float4 zv = *reinterpret_cast<const float4*>(&Zs[kk][4 * tx]);
            const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
            const float za[4] = {zv.x, zv.y, zv.z, zv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xa[i], za[j], acc[i][j]);
        }
        __syncthreads();
    }
    // symmetric: only tiles touching the upper triangle are needed (the reduction reads i <= j)
    if (symmetric && ri == rj && ty > tx) return;
    TW* o = out + (int64_t)blockIdx.y * slab_stride;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t row = xc0 + 4 * ty + i;
        if (row >= s) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t col = zc0 + 4 * tx + j;
            if (col < b) o[row * ldo + col] = (TW)acc[i][j];
        }
    }
}

// 256 threads: thread (ty, tx) in 16 x 16 owns rows 4ty..4ty+3 of a 64-row tile and
// columns {4tx..4tx+3} + 64 p, p < NP, of the output (NP = 1: b <= 64, NP = 2: b <= 128).
// All panels are accumulated before any store, so Y may alias X (s == b).
constexpr int kNnRows = 64;
constexpr int kNnK = 16;

template <int NP, typename TM, typename TY>
__global__ void __launch_bounds__(256) gemm_nn_f32_kernel(int64_t q, int64_t s, int64_t b, float alpha,
                                                          const float* __restrict__ X, int64_t ldx,
                                                          const TM* __restrict__ M, int64_t ldm, float beta, TY* Y,
                                                          int64_t ldy, int upper) {
    __shared__ __align__(16) float XsT[kNnK][kNnRows + 4];
    __shared__ __align__(16) float Ms[kNnK][64 * NP];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int64_t r0 = (int64_t)blockIdx.x * kNnRows;
    float acc[4][4 * NP];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4 * NP; ++j) acc[i][j] = 0.f;
    const int64_t kmax = upper ? min(s, b) : s;
    for (int64_t k0 = 0; k0 < kmax; k0 += kNnK) {
        for (int idx = tid; idx < kNnRows * kNnK; idx += 256) {
            const int rr = idx / kNnK, kk = idx % kNnK;
            const int64_t row = r0 + rr, k = k0 + kk;
            XsT[kk][rr] = (row < q && k < s) ? X[row * ldx + k] : 0.f;
        }
        for (int idx = tid; idx < kNnK * 64 * NP; idx += 256) {
            const int kk = idx / (64 * NP), cc = idx % (64 * NP);
            const int64_t k = k0 + kk;
            const bool in = k < s && cc < b && !(upper && k > cc);
            Ms[kk][cc] = in ? (float)M[k * ldm + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kNnK; ++kk) {
            const float4 xv = *reinterpret_cast<const float4*>(&XsT[kk][4 * ty]);
            const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float4 mv = *reinterpret_cast<const float4*>(&Ms[kk][64 * p + 4 * tx]);
                const float ma[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][4 * p + j] = fmaf(xa[i], ma[j], acc[i][4 * p + j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t row = r0 + 4 * ty + i;
        if (row >= q) continue;
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t col = 64 * p + 4 * tx + j;
                if (col < b) {
                    TY* y = Y + row * ldy + col;
                    const float v = alpha * acc[i][4 * p + j];
                    *y = (beta != 0.f) ? (TY)fmaf(beta, (float)*y, v) : (TY)v;
                }
            }
    }
}

}  // namespace

template <typename TW>
cudaError_t launch_gemm_tn_f32(dim3 grid, cudaStream_t st, int64_t q, int64_t s, int64_t b, const float* X,
                               int64_t ldx, const float* Z, int64_t ldz, TW* out, int64_t ldo, int64_t slab_stride,
                               int64_t slab_rows, int symmetric, int nreg_s, int nreg_b) {
    gemm_tn_f32_kernel<TW><<<grid, 64, 0, st>>>(q, s, b, X, ldx, Z, ldz, out, ldo, slab_stride, slab_rows, symmetric,
                                                nreg_s, nreg_b);
    return cudaGetLastError();
}
template cudaError_t launch_gemm_tn_f32<double>(dim3, cudaStream_t, int64_t, int64_t, int64_t, const float*, int64_t,
                                                const float*, int64_t, double*, int64_t, int64_t, int64_t, int, int,
                                                int);
template cudaError_t launch_gemm_tn_f32<float>(dim3, cudaStream_t, int64_t, int64_t, int64_t, const float*, int64_t,
                                               const float*, int64_t, float*, int64_t, int64_t, int64_t, int, int, int);

template <typename TM, typename TY>
cudaError_t launch_gemm_nn_f32(cudaStream_t st, int64_t q, int64_t s, int64_t b, double alpha, const float* X,
                               int64_t ldx, const TM* M, int64_t ldm, double beta, TY* Y, int64_t ldy, bool upper) {
    const unsigned grid = (unsigned)((q + kNnRows - 1) / kNnRows);
    if (b <= 64)
        gemm_nn_f32_kernel<1, TM, TY><<<grid, 256, 0, st>>>(q, s, b, (float)alpha, X, ldx, M, ldm, (float)beta, Y,
                                                            ldy, upper ? 1 : 0);
    else
        gemm_nn_f32_kernel<2, TM, TY><<<grid, 256, 0, st>>>(q, s, b, (float)alpha, X, ldx, M, ldm, (float)beta, Y,
                                                            ldy, upper ? 1 : 0);
    return cudaGetLastError();
}
template cudaError_t launch_gemm_nn_f32<double, float>(cudaStream_t, int64_t, int64_t, int64_t, double, const float*,
                                                       int64_t, const double*, int64_t, double, float*, int64_t, bool);
template cudaError_t launch_gemm_nn_f32<float, float>(cudaStream_t, int64_t, int64_t, int64_t, double, const float*,
                                                      int64_t, const float*, int64_t, double, float*, int64_t, bool);
template cudaError_t launch_gemm_nn_f32<double, double>(cudaStream_t, int64_t, int64_t, int64_t, double, const float*,
                                                        int64_t, const double*, int64_t, double, double*, int64_t,
                                                        bool);

}  // namespace tsvd
