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
__global__ void __launch_bounds__(64, 16) gemm_tn_f32_kernel(int64_t q, int64_t s, int64_t b,
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

// Fused update + Gram (CGS-CQR2, Alg. 5: the update Q - P H and the Gram matrix of
// the updated block that the next CholeskyQR step factors; CholeskyQR2, Alg. 4: the
// first step's Q L^{-T} and the second step's Gram matrix).  A CTA owns a slab of
// consecutive 64-row tiles.  Per tile it forms Y' = beta Y + alpha X M exactly as
// gemm_nn_f32 does (same products, same FMA order, so Y' has the same bits), stores
// Y', keeps the tile in shared memory and adds its Y'^T Y' into the CTA's b x b
// accumulator: Y' is never read back from memory for its Gram matrix.  The slab's
// Gram sum is FP32 (like gemm_tn_f32's slabs) and is written as an FP64 partial
// (slab, b x b), reduced across slabs in a fixed order by the caller.  Thread
// (ty, tx) in 16 x 16 owns Gram rows 4ty..4ty+3 + 64p and columns 4tx..4tx+3 + 64p'
// for the upper quadrants p <= p' (the reduction reads only the upper half).
//
// The next K chunk of X and M is loaded into registers while the current one is
// multiplied (one shared buffer, two barriers a chunk), and the chunk buffers share
// their memory with the Y' tile, which is only live after the last chunk.  With
// that, b <= 64 runs 4 CTAs (32 warps) per SM and b <= 128 runs 2; the slab plan
// (update_gram) sizes one wave to match (kUgMinBlocks).
constexpr int kUgRows = 64;

template <int NP>
struct UgCfg {
    static constexpr int kMinBlocks = NP == 1 ? 4 : 2;
    static constexpr int kGramUnroll = NP == 1 ? 2 : 4;  // keeps NP = 1 within 64 registers
};

template <int NP, typename TM>
__global__ void __launch_bounds__(256, UgCfg<NP>::kMinBlocks)
    update_gram_f32_kernel(int64_t q, int64_t s, int64_t b, float alpha, const float* X, int64_t ldx,
                           const TM* __restrict__ M, int64_t ldm, float beta, float* Y, int64_t ldy, int upper,
                           double* __restrict__ partial, int64_t slab_rows) {
    constexpr int BW = 64 * NP;
    constexpr int NQ = NP == 1 ? 1 : 3;  // upper quadrants (0,0) [, (0,1), (1,1)]
    constexpr int XS = kNnK * (kNnRows + 4), MS = kNnK * BW, YS = kUgRows * (BW + 4);
    constexpr int SMEM = (XS + MS) > YS ? (XS + MS) : YS;
    __shared__ __align__(16) float sm[SMEM];
    float(*XsT)[kNnRows + 4] = reinterpret_cast<float(*)[kNnRows + 4]>(sm);
    float(*Ms)[BW] = reinterpret_cast<float(*)[BW]>(sm + XS);
    float(*Ys)[BW + 4] = reinterpret_cast<float(*)[BW + 4]>(sm);
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int64_t s0 = (int64_t)blockIdx.x * slab_rows;
    const int64_t s1 = min(q, s0 + slab_rows);
    const int64_t kmax = upper ? min(s, b) : s;
    float g[NQ][4][4];
#pragma unroll
    for (int c = 0; c < NQ; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) g[c][i][j] = 0.f;
    for (int64_t r0 = s0; r0 < s1; r0 += kUgRows) {
        float acc[4][4 * NP];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4 * NP; ++j) acc[i][j] = 0.f;
        // chunk k0 of X (64 rows x 16, element tid + 256 t) and of M (16 x BW)
        float xr[4], mr[4 * NP];
        auto load = [&](int64_t k0) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int idx = tid + 256 * t;
                const int64_t row = r0 + idx / kNnK, k = k0 + idx % kNnK;
                xr[t] = (row < s1 && k < s) ? X[row * ldx + k] : 0.f;
            }
#pragma unroll
            for (int t = 0; t < 4 * NP; ++t) {
                const int idx = tid + 256 * t;
                const int cc = idx % BW;
                const int64_t k = k0 + idx / BW;
                const bool in = k < s && cc < b && !(upper && k > cc);
                mr[t] = in ? (float)M[k * ldm + cc] : 0.f;
            }
        };
        load(0);
        for (int64_t k0 = 0; k0 < kmax; k0 += kNnK) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int idx = tid + 256 * t;
                XsT[idx % kNnK][idx / kNnK] = xr[t];
            }
#pragma unroll
            for (int t = 0; t < 4 * NP; ++t) {
                const int idx = tid + 256 * t;
                Ms[idx / BW][idx % BW] = mr[t];
            }
            __syncthreads();
            if (k0 + kNnK < kmax) load(k0 + kNnK);
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
        // Y' of the tile: global store (rows of the slab, columns < b) and the shared
        // copy (zero outside), after every read of X's tile rows (Y may alias X).
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t row = r0 + 4 * ty + i;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float4 yv;
                float* ya = reinterpret_cast<float*>(&yv);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t col = 64 * p + 4 * tx + j;
                    float v = 0.f;
                    if (row < s1 && col < b) {
                        float* y = Y + row * ldy + col;
                        v = alpha * acc[i][4 * p + j];
                        if (beta != 0.f) v = fmaf(beta, *y, v);
                        *y = v;
                    }
                    ya[j] = v;
                }
                *reinterpret_cast<float4*>(&Ys[4 * ty + i][64 * p + 4 * tx]) = yv;
            }
        }
        __syncthreads();
#pragma unroll UgCfg<NP>::kGramUnroll
        for (int kk = 0; kk < kUgRows; ++kk) {
            float xa[NP][4], za[NP][4];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float4 xv = *reinterpret_cast<const float4*>(&Ys[kk][64 * p + 4 * ty]);
                const float4 zv = *reinterpret_cast<const float4*>(&Ys[kk][64 * p + 4 * tx]);
                xa[p][0] = xv.x, xa[p][1] = xv.y, xa[p][2] = xv.z, xa[p][3] = xv.w;
                za[p][0] = zv.x, za[p][1] = zv.y, za[p][2] = zv.z, za[p][3] = zv.w;
            }
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                const int pi = c == 2 ? 1 : 0, pj = c == 0 ? 0 : 1;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) g[c][i][j] = fmaf(xa[pi][i], za[pj][j], g[c][i][j]);
            }
        }
        __syncthreads();  // the next tile's chunks overwrite the Y' tile
    }
    double* o = partial + (int64_t)blockIdx.x * b * b;
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        const int pi = c == 2 ? 1 : 0, pj = c == 0 ? 0 : 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t row = 64 * pi + 4 * ty + i;
            if (row >= b) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t col = 64 * pj + 4 * tx + j;
                if (col < b) o[row * b + col] = (double)g[c][i][j];
            }
        }
    }
}

}  // namespace

template <typename TM>
cudaError_t launch_update_gram_f32(cudaStream_t st, int slabs, int64_t slab_rows, int64_t q, int64_t s, int64_t b,
                                   double alpha, const float* X, int64_t ldx, const TM* M, int64_t ldm, double beta,
                                   float* Y, int64_t ldy, bool upper, double* partial) {
    if (b <= 64)
        update_gram_f32_kernel<1, TM><<<(unsigned)slabs, 256, 0, st>>>(q, s, b, (float)alpha, X, ldx, M, ldm,
                                                                       (float)beta, Y, ldy, upper ? 1 : 0, partial,
                                                                       slab_rows);
    else
        update_gram_f32_kernel<2, TM><<<(unsigned)slabs, 256, 0, st>>>(q, s, b, (float)alpha, X, ldx, M, ldm,
                                                                       (float)beta, Y, ldy, upper ? 1 : 0, partial,
                                                                       slab_rows);
    return cudaGetLastError();
}
template cudaError_t launch_update_gram_f32<double>(cudaStream_t, int, int64_t, int64_t, int64_t, int64_t, double,
                                                    const float*, int64_t, const double*, int64_t, double, float*,
                                                    int64_t, bool, double*);

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
