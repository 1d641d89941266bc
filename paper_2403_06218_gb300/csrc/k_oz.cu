// FP64-accurate products on the tensor cores for the FP64 method: the Gram and
// projection products of CholeskyQR2 and CGS-CQR2 (Alg. 4 S1/S4, Alg. 5 S1/S6:
// C = X^T Z), the updates and triangular solves (Alg. 5 S2/S7, Alg. 4 S3/S6:
// Y = beta Y + alpha X M), and the Ritz / restart products (Alg. 2 S7-S9).
// GB300's FP64 pipe issues 2 DFMA/clk/SM; its BF16 tensor cores are about 1500x
// faster, so these products are run as exact integer arithmetic on BF16 digits
// (the exponent-aligned slicing of Ozaki, Ogita, Oishi and Rump, 2012, with the
// fixed-point digits of Ootomo, Ozaki and Yokota, 2024):
//
//  * every row of the left operand A and every column of the right operand B
//    gets one exponent e (the smallest e with |x| < 2^e over that row or
//    column); each entry becomes the 56-bit integer F = round(x 2^(55 - e)),
//    split into 7 balanced base-256 digits d_0..d_6 (F = sum d_p 2^(8(6-p)),
//    |d_p| <= 128).  Digit p is stored as the BF16 value d_p 2^(-8p) (exact);
//  * the 28 digit products with p + q <= 6 are issued as tcgen05 MMAs (M = 128,
//    K = 16, FP32 accumulators in tensor memory), one accumulator per value of
//    p + q (7 accumulators side by side, 448 TMEM columns); the products of one
//    A digit plane with all its B planes form a single MMA of N up to 256.  Over 128 consecutive k
//    each product is an integer times 2^(-8(p+q)) of magnitude <= 2^14 and each
//    group sum T_{p+q} is an integer below 2^24, so every accumulation is exact
//    whatever the tensor core's internal rounding;
//  * every 128 k the epilogue converts the accumulators to integers and adds
//    T_0..T_4 into a 64-bit integer (units of 2^-32 of the leading digit
//    product), T_5 and T_6 (rounded to 2^-40) into a 32-bit one, and at the end
//    of its K range writes C = 2^(ea + eb - 46) (hi + lo 2^-8) in FP64.
// Each operand entry is represented to 2^-56 of its row (column) scale 2^e, the
// dropped digit products are below 6.1 K 2^(ea + eb - 56), and the result is
// rounded once to FP64: normwise FP64 accuracy (checked against exact products
// in the CPU tests of the scheme and on the GPU).
//
// Layout: every operand is sliced into 7 BF16 digit planes stored K-block major
// (the 7 planes of each 16-wide K block are [7][rows][16], so one TMA box reads
// contiguous runs), by one of two slicing kernels:
//   rows  the source rows are the stored rows (A = X of X M: one exponent per
//         source row, computed by the warp that slices the row);
//   cols  the source columns are the stored rows (A = X^T and B = Z of X^T Z,
//         B = M of X M: one exponent per source column, from a column-max pass
//         with atomicMax, then a tiled transpose).
// Operands that many products read (a Lanczos basis, a dense A) keep their planes
// in a cache that the owner extends block by block.
// The product kernel (one CTA per SM, 320 threads) is the TMA / tcgen05
// pipeline of the split-BF16 product: warp 0 loads 3-D boxes (16 K x rows x 7
// planes, 32-byte swizzle) of both operands into a 5-stage ring, warp 1 owns 512
// TMEM columns and issues the 10 MMAs of each stage from one thread, warps 2-9
// drain the accumulators (two warps per 32 TMEM lanes, 32 columns each).  Work
// units (output tile, 16-wide K block) are split evenly over one wave of CTAs,
// so no CTA runs a third tile while the others idle (314 tiles on 152 SMs would
// take three rounds for 2.07 rounds of work): a tile whose K range lies inside
// one CTA's share is written by its epilogue, the few tiles cut between CTAs
// leave partial tiles that a fix-up kernel adds in CTA order, so the result is
// deterministic.  Every mbarrier wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "tc_ptx.cuh"
#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

using namespace tcx;

constexpr int kOzDig = 7;                                   // digits per operand entry
constexpr int kOzM = 128;                                   // output rows per tile (TMEM lanes)
constexpr int kOzN = 64;                                    // output columns per tile
constexpr int kOzBK = 16;                                   // K per stage (one 32-byte row, one MMA)
constexpr int kOzRowB = 2 * kOzBK;
constexpr int kOzStages = 5;
constexpr int kOzPlaneA = kOzM * kOzRowB;                   // 4 KB
constexpr int kOzPlaneB = kOzN * kOzRowB;                   // 2 KB
constexpr int kOzStageBytes = kOzDig * (kOzPlaneA + kOzPlaneB);  // 42 KB
constexpr int kOzSmem = kOzStages * kOzStageBytes + 1024;
constexpr int kOzChunk = 8;          // K blocks per exact accumulation (128 k)
constexpr int kOzFlushChunks = 64;   // chunks between FP64 flushes of the integer sums (8192 k)
constexpr int kOzSlots = 7;          // accumulators: p + q = 0 .. 6
constexpr int kOzEpiWarps = 8;   // two per TMEM lane quarter, 32 columns each
constexpr int kOzThreads = 64 + 32 * kOzEpiWarps;
constexpr int kOzWave = 152;
constexpr int kOzTmemCols = 512;
constexpr int kOzNanExp = 1 << 20;      // exponent of a row holding Inf or NaN
constexpr int kOzZeroExp = -(1 << 20);  // exponent of a zero entry

// ---- digits ------------------------------------------------------------------
__device__ inline int oz_exp(double x) {
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    const int be = (int)((u >> 52) & 0x7FF);
    const uint64_t mant = u & ((1ull << 52) - 1);
    if (be == 0x7FF) return kOzNanExp;
    if (be == 0) return mant == 0 ? kOzZeroExp : (63 - __clzll((long long)mant)) - 1073;
    return be - 1022;
}

__device__ inline int oz_norm_exp(int e) { return e <= kOzZeroExp ? 0 : e; }

// round(x 2^(55 - e)) (ties away from zero) as balanced base-256 digits.
__device__ inline void oz_digits(double x, int e, int d[kOzDig]) {
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    const int be = (int)((u >> 52) & 0x7FF);
    uint64_t m = u & ((1ull << 52) - 1);
    int q = -1074;
    if (be != 0) {
        m |= 1ull << 52;
        q = be - 1075;
    }
    int64_t F = 0;
    if (be != 0x7FF && e < kOzNanExp && m != 0) {
        const int sh = q + 55 - e;  // <= 2 when |x| < 2^e
        if (sh >= 0) {
            F = (int64_t)(m << sh);
        } else if (sh > -54) {
            F = (int64_t)((m + (1ull << (-sh - 1))) >> (-sh));
        }
        if (u >> 63) F = -F;
    }
    int64_t r = F;
#pragma unroll
    for (int p = kOzDig - 1; p >= 1; --p) {
        const int lo = (int)((r + 128) & 255) - 128;
        d[p] = lo;
        r = (r - lo) >> 8;
    }
    d[0] = (int)r;
}

__device__ inline float oz_digit_scale(int p) { return __int_as_float((127 - 8 * p) << 23); }  // 2^(-8p)

__device__ inline __nv_bfloat162 oz_pack(int d0, int d1, int p) {
    const float s = oz_digit_scale(p);
    return __floats2bfloat162_rn((float)d0 * s, (float)d1 * s);  // exact: |d| <= 128
}

// Global layout of the digit planes: K-block major.  Element (digit p, stored row r,
// column k) of an operand with Ra allocated stored rows sits at
//   ((k / 16) * 7 + p) * Ra * 16 + r * 16 + k % 16,
// so the 7 planes of one 16-wide K block are [7][Ra][16] and a TMA box of 16 K x
// 128 rows x 7 planes reads 7 contiguous runs of 4 KB.  Columns past K up to the
// next multiple of 16 hold zeros.
__host__ __device__ inline int64_t oz_off(int64_t Ra, int64_t r, int64_t k, int p) {
    return ((k >> 4) * kOzDig + p) * Ra * 16 + r * 16 + (k & 15);
}
__host__ __device__ inline int64_t oz_k16(int64_t K) { return (K + 15) / 16 * 16; }

// Stores the digits of (x0, x1) at columns (k, k + 1), k even, of stored row r.
__device__ inline void oz_store_pair(__nv_bfloat16* planes, int64_t Ra, int64_t r, int64_t k, const int* da,
                                     const int* db) {
    __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(planes + oz_off(Ra, r, k, 0));
#pragma unroll
    for (int p = 0; p < kOzDig; ++p) dst[p * Ra * 8] = oz_pack(da[p], db[p], p);  // plane step Ra*16 elements
}

// Rows slicer: row i of S (R x K, lds) -> stored row i; one warp per row.
__global__ void __launch_bounds__(256, 4) oz_slice_rows_kernel(int64_t R, int64_t K, const double* __restrict__ S,
                                                            int64_t lds, __nv_bfloat16* __restrict__ planes,
                                                            int64_t Ra, int* __restrict__ eexp) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t K16 = oz_k16(K);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < R; i += nw) {
        const double* src = S + i * lds;
        int e = kOzZeroExp;
        for (int64_t k = lane; k < K; k += 32) e = max(e, oz_exp(src[k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        e = oz_norm_exp(e);
        if (lane == 0) eexp[i] = e;
        for (int64_t k = 2 * lane; k < K16; k += 64) {
            int da[kOzDig], db[kOzDig];
            oz_digits(k < K ? src[k] : 0.0, e, da);
            oz_digits(k + 1 < K ? src[k + 1] : 0.0, e, db);
            oz_store_pair(planes, Ra, i, k, da, db);
        }
    }
}

// Rows slicer with one fixed exponent e for every row (an orthonormal basis: every
// entry below 2^e in magnitude), over the columns [a0, a1) of S (R rows, lds), a0
// even and a1 a multiple of 16; columns from c1 on are written as zeros (a column
// a0 - 1 < c1 is sliced again with its own value).  A row holding an entry at or
// above 2^e, or Inf/NaN, gets the exponent of a non-finite row.
__global__ void __launch_bounds__(256) oz_slice_rows_fixed_kernel(int64_t R, int64_t a0, int64_t a1, int64_t c1,
                                                                  const double* __restrict__ S, int64_t lds,
                                                                  __nv_bfloat16* __restrict__ planes, int64_t Ra,
                                                                  int e, int* __restrict__ eexp) {
    const int64_t halfk = (a1 - a0) / 2;
    const int64_t tot = R * halfk;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / halfk, k = a0 + 2 * (t % halfk);
        const double x0 = k < c1 ? S[i * lds + k] : 0.0, x1 = k + 1 < c1 ? S[i * lds + k + 1] : 0.0;
        if (oz_exp(x0) > e || oz_exp(x1) > e) eexp[i] = kOzNanExp;
        int da[kOzDig], db[kOzDig];
        oz_digits(x0, e, da);
        oz_digits(x1, e, db);
        oz_store_pair(planes, Ra, i, k, da, db);
    }
}

// Zeros of columns [v, v16) of every stored row (rows layout; v16 a multiple of 16).
__global__ void oz_zero_cols_kernel(int64_t R, int64_t v, int64_t v16, __nv_bfloat16* __restrict__ planes,
                                    int64_t Ra) {
    const int64_t w = v16 - v;
    const int64_t tot = R * w * kOzDig;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(t % kOzDig);
        const int64_t rest = t / kOzDig;
        const int64_t i = rest / w, k = v + rest % w;
        planes[oz_off(Ra, i, k, p)] = __float2bfloat16_rn(0.0f);
    }
}

// Column maxima of the exponents of S (K x R, lds); upper: entries with k > j are zero.
__global__ void __launch_bounds__(256) oz_colmax_kernel(int64_t K, int64_t R, const double* __restrict__ S,
                                                        int64_t lds, int upper, int64_t rows_per,
                                                        int* __restrict__ eexp) {
    __shared__ int red[8][33];
    const int64_t j = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.y * rows_per, k1 = min(K, k0 + rows_per);
    int e = kOzZeroExp;
    if (j < R)
        for (int64_t k = k0 + threadIdx.y; k < k1; k += 8)
            if (!(upper && k > j)) e = max(e, oz_exp(S[k * lds + j]));
    red[threadIdx.y][threadIdx.x] = e;
    __syncthreads();
    if (threadIdx.y == 0 && j < R) {
#pragma unroll
        for (int y = 1; y < 8; ++y) e = max(e, red[y][threadIdx.x]);
        atomicMax(&eexp[j], e);
    }
}

// Cols slicer: column j of S (K x R, lds) -> stored row r0 + j, tiles of 64 k x 32 j,
// zeros past K up to the next multiple of 16.
__global__ void __launch_bounds__(256) oz_slice_cols_kernel(int64_t K, int64_t R, const double* __restrict__ S,
                                                            int64_t lds, int upper, const int* __restrict__ eexp,
                                                            __nv_bfloat16* __restrict__ planes, int64_t Ra,
                                                            int64_t r0) {
    __shared__ double tile[64][33];
    const int64_t k0 = (int64_t)blockIdx.x * 64, j0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 64; r += 8) {
        const int64_t k = k0 + r, j = j0 + tx;
        double v = 0.0;
        if (k < K && j < R && !(upper && k > j)) v = S[k * lds + j];
        tile[r][tx] = v;
    }
    __syncthreads();
    const int kp = tx;  // k pair within the tile
    const int64_t k = k0 + 2 * kp;
    if (k >= oz_k16(K)) return;
    for (int jj = ty; jj < 32; jj += 8) {
        const int64_t j = j0 + jj;
        if (j >= R) break;
        const int e = oz_norm_exp(eexp[j]);
        int da[kOzDig], db[kOzDig];
        oz_digits(tile[2 * kp][jj], e, da);
        oz_digits(tile[2 * kp + 1][jj], e, db);
        oz_store_pair(planes, Ra, r0 + j, k, da, db);
    }
}

__global__ void oz_fill_kernel(int64_t n, int v, int* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// ---- the product kernel ------------------------------------------------------
struct OzArgs {
    int64_t M, N, KB, tiles, totalg;  // totalg: (row tile, K block) units of one column tile
    int NT, Npad, G, Gg, maxseg;       // CTA c: column tile c % NT, unit group c / NT of Gg
    const int* ea;
    const int* eb;
    double* out;  // C (direct tiles)
    int64_t ldo;
    double alpha, beta;
    int symmetric;
    double* partial;  // [G][maxseg][128][64]
    int* status;
    long long max_wait;  // limit of one pipeline wait (SM clock cycles)
};

// First unit of group g: the (row tile, K block) units of a column tile are split
// evenly over Gg groups; the NT CTAs of a group (one per column tile) cover the same
// units at the same time, so the A planes they all read come from DRAM once.
__host__ __device__ inline int64_t oz_glo(int g, const OzArgs& a) {
    return (int64_t)g * a.totalg / a.Gg;
}

// C = 2^(ea + eb - 14) (hi 2^-32 + lo 2^-40) in FP64.
__device__ inline double oz_value(long long hi, int lo, int ea, int eb) {
    if (ea >= kOzNanExp || eb >= kOzNanExp) return __longlong_as_double(0x7ff8000000000000LL);
    const double x = fma((double)lo, 0.00390625, (double)hi);  // hi + lo 2^-8
    const int E = ea + eb - 46;
    if (E >= -1022 && E <= 1023) return x * __longlong_as_double((long long)(E + 1023) << 52);  // exact scaling
    return ldexp(x, E);
}

// The output rule: out = alpha v + beta out (beta == 0: no read); a symmetric
// product writes each pair (i, j), (j, i) once, from the entry with i <= j.
__device__ inline void oz_store(const OzArgs& a, int64_t i, int64_t j, double v) {
    if (a.symmetric) {
        if (i > j) return;
        a.out[i * a.ldo + j] = v;
        a.out[j * a.ldo + i] = v;
        return;
    }
    double* o = a.out + i * a.ldo + j;
    *o = (a.beta != 0.0) ? fma(a.beta, *o, a.alpha * v) : a.alpha * v;
}

__global__ void __launch_bounds__(kOzThreads, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzArgs a) {
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t bars[2 * kOzStages + 2 * kOzSlots + 1];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty = [&](int s) { return bar0 + 8u * (uint32_t)(kOzStages + s); };
    auto accf = [&](int g) { return bar0 + 8u * (uint32_t)(2 * kOzStages + g); };
    auto acce = [&](int g) { return bar0 + 8u * (uint32_t)(2 * kOzStages + kOzSlots + g); };
    const uint32_t drain = bar0 + 8u * (uint32_t)(2 * kOzStages + 2 * kOzSlots);
    volatile int* abort_flag = &s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x;
    const int ntc = c % a.NT, gc = c / a.NT;  // this CTA's column tile and unit group
    const int64_t lo = oz_glo(gc, a), hi = oz_glo(gc + 1, a);
    const int64_t KB = a.KB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kOzStages; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int g = 0; g < kOzSlots; ++g) {
            mbar_init(accf(g), 1);
            mbar_init(acce(g), 32 * kOzEpiWarps);
        }
        mbar_init(drain, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(&s_tmem), kOzTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t stage_tx = (uint32_t)(kOzDig * (kOzPlaneA + a.Npad * kOzRowB));

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer: both operands' 7 planes of one 32-wide K block per stage
            int64_t it = 0;
            bool ok = true;
            for (int64_t i = lo; i < hi && ok; ++i, ++it) {
                const int st = (int)(it % kOzStages);
                if (it >= kOzStages) ok = mbar_wait(empty(st), (uint32_t)(((it / kOzStages) - 1) & 1), abort_flag, a.max_wait);
                if (!ok) break;
                const int64_t mt = i / KB;
                const int kz = (int)((i - mt * KB) * kOzDig);  // the 7 planes of K block i - mt KB
                const int nt = ntc;
                const uint32_t sA = base + (uint32_t)st * kOzStageBytes;
                mbar_arrive_expect_tx(full(st), stage_tx);
                tma_load_3d(sA, &tmA, 0, mt * kOzM, kz, full(st));
                tma_load_3d(sA + kOzDig * kOzPlaneA, &tmB, 0, nt * kOzN, kz, full(st));
            }
            if (!ok) {
                atomicOr(&a.status[kStTimeout], 1);
                s_abort = 1;
            }
            const int64_t first = it > kOzStages ? it - kOzStages : 0;
            for (int64_t j = first; j < it; ++j) mbar_drain(full((int)(j % kOzStages)), (uint32_t)((j / kOzStages) & 1));
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            const uint32_t bstep = (uint32_t)(a.Npad * kOzRowB) >> 4;  // one B plane in 16-byte units
            int64_t it = 0, ch = 0;  // K blocks and chunks issued by this CTA
            bool ok = true;
            for (int64_t i = lo; i < hi && ok;) {
                const int64_t mt = i / KB;
                const int64_t e = min(hi, (mt + 1) * KB);
                for (; i < e && ok; ++ch) {
                    const int64_t ce = min(e, i + kOzChunk);
                    for (int64_t i0 = i; i < ce; ++i, ++it) {
                        const int st = (int)(it % kOzStages);
                        ok = mbar_wait(full(st), (uint32_t)((it / kOzStages) & 1), abort_flag, a.max_wait);
                        if (!ok) break;
                        fence_after();
                        const bool first_kb = (i == i0), last_kb = (i + 1 == ce);
                        const uint32_t sA = base + (uint32_t)st * kOzStageBytes;
                        const uint64_t a0 = sdesc_sw32(sA);
                        const uint64_t b0 = sdesc_sw32(sA + kOzDig * kOzPlaneA);
                        // Digit plane p of A meets B planes q = 0 .. 6 - p; their products go to
                        // the accumulators of p + q, which sit side by side in TMEM (slot d at
                        // column d Npad), and the B planes sit side by side in shared memory, so
                        // one MMA with N = (7 - p) Npad (cut at 256 columns) covers them all:
                        // 10 MMAs a stage instead of 28, each reading its A plane once.  Slot p is
                        // final once the MMAs of plane p are done (later planes start at p + 1).
#pragma unroll
                        for (int p = 0; p < kOzDig; ++p) {
                            const uint64_t ad = a0 + (uint64_t)(p * (kOzPlaneA >> 4));
#pragma unroll
                            for (int q0 = 0; q0 < kOzDig - p; q0 += 4) {
                                const int cnt = min(4, kOzDig - p - q0);  // slots p + q0 .. + cnt - 1
                                const bool piece_ok = cnt * a.Npad <= 256;
                                if (first_kb && ch > 0 && p == 0) {
                                    // the epilogue has drained these accumulators of the previous chunk
                                    for (int dd = q0; dd < q0 + cnt && ok; ++dd) {
                                        ok = mbar_wait(acce(dd), (uint32_t)((ch - 1) & 1), abort_flag, a.max_wait);
                                    }
                                    if (!ok) break;
                                    fence_after();
                                }
                                if (!piece_ok) continue;  // (Npad <= 64 and cnt <= 4 keep N <= 256)
                                const uint32_t d = tmem + (uint32_t)((p + q0) * a.Npad);
                                const uint64_t bd = b0 + (uint64_t)(q0 * bstep);
                                mma_bf16(d, ad, bd, idesc_bf16(kOzM, cnt * a.Npad), (first_kb && p == 0) ? 0u : 1u);
                            }
                            if (!ok) break;
                            if (last_kb) commit(accf(p));
                        }
                        if (!ok) break;
                        commit(empty(st));
                    }
                }
            }
            if (!ok) {
                atomicOr(&a.status[kStTimeout], 1);
                s_abort = 1;
            }
            commit(drain);
            mbar_drain(drain, 0);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 and 32 of the columns
        const int quarter = warp & 3;
        const int cg = (warp - 2) >> 2;        // column half: columns 32 cg .. 32 cg + 31
        const int ncol = a.Npad >> 1;          // 16 or 32 valid columns in this half
        const int r = quarter * 32 + lane;
        const uint32_t tlane = (uint32_t)(quarter * 32) << 16;
        int64_t ch = 0;
        int seg = 0;
        bool ok = true;
        for (int64_t i = lo; i < hi && ok; ++seg) {
            const int64_t mt = i / KB;
            const int64_t e = min(hi, (mt + 1) * KB);
            const int nt = ntc;
            const int64_t row = (int64_t)mt * kOzM + r;
            const int64_t col0 = (int64_t)nt * kOzN + cg * ncol;
            const bool direct = (i == mt * KB) && (e == (mt + 1) * KB) && KB <= (int64_t)kOzChunk * kOzFlushChunks;
            const int ea = row < a.M ? a.ea[row] : 0;
            double* slot = a.partial + (((int64_t)c * a.maxseg + seg) * kOzM + r) * kOzN + cg * ncol;
            // integer sums of the digit products: hi in units of 2^-32 (p + q <= 4, exact),
            // lo in units of 2^-40 (p + q = 5 exact, p + q = 6 rounded to 2^-40)
            long long hi[32];
            int lo[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0;
            int nchunks = 0;
            bool stored = false;
            for (; i < e && ok; ++ch) {
                const int64_t ce = min(e, i + kOzChunk);
#pragma unroll
                for (int g = 0; g < kOzSlots; ++g) {
                    int w_ok = 1;
                    if (lane == 0) w_ok = mbar_wait_sleep(accf(g), (uint32_t)(ch & 1), abort_flag, a.max_wait) ? 1 : 0;
                    w_ok = __shfl_sync(0xffffffffu, w_ok, 0);
                    if (!w_ok) {
                        if (lane == 0) {
                            atomicOr(&a.status[kStTimeout], 1);
                            s_abort = 1;
                        }
                        ok = false;
                        break;
                    }
                    fence_after();
                    // slot g holds T_g 2^(-8g), T_g an integer below 2^24: read it in one
                    // load and hand the accumulator back before converting, so the next
                    // chunk's products into it need not wait for the conversion
                    const uint32_t taddr = tmem + tlane + (uint32_t)(g * a.Npad + cg * ncol);
                    float v[32];
                    if (ncol == 32)
                        tmem_ld32(taddr, v);
                    else
                        tmem_ld16(taddr, v);
                    fence_before();
                    mbar_arrive(acce(g));
                    const float mul = oz_digit_scale(-g);
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        if (q < ncol) {
                            if (g <= 4)
                                hi[q] += (long long)__float2int_rn(v[q] * mul) << (8 * (4 - g));
                            else if (g == 5)
                                lo[q] += __float2int_rn(v[q] * mul);
                            else
                                lo[q] += (__float2int_rn(v[q] * mul) + 128) >> 8;
                        }
                    }
                }
                if (!ok) break;
                i = ce;
                ++nchunks;
                const bool seg_end = (i == e);
                if (!(seg_end || nchunks % kOzFlushChunks == 0)) continue;
                if (direct) {
                    // the whole tile's K range in this CTA: the final output
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int64_t col = col0 + j;
                        if (j < ncol && row < a.M && col < a.N)
                            oz_store(a, row, col, oz_value(hi[j], lo[j], ea, a.eb[col]));
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int64_t col = col0 + j;
                        if (j < ncol) {
                            const double v = (row < a.M && col < a.N) ? oz_value(hi[j], lo[j], ea, a.eb[col]) : 0.0;
                            slot[j] = stored ? slot[j] + v : v;
                        }
                        hi[j] = lo[j] = 0;
                    }
                    stored = true;
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, kOzTmemCols);
    }
}

// Tiles whose K range is split over CTAs (or longer than one 64-bit
// accumulation): the parts are added in CTA order and the output rule applied.
__global__ void oz_fixup_kernel(OzArgs a) {
    __shared__ int s_g0, s_g1;
    const int64_t t = blockIdx.y;
    const int64_t KB = a.KB;
    const int mt = (int)(t / a.NT), nt = (int)(t % a.NT);
    if (threadIdx.x == 0) {
        auto group_of = [&](int64_t u) {
            int g = (int)(u * a.Gg / a.totalg);
            while (g + 1 < a.Gg && oz_glo(g + 1, a) <= u) ++g;
            while (g > 0 && oz_glo(g, a) > u) --g;
            return g;
        };
        s_g0 = group_of((int64_t)mt * KB);
        s_g1 = group_of((int64_t)(mt + 1) * KB - 1);
    }
    __syncthreads();
    if (s_g0 == s_g1 && KB <= (int64_t)kOzChunk * kOzFlushChunks) return;  // written by its CTA
    // the partial tile of each contributing CTA (column tile nt of groups g0..g1, in order)
    __shared__ int64_t s_slot[kOzWave];
    const int nc = s_g1 - s_g0 + 1;
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        const int g = s_g0 + j;
        const int cc = g * a.NT + nt;
        const int seg = (int)(mt - oz_glo(g, a) / KB);
        s_slot[j] = ((int64_t)cc * a.maxseg + seg) * kOzM * kOzN;
    }
    __syncthreads();
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kOzM * kOzN) return;
    const int r = idx / kOzN, cl = idx % kOzN;
    const int64_t row = (int64_t)mt * kOzM + r, col = (int64_t)nt * kOzN + cl;
    if (row >= a.M || col >= a.N) return;
    // eight loads in flight, added in CTA order (the same sum as a sequential loop)
    double acc = 0.0;
    int j = 0;
    for (; j + 8 <= nc; j += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = a.partial[s_slot[j + u] + idx];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
    }
    for (; j < nc; ++j) acc += a.partial[s_slot[j] + idx];
    oz_store(a, row, col, acc);
}

// ---- host side -------------------------------------------------------------------
struct OzPlan {
    int64_t M, N, K, KB, tiles, totalg;
    int MT, NT, Npad, G, Gg, maxseg;
};

OzPlan oz_plan(int64_t M, int64_t N, int64_t K) {
    OzPlan p{};
    p.M = M;
    p.N = N;
    p.K = K;
    p.MT = (int)((M + kOzM - 1) / kOzM);
    p.NT = (int)((N + kOzN - 1) / kOzN);
    p.Npad = N <= 32 ? 32 : kOzN;
    p.KB = std::max<int64_t>(1, (K + kOzBK - 1) / kOzBK);
    p.tiles = (int64_t)p.MT * p.NT;
    p.totalg = (int64_t)p.MT * p.KB;
    p.Gg = (int)std::max<int64_t>(1, std::min<int64_t>(kOzWave / p.NT, p.totalg));
    p.G = p.Gg * p.NT;
    p.maxseg = 1;
    OzArgs a{};
    a.KB = p.KB;
    a.tiles = p.tiles;
    a.totalg = p.totalg;
    a.G = p.G;
    a.Gg = p.Gg;
    for (int g = 0; g < p.Gg; ++g) {
        const int64_t lo = oz_glo(g, a), hi = oz_glo(g + 1, a);
        if (hi > lo) p.maxseg = std::max<int>(p.maxseg, (int)((hi - 1) / p.KB - lo / p.KB + 1));
    }
    return p;
}

inline size_t oz_planes_bytes(int64_t rows, int64_t K) {
    return align256((size_t)kOzDig * (size_t)rows * (size_t)oz_k16(K) * 2);
}

// 3-D tensor map of one operand: dims {16, rows, 7 x K blocks}, strides {32 B,
// Ra x 32 B}, box 16 x box_rows x 7, 32-byte swizzle (rows past `rows` read zeros).
bool make_oz_map(CUtensorMap* map, const void* planes, int64_t rows, int64_t Ra, int64_t K, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {16, (cuuint64_t)rows, (cuuint64_t)(kOzDig * (oz_k16(K) / 16))};
    const cuuint64_t strides[2] = {32, (cuuint64_t)Ra * 32};
    const cuuint32_t box[3] = {16u, (cuuint32_t)box_rows, (cuuint32_t)kOzDig};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(planes), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
inline size_t oz_partial_bytes(const OzPlan& p) {
    return align256(sizeof(double) * (size_t)p.G * p.maxseg * kOzM * kOzN);
}

// One operand of the product kernel: `rows` stored rows of K digits each in the
// K-block-major layout with Ra allocated stored rows, one exponent per stored row.
struct OzView {
    const __nv_bfloat16* planes;
    int64_t rows, K, Ra;
    const int* exps;
};

int oz_slice_rows(tsvd_handle* h, int64_t R, int64_t K, const double* S, int64_t lds, __nv_bfloat16* planes,
                  int* eexp, cudaStream_t st) {
    if (R == 0) return TSVD_OK;
    const int64_t blocks = std::min<int64_t>((R + 7) / 8, (int64_t)h->sm_count * 16);
    h->launches++;
    oz_slice_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(R, K, S, lds, planes, R, eexp);
    TSVD_TRY_CUDA(cudaGetLastError());
    return TSVD_OK;
}

// Ra: allocated stored rows of `planes` (default R); r0: first stored row written.
int oz_slice_cols(tsvd_handle* h, int64_t K, int64_t R, const double* S, int64_t lds, bool upper,
                  __nv_bfloat16* planes, int* eexp, cudaStream_t st, int64_t Ra = -1, int64_t r0 = 0) {
    if (R == 0) return TSVD_OK;
    if (Ra < 0) Ra = R;
    const unsigned gx = (unsigned)((R + 31) / 32);
    int64_t gy = std::min<int64_t>((K + 255) / 256, std::max<int64_t>(1, (int64_t)h->sm_count * 8 / gx));
    const int64_t rows_per = (K + gy - 1) / gy;
    gy = (K + rows_per - 1) / rows_per;
    h->launches += 3;
    oz_fill_kernel<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(R, kOzZeroExp - 1, eexp);
    oz_colmax_kernel<<<dim3(gx, (unsigned)std::max<int64_t>(1, gy)), dim3(32, 8), 0, st>>>(K, R, S, lds,
                                                                                           upper ? 1 : 0, rows_per,
                                                                                           eexp);
    const dim3 sg((unsigned)((oz_k16(K) + 63) / 64), gx);
    oz_slice_cols_kernel<<<sg, 256, 0, st>>>(K, R, S, lds, upper ? 1 : 0, eexp, planes, Ra, r0);
    TSVD_TRY_CUDA(cudaGetLastError());
    return TSVD_OK;
}

int oz_run(tsvd_handle* h, const OzPlan& p, const OzView& va, const OzView& vb, double* partial, double* out,
           int64_t ldo, double alpha, double beta, bool symmetric, int* status, cudaStream_t st) {
    if (p.tiles > 65535) return TSVD_ERR_UNSUPPORTED;  // one fix-up grid row per tile
    static thread_local int configured = -1;
    if (configured != h->device) {
        TSVD_TRY_CUDA(cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem));
        configured = h->device;
    }
    CUtensorMap mA, mB;
    if (!make_oz_map(&mA, va.planes, p.M, va.Ra, p.K, kOzM)) return TSVD_ERR_CUDA;
    if (!make_oz_map(&mB, vb.planes, p.N, vb.Ra, p.K, p.Npad)) return TSVD_ERR_CUDA;
    OzArgs a{};
    a.M = p.M;
    a.N = p.N;
    a.KB = p.KB;
    a.tiles = p.tiles;
    a.totalg = p.totalg;
    a.NT = p.NT;
    a.Npad = p.Npad;
    a.G = p.G;
    a.Gg = p.Gg;
    a.maxseg = p.maxseg;
    a.ea = va.exps;
    a.eb = vb.exps;
    a.out = out;
    a.ldo = ldo;
    a.alpha = alpha;
    a.beta = beta;
    a.symmetric = symmetric ? 1 : 0;
    a.partial = partial;
    a.status = status;
    a.max_wait = h->max_wait;
    h->launches++;
    oz_gemm_kernel<<<p.G, kOzThreads, kOzSmem, st>>>(mA, mB, a);
    TSVD_TRY_CUDA(cudaGetLastError());
    if (partial) {
        h->launches++;
        oz_fixup_kernel<<<dim3((kOzM * kOzN + 255) / 256, (unsigned)p.tiles), 256, 0, st>>>(a);
        TSVD_TRY_CUDA(cudaGetLastError());
    }
    return TSVD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
bool oz_worth(int64_t M, int64_t N, int64_t K) {
    // below ~30 MFLOP the FP64 pipe finishes before the slicing passes would
    const int64_t tiles = ((M + kOzM - 1) / kOzM) * ((N + kOzN - 1) / kOzN);
    return M > 0 && N > 0 && K >= 32 && tiles <= 65535 && N <= 65535 * 32 && 2.0 * (double)M * N * K >= 3.0e7;
}

size_t oz_ws_bound(int64_t qmax, int64_t smax, int64_t bmax) {
    // planes and exponents of the largest operands of either product, and split-K
    // partial tiles for at most (tiles + 2 per CTA of one wave) tiles
    const size_t tn = oz_planes_bytes(smax, qmax) + oz_planes_bytes(bmax, qmax);
    const size_t nn = oz_planes_bytes(qmax, smax) + oz_planes_bytes(bmax, smax);
    const size_t ex = align256(sizeof(int) * (size_t)(qmax + smax)) + align256(sizeof(int) * (size_t)(smax + bmax));
    const int64_t tiles = ((smax + kOzM - 1) / kOzM) * ((bmax + kOzN - 1) / kOzN);
    const size_t part = align256(sizeof(double) * (size_t)(tiles + 2 * kOzWave) * kOzM * kOzN);
    return std::max(tn, nn) + ex + part + 4096;
}

namespace {

OzView view_of(const __nv_bfloat16* planes, int64_t rows, int64_t K, const int* exps) {
    return OzView{planes, rows, K, rows, exps};
}

// The cached planes of columns [0, s) (cols layout: stored rows) or of the first s
// columns of every row (rows layout: K = s).
OzView view_of_cache(const OzCache& c, int64_t s) {
    return c.cols_layout ? OzView{c.planes, s, c.rows, c.cols, c.exps} : OzView{c.planes, c.rows, s, c.rows, c.exps};
}

}  // namespace

size_t oz_tn_ws(int64_t q, int64_t s, int64_t b, bool symmetric, bool cached_x) {
    const OzPlan p = oz_plan(s, b, q);
    Arena ar;
    if (!cached_x) {
        ar.take<char>(oz_planes_bytes(p.M, p.K));
        ar.take<int>((size_t)p.M);
    }
    if (!symmetric || cached_x) {
        ar.take<char>(oz_planes_bytes(p.N, p.K));
        ar.take<int>((size_t)p.N);
    }
    ar.take<char>(oz_partial_bytes(p));
    return ar.off;
}

size_t oz_nn_ws(int64_t q, int64_t s, int64_t b, bool cached_x) {
    const OzPlan p = oz_plan(q, b, s);
    Arena ar;
    if (!cached_x) {
        ar.take<char>(oz_planes_bytes(p.M, p.K));
        ar.take<int>((size_t)p.M);
    }
    ar.take<char>(oz_planes_bytes(p.N, p.K));
    ar.take<int>((size_t)p.N);
    ar.take<char>(oz_partial_bytes(p));
    return ar.off;
}

int oz_gemm_tn(tsvd_handle* h, int64_t q, int64_t s, int64_t b, const double* X, int64_t ldx, const double* Z,
               int64_t ldz, double* C, int64_t ldc, bool symmetric, void* ws, size_t ws_bytes, int* status,
               cudaStream_t st, const OzCache* xc) {
    const OzPlan p = oz_plan(s, b, q);
    Arena ar{static_cast<char*>(ws), ws_bytes, 0};
    OzView va{}, vb{};
    if (xc) {
        va = view_of_cache(*xc, s);
    } else {
        __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(ar.take<char>(oz_planes_bytes(p.M, p.K)));
        int* ea = ar.take<int>((size_t)p.M);
        if (!ar.fits()) return TSVD_ERR_WORKSPACE;
        TSVD_TRY(oz_slice_cols(h, q, s, X, ldx, false, pa, ea, st));
        va = view_of(pa, s, q, ea);
    }
    if (symmetric && !xc) {
        vb = va;
    } else {
        __nv_bfloat16* pb = reinterpret_cast<__nv_bfloat16*>(ar.take<char>(oz_planes_bytes(p.N, p.K)));
        int* eb = ar.take<int>((size_t)p.N);
        if (!ar.fits()) return TSVD_ERR_WORKSPACE;
        TSVD_TRY(oz_slice_cols(h, q, b, Z, ldz, false, pb, eb, st));
        vb = view_of(pb, b, q, eb);
    }
    const size_t pbytes = oz_partial_bytes(p);
    double* part = pbytes ? reinterpret_cast<double*>(ar.take<char>(pbytes)) : nullptr;
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    return oz_run(h, p, va, vb, part, C, ldc, 1.0, 0.0, symmetric, status, st);
}

int oz_gemm_nn(tsvd_handle* h, int64_t q, int64_t s, int64_t b, double alpha, const double* X, int64_t ldx,
               const double* Mm, int64_t ldm, double beta, double* Y, int64_t ldy, bool upper, void* ws,
               size_t ws_bytes, int* status, cudaStream_t st, const OzCache* xc) {
    const OzPlan p = oz_plan(q, b, s);
    Arena ar{static_cast<char*>(ws), ws_bytes, 0};
    OzView va{};
    if (xc) {
        va = view_of_cache(*xc, s);
    } else {
        __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(ar.take<char>(oz_planes_bytes(p.M, p.K)));
        int* ea = ar.take<int>((size_t)p.M);
        if (!ar.fits()) return TSVD_ERR_WORKSPACE;
        TSVD_TRY(oz_slice_rows(h, q, s, X, ldx, pa, ea, st));
        va = view_of(pa, q, s, ea);
    }
    __nv_bfloat16* pb = reinterpret_cast<__nv_bfloat16*>(ar.take<char>(oz_planes_bytes(p.N, p.K)));
    int* eb = ar.take<int>((size_t)p.N);
    const size_t pbytes = oz_partial_bytes(p);
    double* part = pbytes ? reinterpret_cast<double*>(ar.take<char>(pbytes)) : nullptr;
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    TSVD_TRY(oz_slice_cols(h, s, b, Mm, ldm, upper, pb, eb, st));
    return oz_run(h, p, va, view_of(pb, b, s, eb), part, Y, ldy, alpha, beta, false, status, st);
}

// ---- caches of operands that many products read ----------------------------------
size_t oz_cache_bytes(int64_t rows, int64_t cols, bool cols_layout) {
    Arena ar;
    OzCache c;
    oz_cache_carve(c, ar, nullptr, 0, rows, cols, cols_layout, kOzNoFixedExp);
    return ar.off;
}

void oz_cache_carve(OzCache& c, Arena& ar, const double* src, int64_t ld, int64_t rows, int64_t cols,
                    bool cols_layout, int fixed_exp) {
    c = OzCache{};
    c.src = src;
    c.ld = ld;
    c.rows = rows;
    c.cols = cols;
    c.cols_layout = cols_layout;
    c.fixed_exp = fixed_exp;
    const int64_t srows = cols_layout ? cols : rows, K = cols_layout ? rows : cols;
    c.planes = reinterpret_cast<__nv_bfloat16*>(ar.take<char>(oz_planes_bytes(srows, K)));
    c.exps = ar.take<int>((size_t)srows);
    c.valid = 0;
}

int oz_cache_slice(tsvd_handle* h, OzCache& c, int64_t c0, int64_t c1, cudaStream_t st) {
    if (c0 > c.valid || c1 > c.cols || c0 > c1) return TSVD_ERR_INVALID_ARG;
    if (c1 > c0) {
        if (c.cols_layout) {
            // stored rows [c0, c1): the columns' own exponents
            TSVD_TRY(oz_slice_cols(h, c.rows, c1 - c0, c.src + c0, c.ld, false, c.planes, c.exps + c0, st, c.cols,
                                   c0));
        } else if (c.fixed_exp != kOzNoFixedExp) {
            if (c0 == 0) {
                h->launches++;
                oz_fill_kernel<<<(unsigned)((c.rows + 255) / 256), 256, 0, st>>>(c.rows, c.fixed_exp, c.exps);
            }
            // the window with the rest of its last 16-wide K block (written as zeros)
            const int64_t a0 = c0 & ~int64_t(1), a1 = oz_k16(c1);
            const int64_t tot = c.rows * ((a1 - a0) / 2);
            const int64_t blocks = std::min<int64_t>((tot + 255) / 256, (int64_t)h->sm_count * 32);
            h->launches++;
            oz_slice_rows_fixed_kernel<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, st>>>(
                c.rows, a0, a1, c1, c.src, c.ld, c.planes, c.rows, c.fixed_exp, c.exps);
            TSVD_TRY_CUDA(cudaGetLastError());
        } else {
            // per-row exponents need the whole rows at once
            if (c0 != 0 || c1 != c.cols) return TSVD_ERR_INVALID_ARG;
            TSVD_TRY(oz_slice_rows(h, c.rows, c.cols, c.src, c.ld, c.planes, c.exps, st));
        }
    }
    c.valid = c1;
    return TSVD_OK;
}

int oz_cache_truncate(tsvd_handle* h, OzCache& c, int64_t v, cudaStream_t st) {
    if (v >= c.valid) return TSVD_OK;
    c.valid = v < 0 ? 0 : v;
    if (!c.cols_layout && c.valid % 16 != 0) {
        // a product of the first `valid` columns reads the whole last K block: zero its rest
        const int64_t tot = c.rows * (oz_k16(c.valid) - c.valid) * kOzDig;
        h->launches++;
        oz_zero_cols_kernel<<<(unsigned)std::min<int64_t>((tot + 255) / 256, (int64_t)h->sm_count * 32), 256, 0,
                              st>>>(c.rows, c.valid, oz_k16(c.valid), c.planes, c.rows);
        TSVD_TRY_CUDA(cudaGetLastError());
    }
    if (!c.cols_layout && c.fixed_exp != kOzNoFixedExp) {
        // a row's exponent may carry the mark of an entry out of range in the columns
        // dropped here (a block that was not orthonormal yet): start again from the
        // fixed exponent; the dropped columns are sliced again when rewritten
        h->launches++;
        oz_fill_kernel<<<(unsigned)((c.rows + 255) / 256), 256, 0, st>>>(c.rows, c.fixed_exp, c.exps);
        TSVD_TRY_CUDA(cudaGetLastError());
    }
    return TSVD_OK;
}

const OzCache* oz_find_cache(const tsvd_handle* h, const double* X, int64_t ldx, int64_t rows, int64_t s,
                             bool cols_layout) {
    for (const OzCache* c : h->oz_caches)
        if (c && c->src == X && c->ld == ldx && c->rows == rows && c->cols_layout == cols_layout && s <= c->valid &&
            // rows layout: the product reads whole 16-wide K blocks, zero past `valid` only
            (cols_layout || s == c->valid || s % 16 == 0))
            return c;
    return nullptr;
}

}  // namespace tsvd
