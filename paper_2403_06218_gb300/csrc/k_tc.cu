// Tensor-core product for dense A in the mixed-precision form: Y = A X with A
// and X each split into three BF16 pieces (A = A0 + A1 + A2 to 24 significant
// bits, the same for X) and the six cross terms A_i X_j with i + j <= 2
// accumulated in FP32 in tensor memory.  The dropped terms are O(2^-24) relative,
// so the product is as accurate as an FP32 product (the dense products of Alg. 1
// S1/S3 and Alg. 2 S2/S4 in the mixed form, whose accuracy the FP64 final
// Rayleigh-Ritz step relies on).
//
// Kernel structure (sm_103a, one CTA per SM, 320 threads):
//   warp 0     TMA producer: per 32-wide K block, one 3-D box of the three A
//              pieces (128 rows) and one of the three X^T pieces (Npad rows),
//              64-byte swizzled, into a 4-stage ring (48 KB a stage) guarded
//              by mbarriers;
//   warp 1     owns the TMEM allocation (256 columns: two 128 x Npad FP32
//              accumulators) and issues tcgen05.mma (M = 128, N = Npad, K = 16,
//              BF16 x BF16 -> FP32) from one thread, 12 per K block.  Each
//              accumulation covers only kTcChunk K blocks (48 MMAs), alternating
//              between the two accumulators;
//   warps 2-9  epilogue: tcgen05.ld of each finished accumulator (two warps per
//              32 TMEM lanes, half the columns each), added into FP32 registers
//              with round-to-nearest, and the tile part stored to a partial
//              buffer when its K range ends.
// The short accumulations matter: the tensor core's FP32 accumulation does not
// round to nearest, and over the few thousand MMAs of a 20,000-long inner
// dimension its error grew to about 3e-4 of the accumulated value on a
// diagonally dominant matrix (measured), while 48-MMA chunks summed on the CUDA
// cores keep the product at FP32 accuracy.
// Work split: the (tile, K block) iterations are divided evenly over a fixed
// number of CTAs (152: one wave on a GB300) so that every SM gets the same
// share however the tile count falls; a CTA that covers parts of several tiles
// writes one partial tile per part, and a fix-up kernel adds the parts of each
// tile in CTA order (deterministic).
//
// Every mbarrier wait is bounded (clock64); a wait that gives up raises the
// timeout status word, makes the other roles stop, drains the copies and
// products in flight (bounded too) and frees the tensor memory before exit.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "tc_ptx.cuh"
#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

constexpr int kTcM = 128;                          // A rows per tile = TMEM lanes
constexpr int kTcBK = 32;                          // K per stage: 32 BF16 = one 64-byte row
constexpr int kTcRowB = kTcBK * 2;                 // bytes of one tile row
constexpr int kTcStages = 4;
constexpr int kTcPieceA = kTcM * kTcRowB;          // one A piece per stage: 8 KB
constexpr int kTcMaxN = 128;
constexpr int kTcStageBytes = 3 * kTcPieceA + 3 * kTcMaxN * kTcRowB;  // 48 KB
constexpr int kTcSmem = kTcStages * kTcStageBytes + 1024;               // + alignment slack
constexpr int kTcChunk = 4;                         // K blocks per tensor-memory accumulation
constexpr int kTcEpiWarps = 8;                      // two per TMEM lane quarter, half the columns each
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;
constexpr int kTcWave = 152;
constexpr int kTcTmemCols = 256;
constexpr long long kTcMaxWait = tcx::kMaxWait;

using namespace tcx;

struct TcPlan {
    int64_t tiles, kb, total;  // row tiles, K blocks per tile, tiles x kb
    int ctas, maxseg;
};

__host__ __device__ inline int64_t tc_lo(int64_t c, int64_t total, int G) { return c * total / G; }

// ---- the product kernel ----------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX, int Npad,
                   int64_t KB, int64_t total, int G, int maxseg, float* __restrict__ partial, int* status,
                   long long max_wait) {
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t bars[2 * kTcStages + 5];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty = [&](int s) { return bar0 + 8u * (uint32_t)(kTcStages + s); };
    auto accf = [&](int a) { return bar0 + 8u * (uint32_t)(2 * kTcStages + a); };
    auto acce = [&](int a) { return bar0 + 8u * (uint32_t)(2 * kTcStages + 2 + a); };
    const uint32_t drain = bar0 + 8u * (uint32_t)(2 * kTcStages + 4);
    volatile int* abort_flag = &s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x;
    const int64_t lo = tc_lo(c, total, G), hi = tc_lo(c + 1, total, G);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf(a), 1);
            mbar_init(acce(a), 32 * kTcEpiWarps);
        }
        mbar_init(drain, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t stage_tx = (uint32_t)(3 * kTcPieceA + 3 * Npad * kTcRowB);

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            int64_t it = 0;
            bool ok = true;
            for (int64_t i = lo; i < hi && ok; ++i, ++it) {
                const int st = (int)(it % kTcStages);
                if (it >= kTcStages) ok = mbar_wait(empty(st), (uint32_t)(((it / kTcStages) - 1) & 1), abort_flag, max_wait);
                if (!ok) break;
                const int64_t t = i / KB;
                const int kx = (int)((i - t * KB) * kTcBK);
                const uint32_t sA = base + (uint32_t)st * kTcStageBytes;
                mbar_arrive_expect_tx(full(st), stage_tx);
                tma_load_3d(sA, &tmA, kx, (int)(t * kTcM), 0, full(st));
                tma_load_3d(sA + 3 * kTcPieceA, &tmX, kx, 0, 0, full(st));
            }
            if (!ok) {
                atomicOr(&status[kStTimeout], 1);
                s_abort = 1;
            }
            // copies in flight land before the CTA can exit
            const int64_t first = it > kTcStages ? it - kTcStages : 0;
            for (int64_t j = first; j < it; ++j) {
                const long long t0 = clock64();
                while (!mbar_try_wait(full((int)(j % kTcStages)), (uint32_t)((j / kTcStages) & 1)))
                    if (clock64() - t0 > kTcMaxWait) break;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: one accumulation per chunk of kTcChunk K blocks, alternating
            // between the two accumulators so that the epilogue drains one while the
            // other fills
            const uint32_t idesc = idesc_bf16(kTcM, Npad);
            // the six cross terms (A piece, X piece) kept by the split product
            constexpr int kTermA[6] = {0, 0, 1, 0, 1, 2};
            constexpr int kTermX[6] = {0, 1, 0, 2, 1, 0};
            int64_t it = 0, g = 0;  // K blocks and chunks issued by this CTA
            bool ok = true;
            for (int64_t i = lo; i < hi && ok;) {
                const int64_t t = i / KB;
                const int64_t e = min(hi, (t + 1) * KB);
                for (; i < e && ok; ++g) {
                    const int64_t ce = min(e, i + kTcChunk);
                    const int a = (int)(g & 1);
                    if (g >= 2) {
                        ok = mbar_wait(acce(a), (uint32_t)(((g >> 1) - 1) & 1), abort_flag, max_wait);
                        if (!ok) break;
                        fence_after();
                    }
                    const uint32_t d = tmem + (uint32_t)(a * kTcMaxN);
                    uint32_t acc = 0;
                    for (; i < ce; ++i, ++it) {
                        const int st = (int)(it % kTcStages);
                        ok = mbar_wait(full(st), (uint32_t)((it / kTcStages) & 1), abort_flag, max_wait);
                        if (!ok) break;
                        fence_after();
                        const uint32_t sA = base + (uint32_t)st * kTcStageBytes;
                        const uint32_t sX = sA + 3 * kTcPieceA;
#pragma unroll
                        for (int kk = 0; kk < kTcBK / 16; ++kk) {
#pragma unroll
                            for (int tm = 0; tm < 6; ++tm) {
                                const uint64_t ad = sdesc_sw64(sA + (uint32_t)(kTermA[tm] * kTcPieceA + kk * 32));
                                const uint64_t bd =
                                    sdesc_sw64(sX + (uint32_t)(kTermX[tm] * Npad * kTcRowB + kk * 32));
                                mma_bf16(d, ad, bd, idesc, acc);
                                acc = 1;
                            }
                        }
                        commit(empty(st));
                    }
                    if (!ok) break;
                    commit(accf(a));
                }
            }
            if (!ok) {
                atomicOr(&status[kStTimeout], 1);
                s_abort = 1;
            }
            // every product issued has finished before the tensor memory is freed
            commit(drain);
            const long long t0 = clock64();
            while (!mbar_try_wait(drain, 0))
                if (clock64() - t0 > kTcMaxWait) break;
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 and one half of the
        // columns; each chunk's accumulator is added into FP32 registers (round to
        // nearest, unlike the tensor core's accumulation) and each finished tile part
        // is stored as a partial tile
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int ncol = Npad >> 1;  // a multiple of 16
        const int row = quarter * 32 + lane;
        const uint32_t tlane = (uint32_t)(quarter * 32) << 16;
        int64_t g = 0;
        int seg = 0;
        bool ok = true;
        for (int64_t i = lo; i < hi && ok; ++seg) {
            const int64_t t = i / KB;
            const int64_t e = min(hi, (t + 1) * KB);
            float sum[kTcMaxN / 2];
#pragma unroll
            for (int j = 0; j < kTcMaxN / 2; ++j) sum[j] = 0.f;
            for (; i < e; i = min(e, i + kTcChunk), ++g) {
                const int a = (int)(g & 1);
                int w_ok = 1;
                if (lane == 0) w_ok = mbar_wait(accf(a), (uint32_t)((g >> 1) & 1), abort_flag, max_wait) ? 1 : 0;
                w_ok = __shfl_sync(0xffffffffu, w_ok, 0);
                if (!w_ok) {
                    if (lane == 0) {
                        atomicOr(&status[kStTimeout], 1);
                        s_abort = 1;
                    }
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t taddr = tmem + tlane + (uint32_t)(a * kTcMaxN + half * ncol);
#pragma unroll
                for (int c0 = 0; c0 < kTcMaxN / 2; c0 += 16) {
                    if (c0 < ncol) {
                        float v[16];
                        tmem_ld16(taddr + (uint32_t)c0, v);
#pragma unroll
                        for (int q = 0; q < 16; ++q) sum[c0 + q] += v[q];
                    }
                }
                fence_before();
                mbar_arrive(acce(a));
            }
            if (!ok) break;
            float* dst = partial + ((int64_t)(c * maxseg + seg) * kTcM + row) * Npad + half * ncol;
#pragma unroll
            for (int c0 = 0; c0 < kTcMaxN / 2; c0 += 4)
                if (c0 < ncol) reinterpret_cast<float4*>(dst)[c0 / 4] = make_float4(sum[c0], sum[c0 + 1], sum[c0 + 2], sum[c0 + 3]);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
    }
}

// Y[t*128 + r][col] = sum over the CTAs covering tile t (in CTA order) of their partial tile.
__global__ void tc_fixup_kernel(int64_t M, int w, int Npad, int64_t KB, int64_t total, int G, int maxseg,
                                const float* __restrict__ partial, float* __restrict__ Y, int64_t ldy) {
    __shared__ int s_c0, s_c1;
    const int64_t t = blockIdx.y;
    if (threadIdx.x == 0) {
        auto cta_of = [&](int64_t i) {
            int64_t cc = i * G / total;
            while (cc + 1 < G && tc_lo(cc + 1, total, G) <= i) ++cc;
            while (cc > 0 && tc_lo(cc, total, G) > i) --cc;
            return (int)cc;
        };
        s_c0 = cta_of(t * KB);
        s_c1 = cta_of((t + 1) * KB - 1);
    }
    __syncthreads();
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)kTcM * w) return;
    const int r = (int)(idx / w), col = (int)(idx % w);
    const int64_t row = t * kTcM + r;
    if (row >= M) return;
    float acc = 0.f;
    for (int cc = s_c0; cc <= s_c1; ++cc) {
        const int seg = (int)(t - tc_lo(cc, total, G) / KB);
        acc += partial[((int64_t)(cc * maxseg + seg) * kTcM + r) * Npad + col];
    }
    Y[row * ldy + col] = acc;
}

// Three-way BF16 split: p0 = bf16(v), p1 = bf16(v - p0), p2 = bf16(v - p0 - p1);
// each difference is exact in the source precision.
template <typename T>
__device__ inline void split3(T v, __nv_bfloat16& p0, __nv_bfloat16& p1, __nv_bfloat16& p2) {
    if constexpr (std::is_same<T, double>::value) {
        p0 = __double2bfloat16(v);
        const double r1 = v - (double)__bfloat162float(p0);
        p1 = __double2bfloat16(r1);
        const double r2 = r1 - (double)__bfloat162float(p1);
        p2 = __double2bfloat16(r2);
    } else {
        p0 = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(p0);
        p1 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(p1);
        p2 = __float2bfloat16_rn(r2);
    }
}

// Pieces of S (rows x cols, lds) or of its transpose: out[p][i][j] with the output
// rows x cols = (trans ? cols x rows : rows x cols), leading dimension ldo.
template <typename T>
__global__ void split3_kernel(int64_t rows, int64_t cols, const T* __restrict__ S, int64_t lds, int trans,
                              __nv_bfloat16* __restrict__ out, int64_t ldo, int64_t piece) {
    __shared__ T tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (!trans) {
        for (int k = ty; k < 32; k += 8) {
            const int64_t r = r0 + k, cc = c0 + tx;
            if (r < rows && cc < cols) {
                __nv_bfloat16 a, b, d;
                split3(S[r * lds + cc], a, b, d);
                out[r * ldo + cc] = a;
                out[piece + r * ldo + cc] = b;
                out[2 * piece + r * ldo + cc] = d;
            }
        }
        return;
    }
    for (int k = ty; k < 32; k += 8) {
        const int64_t r = r0 + k, cc = c0 + tx;
        tile[k][tx] = (r < rows && cc < cols) ? S[r * lds + cc] : T(0);
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int64_t orow = c0 + k, ocol = r0 + tx;  // output (transposed) coordinates
        if (orow < cols && ocol < rows) {
            __nv_bfloat16 a, b, d;
            split3(tile[tx][k], a, b, d);
            out[orow * ldo + ocol] = a;
            out[piece + orow * ldo + ocol] = b;
            out[2 * piece + orow * ldo + ocol] = d;
        }
    }
}

// ---- host side ---------------------------------------------------------------
// 3-D map over pieces [3][rows][ld] (BF16), box 32 (K) x box_rows x 3, 64-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, int64_t cols, int64_t rows, int64_t ld, int box_rows) {
    return make_plane_map(map, base, cols, rows, ld, box_rows, 3);
}

TcPlan tc_plan(int64_t rows, int64_t cols) {
    TcPlan p;
    p.tiles = (rows + kTcM - 1) / kTcM;
    p.kb = std::max<int64_t>(1, (cols + kTcBK - 1) / kTcBK);
    p.total = p.tiles * p.kb;
    p.ctas = (int)std::min<int64_t>(kTcWave, p.total);
    p.maxseg = 1;
    for (int c = 0; c < p.ctas; ++c) {
        const int64_t lo = tc_lo(c, p.total, p.ctas), hi = tc_lo(c + 1, p.total, p.ctas);
        if (hi > lo) p.maxseg = std::max<int>(p.maxseg, (int)((hi - 1) / p.kb - lo / p.kb + 1));
    }
    return p;
}

// N of the MMA: a multiple of 32 so that each epilogue half is a whole number of 16-column loads.
int npad_of(int w) { return std::min(kTcMaxN, (w + 31) / 32 * 32); }

}  // namespace

int64_t bf16x3_ld(int64_t cols) { return (cols + 7) / 8 * 8; }

size_t bf16x3_bytes(int64_t rows, int64_t cols) { return align256((size_t)3 * rows * bf16x3_ld(cols) * 2); }

template <typename T>
cudaError_t bf16x3_split(tsvd_handle* h, int64_t rows, int64_t cols, const T* S, int64_t lds, bool trans, void* out,
                         cudaStream_t st) {
    const int64_t orow = trans ? cols : rows, ocol = trans ? rows : cols;
    if (orow == 0 || ocol == 0) return cudaSuccess;
    const int64_t ldo = bf16x3_ld(ocol);
    const int64_t piece = orow * ldo;
    // the K padding of a row (ldo > ocol) is never read: the tensor maps stop at ocol
    h->launches++;
    const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    split3_kernel<T><<<grid, dim3(32, 8), 0, st>>>(rows, cols, S, lds, trans ? 1 : 0,
                                                   static_cast<__nv_bfloat16*>(out), ldo, piece);
    return cudaGetLastError();
}
template cudaError_t bf16x3_split<double>(tsvd_handle*, int64_t, int64_t, const double*, int64_t, bool, void*,
                                          cudaStream_t);
template cudaError_t bf16x3_split<float>(tsvd_handle*, int64_t, int64_t, const float*, int64_t, bool, void*,
                                         cudaStream_t);

size_t tc_mm_ws(int64_t rows, int64_t cols, int w) {
    const TcPlan p = tc_plan(rows, cols);
    const int np = npad_of(std::max(w, 1));
    return bf16x3_bytes(np, cols) + align256(sizeof(float) * (size_t)p.ctas * p.maxseg * kTcM * np);
}

cudaError_t tc_mm(tsvd_handle* h, int64_t rows, int64_t cols, const void* pieces, int w, const float* X, int64_t ldx,
                  float* Y, int64_t ldy, void* ws, int* status, cudaStream_t st) {
    if (rows == 0 || w == 0) return cudaSuccess;
    if (cols == 0) {
        for (int64_t i = 0; i < rows; ++i) {
            cudaError_t e = cudaMemsetAsync(Y + i * ldy, 0, sizeof(float) * w, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    static thread_local int configured = -1;
    if (configured != h->device) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
        if (e != cudaSuccess) return e;
        configured = h->device;
    }
    const TcPlan p = tc_plan(rows, cols);
    const int64_t lda = bf16x3_ld(cols);
    ProfScope prof(h, TSVD_K_APROD, 2.0 * rows * cols * w, 2.0 * 3 * rows * cols + 4.0 * (cols + rows) * w, st);
    for (int c0 = 0; c0 < w; c0 += kTcMaxN) {
        const int wp = std::min(kTcMaxN, w - c0);
        const int np = npad_of(wp);
        uint8_t* xp = static_cast<uint8_t*>(ws);
        float* part = reinterpret_cast<float*>(xp + bf16x3_bytes(np, cols));
        // X^T pieces: wp x cols (K-major), rows wp..np-1 come from the map's zero fill
        cudaError_t e = bf16x3_split<float>(h, cols, wp, X + c0, ldx, true, xp, st);
        if (e != cudaSuccess) return e;
        CUtensorMap mA, mX;
        if (!make_map(&mA, pieces, cols, rows, lda, kTcM)) return cudaErrorInvalidValue;
        if (!make_map(&mX, xp, cols, wp, bf16x3_ld(cols), np)) return cudaErrorInvalidValue;
        h->launches += 2;
        tc_gemm_kernel<<<p.ctas, kTcThreads, kTcSmem, st>>>(mA, mX, np, p.kb, p.total, p.ctas, p.maxseg, part,
                                                            status, h->max_wait);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const dim3 fg((unsigned)((kTcM * wp + 255) / 256), (unsigned)p.tiles);
        tc_fixup_kernel<<<fg, 256, 0, st>>>(rows, wp, np, p.kb, p.total, p.ctas, p.maxseg, part, Y + c0, ldy);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace tcx {

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

bool make_plane_map(CUtensorMap* map, const void* base, int64_t cols, int64_t rows, int64_t ld, int box_rows,
                    int planes, int box_k, int64_t pstride) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || (box_k != 32 && box_k != 16)) return false;
    if (pstride < 0) pstride = ld * rows;
    const cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)pstride * 2};
    const cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows, (cuuint32_t)planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, box_k == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tcx
}  // namespace tsvd
