// Sparse kernels: CSR SpMM Y = A X with a tall-skinny dense block (Table 1 "SpMM",
// Alg. 1 S1/S3, Alg. 2 S2/S4) and the one-time build of CSR(A^T) that turns the
// A^T products into the same row-oriented kernel.
//
// A sub-warp of G lanes owns one row; each lane gathers a 16-byte slice of every
// X row the row touches (float4 / double2), so G = w / (16 / sizeof(T)) lanes
// cover a block of w columns and narrow blocks put several rows in a warp.  The
// gathers (nnz w sizeof(T) bytes, from L2 for a block that fits there) bound the
// kernel, not the compulsory HBM bytes: measured ~13 TB/s of gathered data on
// GB300.  FP64 is also close to the FP64 pipe's rate (2 DFMA/clk/SM).  Every y_ij
// is accumulated in CSR order with FMA, so the result is deterministic.
//
// Long rows (power-law degrees; CSR(A^T) of a matrix with popular columns holds
// rows of up to ~10^6 entries) would leave one warp working long after the rest.
// A plan built once per matrix cuts every row longer than kSpmmChunk entries into
// chunks of kSpmmChunk: one warp per chunk writes a partial row, and a second
// kernel adds each row's partials in chunk order (still deterministic).
#include <climits>

#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

constexpr unsigned kFull = 0xffffffffu;


// VW consecutive values of the SpMM element type, loaded as one vector.
template <typename T, int VW>
struct VecLoad;
template <>
struct VecLoad<double, 2> {
    __device__ static void get(const double* p, double* o) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = v.x;
        o[1] = v.y;
    }
};
template <>
struct VecLoad<float, 4> {
    __device__ static void get(const float* p, float* o) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
};
template <typename T>
struct VecLoad<T, 1> {
    __device__ static void get(const T* p, T* o) { o[0] = __ldg(p); }
};

// One output row y = sum over the entries [beg, end) of a_e x_{col(e)}, written to
// out[0 .. w), by a sub-warp of G lanes: lane sl owns VW consecutive columns of each
// panel of VW G columns and gathers them with one vector load per entry (the
// entry's (col, val) is read by all G lanes: a broadcast).  Each y_ij is
// accumulated in CSR order with FMA, so the result is deterministic.
template <typename T, int VW, int G>
__device__ inline void spmm_segment(int64_t beg, int64_t end, int64_t n, const int32_t* __restrict__ ci,
                                    const T* __restrict__ va, int w, const T* __restrict__ X, int64_t ldx,
                                    T* __restrict__ out, int* status, int sl) {
    for (int c0 = 0; c0 < w; c0 += VW * G) {
        const int col = c0 + VW * sl;
        if (col >= w) continue;  // lanes past the last column of a narrow panel
        const bool full = col + VW <= w;
        T acc[VW];
#pragma unroll
        for (int q = 0; q < VW; ++q) acc[q] = T(0);
        for (int64_t e = beg; e < end; ++e) {
            const int c = __ldg(ci + e);
            const T a = __ldg(va + e);
            if ((uint64_t)(int64_t)c >= (uint64_t)n) {  // skipped, and reported
                if (sl == 0) atomicOr(&status[kStBadCsr], 1);
                continue;
            }
            const T* xr = X + (int64_t)c * ldx + col;
            T x[VW];
            if (full) {
                VecLoad<T, VW>::get(xr, x);
            } else {
#pragma unroll
                for (int q = 0; q < VW; ++q) x[q] = (col + q < w) ? __ldg(xr + q) : T(0);
            }
#pragma unroll
            for (int q = 0; q < VW; ++q) acc[q] = fma(a, x[q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < VW; ++q)
            if (col + q < w) out[col + q] = acc[q];
    }
}

// Sub-warp of G lanes per row; rows longer than `split` entries are left to the chunk kernels.
template <typename T, int VW, int G>
__global__ void __launch_bounds__(256) spmm_rows_kernel(int64_t m, int64_t n, const int32_t* __restrict__ rp,
                                                        const int32_t* __restrict__ ci, const T* __restrict__ va,
                                                        int w, const T* __restrict__ X, int64_t ldx,
                                                        T* __restrict__ Y, int64_t ldy, int64_t split, int* status) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int sl = threadIdx.x % G;
    if (row >= m) return;
    const int64_t beg = rp[row], end = rp[row + 1];
    if (end - beg > split) return;
    spmm_segment<T, VW, G>(beg, end, n, ci, va, w, X, ldx, Y + row * ldy, status, sl);
}

// Sub-warp per chunk of a long row: entries [rp[row] + j C, min(rp[row + 1], rp[row] + (j+1) C))
// into partial[chunk][0 .. w).
template <typename T, int VW, int G>
__global__ void __launch_bounds__(256) spmm_chunks_kernel(int64_t nchunks, const int4* __restrict__ chunks,
                                                          int64_t n, const int32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci, const T* __restrict__ va,
                                                          int w, const T* __restrict__ X, int64_t ldx,
                                                          T* __restrict__ partial, int64_t ldp, int* status) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int sl = threadIdx.x % G;
    if (c >= nchunks) return;
    const int4 d = chunks[c];
    const int64_t beg = (int64_t)rp[d.x] + (int64_t)d.y * kSpmmChunk;
    const int64_t end = min((int64_t)rp[d.x + 1], beg + kSpmmChunk);
    spmm_segment<T, VW, G>(beg, end, n, ci, va, w, X, ldx, partial + c * ldp, status, sl);
}

// Y[row] = sum of the row's chunk partials in chunk order (the first chunk's warp does the row).
template <typename T>
__global__ void __launch_bounds__(256) spmm_chunk_sum_kernel(int64_t nchunks, const int4* __restrict__ chunks,
                                                             int w, const T* __restrict__ partial, int64_t ldp,
                                                             T* __restrict__ Y, int64_t ldy) {
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= nchunks) return;
    const int4 d = chunks[c];
    if (d.y != 0) return;
    for (int col = lane; col < w; col += 32) {
        T acc = T(0);
        for (int t = 0; t < d.z; ++t) acc += partial[(c + t) * ldp + col];
        Y[(int64_t)d.x * ldy + col] = acc;
    }
}

// Plan: chunks of each row longer than kSpmmChunk entries.
__global__ void spmm_plan_count_kernel(int64_t m, const int32_t* __restrict__ rp, int32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t len = (int64_t)rp[i + 1] - rp[i];
    cnt[i] = len > kSpmmChunk ? (int32_t)((len + kSpmmChunk - 1) / kSpmmChunk) : 0;
}

__global__ void spmm_plan_fill_kernel(int64_t m, const int32_t* __restrict__ cnt, const int32_t* __restrict__ off,
                                      int4* __restrict__ chunks) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int32_t k = cnt[i];
    for (int32_t j = 0; j < k; ++j) chunks[off[i] + j] = make_int4((int)i, j, k, 0);
}

// ---- CSR transpose ---------------------------------------------------------

// Warp per row: validates the row's extent and columns, counts per column.
__global__ void csr_count_kernel(int64_t m, int64_t n, int64_t nnz, const int32_t* __restrict__ rp,
                                 const int32_t* __restrict__ ci, int32_t* __restrict__ cnt, int* status) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    const int64_t beg = rp[row], end = rp[row + 1];
    if (row == 0 && lane == 0 && beg != 0) atomicOr(&status[kStBadCsr], 1);
    if (row == m - 1 && lane == 0 && end != nnz) atomicOr(&status[kStBadCsr], 1);
    if (beg < 0 || end > nnz || beg > end) {
        if (lane == 0) atomicOr(&status[kStBadCsr], 1);
        return;
    }
    for (int64_t e = beg + lane; e < end; e += 32) {
        const int c = ci[e];
        if ((uint64_t)(int64_t)c >= (uint64_t)n) {
            atomicOr(&status[kStBadCsr], 1);
        } else {
            atomicAdd(&cnt[c], 1);
        }
    }
}

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

// Exclusive scan of a tile of cnt into out, tile total into bsum.
__global__ void __launch_bounds__(kScanThreads) scan_tile_kernel(int64_t n, const int32_t* __restrict__ cnt,
                                                                 int32_t* __restrict__ out,
                                                                 int32_t* __restrict__ bsum) {
    __shared__ int32_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int32_t v[kScanPer];
    int32_t run = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int64_t idx = base + i;
        v[i] = idx < n ? cnt[idx] : 0;
        const int32_t t = v[i];
        v[i] = run;
        run += t;
    }
    // inclusive warp scan of per-thread totals
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t inc = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    int32_t woff = 0;
    for (int i = 0; i < warp; ++i) woff += warp_tot[i];
    const int32_t toff = woff + inc - run;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int64_t idx = base + i;
        if (idx < n) out[idx] = v[i] + toff;
    }
    if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = woff + inc;
}

// Single CTA: exclusive scan of the tile totals in place (sequential carry over chunks).
__global__ void __launch_bounds__(1024) scan_sums_kernel(int64_t nb, int32_t* __restrict__ bsum) {
    __shared__ int32_t wt[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c0 = 0; c0 < nb; c0 += 1024) {
        const int64_t idx = c0 + threadIdx.x;
        const int32_t x = idx < nb ? bsum[idx] : 0;
        int32_t inc = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane == 31) wt[warp] = inc;
        __syncthreads();
        int32_t woff = 0;
        for (int i = 0; i < warp; ++i) woff += wt[i];
        const int32_t c = carry;
        if (idx < nb) bsum[idx] = c + woff + inc - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + woff + inc;
        __syncthreads();
    }
}

__global__ void scan_add_kernel(int64_t n, int32_t* __restrict__ out, const int32_t* __restrict__ bsum,
                                int32_t* __restrict__ cursor) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = out[i] + bsum[i / kScanTile];
    out[i] = v;
    cursor[i] = v;
}

// Warp per row: scatter (row, val) into the transposed arrays.
template <typename T>
__global__ void csr_scatter_kernel(int64_t m, int64_t n, int64_t nnz, const int32_t* __restrict__ rp,
                                   const int32_t* __restrict__ ci, const T* __restrict__ va,
                                   int32_t* __restrict__ cursor, int32_t* __restrict__ tci,
                                   T* __restrict__ tva) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    const int64_t beg = rp[row], end = rp[row + 1];
    if (beg < 0 || end > nnz || beg > end) return;
    for (int64_t e = beg + lane; e < end; e += 32) {
        const int c = ci[e];
        if ((uint64_t)(int64_t)c >= (uint64_t)n) continue;
        const int32_t pos = atomicAdd(&cursor[c], 1);
        tci[pos] = (int32_t)row;
        tva[pos] = va[e];
    }
}

// Segments of at most 32 entries: warp bitonic sort of (row, val) by row.
template <typename T>
__global__ void seg_sort_warp_kernel(int64_t n, const int32_t* __restrict__ trp, int32_t* __restrict__ tci,
                                     T* __restrict__ tva) {
    const int64_t seg = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (seg >= n) return;
    const int beg = trp[seg], len = trp[seg + 1] - beg;
    if (len <= 1 || len > 32) return;
    int key = lane < len ? tci[beg + lane] : INT_MAX;
    T val = lane < len ? tva[beg + lane] : T(0);
    for (int k = 2; k <= 32; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int okey = __shfl_xor_sync(kFull, key, j);
            const T oval = __shfl_xor_sync(kFull, val, j);
            const bool up = (lane & k) == 0 || k == 32;
            const bool lower = (lane & j) == 0;
            const bool take_other = (lower == up) ? (okey < key) : (okey > key);
            if (take_other) {
                key = okey;
                val = oval;
            }
        }
    }
    if (lane < len) {
        tci[beg + lane] = key;
        tva[beg + lane] = val;
    }
}

constexpr int kSegSmem = 4096;

// Segments of 33..4096 entries: one CTA, bitonic sort (all blocks ascending,
// first step of each merge compares i with i ^ (k-1)) in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) seg_sort_cta_kernel(int64_t n, const int32_t* __restrict__ trp,
                                                           int32_t* __restrict__ tci,
                                                           T* __restrict__ tva) {
    __shared__ int32_t sk[kSegSmem];
    __shared__ T sv[kSegSmem];
    for (int64_t seg = blockIdx.x; seg < n; seg += gridDim.x) {
        const int beg = trp[seg], len = trp[seg + 1] - beg;
        if (len <= 32 || len > kSegSmem) continue;
        int P = 64;
        while (P < len) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            sk[i] = i < len ? tci[beg + i] : INT_MAX;
            sv[i] = i < len ? tva[beg + i] : T(0);
        }
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    const int p = (j == (k >> 1)) ? (i ^ (k - 1)) : (i ^ j);
                    if (p > i && sk[p] < sk[i]) {
                        const int tk = sk[i];
                        sk[i] = sk[p];
                        sk[p] = tk;
                        const T tv = sv[i];
                        sv[i] = sv[p];
                        sv[p] = tv;
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            tci[beg + i] = sk[i];
            tva[beg + i] = sv[i];
        }
        __syncthreads();
    }
}

// Lists segments longer than kSegSmem and their maximal length.
__global__ void seg_heavy_kernel(int64_t n, const int32_t* __restrict__ trp, int32_t* __restrict__ list,
                                 int32_t* __restrict__ info /* [0] count, [1] max len */) {
    const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= n) return;
    const int len = trp[seg + 1] - trp[seg];
    if (len > kSegSmem) {
        const int slot = atomicAdd(&info[0], 1);
        list[slot] = (int32_t)seg;
        atomicMax(&info[1], len);
    }
}

// One comparator stage of the same bitonic network in global memory, for the
// long segments; comparators whose partner lies past the segment end are skipped
// (those slots act as +infinity and never move below the end).
template <typename T>
__global__ void seg_sort_global_stage(const int32_t* __restrict__ trp, const int32_t* __restrict__ list,
                                      int32_t* __restrict__ tci, T* __restrict__ tva, int k, int j,
                                      int64_t half_p) {
    const int seg = list[blockIdx.y];
    const int beg = trp[seg], len = trp[seg + 1] - beg;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < half_p;
         t += (int64_t)gridDim.x * blockDim.x) {
        // t-th comparator: i has bit log2(j) clear
        const int64_t i = ((t / j) * (2 * j)) + (t % j);
        const int64_t p = (j == (k >> 1)) ? (i ^ (int64_t)(k - 1)) : (i + j);
        const int64_t lo = i < p ? i : p, hi = i < p ? p : i;
        if (hi >= len) continue;
        const int a = tci[beg + lo], b = tci[beg + hi];
        if (b < a) {
            tci[beg + lo] = b;
            tci[beg + hi] = a;
            const T tv = tva[beg + lo];
            tva[beg + lo] = tva[beg + hi];
            tva[beg + hi] = tv;
        }
    }
}

__global__ void to_float_kernel(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

}  // namespace

cudaError_t convert_to_float(tsvd_handle* h, int64_t n, const double* x, float* y, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    h->launches++;
    to_float_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, x, y);
    return cudaGetLastError();
}

template <typename T, int VW, int G>
static void spmm_launch_all(int64_t m, int64_t n, const int32_t* rp, const int32_t* ci, const T* va, int w, const T* X,
                            int64_t ldx, T* Y, int64_t ldy, const SpmmPlan* plan, int* status, cudaStream_t st) {
    const bool split = plan && plan->nchunks > 0;
    const int64_t per_block = 256 / G;
    spmm_rows_kernel<T, VW, G><<<(unsigned)((m + per_block - 1) / per_block), 256, 0, st>>>(
        m, n, rp, ci, va, w, X, ldx, Y, ldy, split ? (int64_t)kSpmmChunk : INT64_MAX, status);
    if (!split) return;
    T* part = static_cast<T*>(plan->partial);
    const int64_t ldp = spmm_partial_ld(w);
    spmm_chunks_kernel<T, VW, G><<<(unsigned)((plan->nchunks + per_block - 1) / per_block), 256, 0, st>>>(
        plan->nchunks, plan->chunks, n, rp, ci, va, w, X, ldx, part, ldp, status);
    spmm_chunk_sum_kernel<T><<<(unsigned)((plan->nchunks + 7) / 8), 256, 0, st>>>(plan->nchunks, plan->chunks, w,
                                                                                  part, ldp, Y, ldy);
}

// Lanes per row: enough 16-byte slices to cover w, at most a warp (wider blocks loop over panels).
template <typename T, int VW>
static void spmm_dispatch(int64_t m, int64_t n, const int32_t* rp, const int32_t* ci, const T* va, int w, const T* X,
                          int64_t ldx, T* Y, int64_t ldy, const SpmmPlan* plan, int* status, cudaStream_t st) {
    const int slices = (w + VW - 1) / VW;
    if (slices <= 4)
        spmm_launch_all<T, VW, 4>(m, n, rp, ci, va, w, X, ldx, Y, ldy, plan, status, st);
    else if (slices <= 8)
        spmm_launch_all<T, VW, 8>(m, n, rp, ci, va, w, X, ldx, Y, ldy, plan, status, st);
    else if (slices <= 16)
        spmm_launch_all<T, VW, 16>(m, n, rp, ci, va, w, X, ldx, Y, ldy, plan, status, st);
    else
        spmm_launch_all<T, VW, 32>(m, n, rp, ci, va, w, X, ldx, Y, ldy, plan, status, st);
}

template <typename T>
cudaError_t launch_spmm(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr,
                        const int32_t* col_idx, const T* val, int w, const T* X, int64_t ldx, T* Y,
                        int64_t ldy, int* status, cudaStream_t st, const SpmmPlan* plan) {
    if (m == 0 || w == 0) return cudaSuccess;
    if (plan && plan->nchunks > 0 && w > plan->wmax) return cudaErrorInvalidValue;
    // compulsory traffic: the CSR arrays, X and Y once each
    const double es = (double)sizeof(T);
    ProfScope prof(h, TSVD_K_APROD, 2.0 * nnz * w,
                   (4.0 + es) * nnz + 4.0 * (m + 1) + es * (double)n * w + es * (double)m * w, st);
    // 16-byte gathers need 16-byte aligned X rows
    const bool v16 = (ldx * sizeof(T)) % 16 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    h->launches += (plan && plan->nchunks > 0) ? 3 : 1;
    if (v16)
        spmm_dispatch<T, 16 / sizeof(T)>(m, n, row_ptr, col_idx, val, w, X, ldx, Y, ldy, plan, status, st);
    else
        spmm_dispatch<T, 1>(m, n, row_ptr, col_idx, val, w, X, ldx, Y, ldy, plan, status, st);
    return cudaGetLastError();
}

size_t spmm_plan_ws(int64_t m, int64_t nnz, int wmax, size_t elem) {
    const int64_t maxc = spmm_max_chunks(nnz);
    Arena ar;
    ar.take<int32_t>(m + 1);                                     // chunks per row
    ar.take<int32_t>(m + 1);                                     // their exclusive scan
    ar.take<int32_t>(m + 1);                                     // scan cursor (unused copy)
    ar.take<int32_t>((m + kScanTile - 1) / kScanTile + 1);       // tile sums
    ar.take<int4>(maxc + 1);                                     // chunk descriptors
    ar.take<char>(elem * (size_t)(maxc + 1) * spmm_partial_ld(wmax));  // partial rows
    return ar.off;
}

int spmm_plan(tsvd_handle* h, int64_t m, int64_t nnz, const int32_t* rp, int wmax, size_t elem, Arena& ar,
              SpmmPlan* plan, cudaStream_t st) {
    const int64_t maxc = spmm_max_chunks(nnz);
    int32_t* cnt = ar.take<int32_t>(m + 1);
    int32_t* off = ar.take<int32_t>(m + 1);
    int32_t* cur = ar.take<int32_t>(m + 1);
    int32_t* bsum = ar.take<int32_t>((m + kScanTile - 1) / kScanTile + 1);
    int4* chunks = ar.take<int4>(maxc + 1);
    void* partial = ar.take<char>(elem * (size_t)(maxc + 1) * spmm_partial_ld(wmax));
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    plan->nchunks = 0;
    plan->chunks = chunks;
    plan->partial = partial;
    plan->wmax = wmax;
    if (m == 0 || nnz <= kSpmmChunk) return TSVD_OK;
    ProfScope prof(h, TSVD_K_OTHER, 0.0, 0.0, st);
    const int64_t nb = (m + kScanTile - 1) / kScanTile;
    h->launches += 5;
    spmm_plan_count_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, rp, cnt);
    scan_tile_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(m, cnt, off, bsum);
    scan_sums_kernel<<<1, 1024, 0, st>>>(nb, bsum);
    scan_add_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, off, bsum, cur);
    spmm_plan_fill_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, cnt, off, chunks);
    TSVD_TRY_CUDA(cudaGetLastError());
    // number of chunks = off[m-1] + cnt[m-1]
    int32_t last[2] = {0, 0};
    TSVD_TRY_CUDA(cudaMemcpyAsync(&last[0], off + (m - 1), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TSVD_TRY_CUDA(cudaMemcpyAsync(&last[1], cnt + (m - 1), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    plan->nchunks = (int64_t)last[0] + last[1];
    if (plan->nchunks > maxc) return TSVD_ERR_INVALID_ARG;  // row_ptr inconsistent with nnz
    return TSVD_OK;
}

template cudaError_t launch_spmm<double>(tsvd_handle*, int64_t, int64_t, int64_t, const int32_t*, const int32_t*,
                                         const double*, int, const double*, int64_t, double*, int64_t, int*,
                                         cudaStream_t, const SpmmPlan*);
template cudaError_t launch_spmm<float>(tsvd_handle*, int64_t, int64_t, int64_t, const int32_t*, const int32_t*,
                                        const float*, int, const float*, int64_t, float*, int64_t, int*,
                                        cudaStream_t, const SpmmPlan*);

size_t csr_transpose_ws(int64_t m, int64_t n, int64_t nnz) {
    (void)m;
    (void)nnz;
    Arena ar;
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    ar.take<int32_t>(n + 1);      // counts
    ar.take<int32_t>(n + 1);      // cursor
    ar.take<int32_t>(nb + 1);     // tile sums
    ar.take<int32_t>(n + 1);      // heavy list
    ar.take<int32_t>(4);          // heavy info
    return ar.off;
}

template <typename T>
int csr_transpose(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr,
                  const int32_t* col_idx, const T* val, int32_t* t_row_ptr, int32_t* t_col_idx,
                  T* t_val, Arena& ar, int* status, cudaStream_t st) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    int32_t* cnt = ar.take<int32_t>(n + 1);
    int32_t* cursor = ar.take<int32_t>(n + 1);
    int32_t* bsum = ar.take<int32_t>(nb + 1);
    int32_t* heavy = ar.take<int32_t>(n + 1);
    int32_t* hinfo = ar.take<int32_t>(4);
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    ProfScope prof(h, TSVD_K_OTHER, 0.0, 0.0, st);
    TSVD_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), st));
    TSVD_TRY_CUDA(cudaMemsetAsync(hinfo, 0, sizeof(int32_t) * 4, st));
    if (m > 0) {
        h->launches++;
        csr_count_kernel<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(m, n, nnz, row_ptr, col_idx, cnt, status);
        TSVD_TRY_CUDA(cudaGetLastError());
    }
    if (n > 0) {
        h->launches += 3;
        scan_tile_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(n, cnt, t_row_ptr, bsum);
        scan_sums_kernel<<<1, 1024, 0, st>>>(nb, bsum);
        scan_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, t_row_ptr, bsum, cursor);
        TSVD_TRY_CUDA(cudaGetLastError());
    }
    // t_row_ptr[n] = nnz (count of valid entries equals nnz when the CSR is valid)
    const int32_t nnz32 = (int32_t)nnz;
    TSVD_TRY_CUDA(cudaMemcpyAsync(t_row_ptr + n, &nnz32, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    int hs[kStCount];
    TSVD_TRY(read_status(st, status, hs));
    if (hs[kStBadCsr]) return TSVD_ERR_INVALID_ARG;
    if (m > 0) {
        h->launches++;
        csr_scatter_kernel<T><<<(unsigned)((m + 7) / 8), 256, 0, st>>>(m, n, nnz, row_ptr, col_idx, val, cursor,
                                                                   t_col_idx, t_val);
        TSVD_TRY_CUDA(cudaGetLastError());
    }
    if (n > 0) {
        h->launches += 3;
        seg_sort_warp_kernel<T><<<(unsigned)((n + 7) / 8), 256, 0, st>>>(n, t_row_ptr, t_col_idx, t_val);
        const unsigned cta_grid = (unsigned)(n < 4 * (int64_t)h->sm_count ? n : 4 * (int64_t)h->sm_count);
        seg_sort_cta_kernel<T><<<cta_grid, 256, 0, st>>>(n, t_row_ptr, t_col_idx, t_val);
        seg_heavy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, t_row_ptr, heavy, hinfo);
        TSVD_TRY_CUDA(cudaGetLastError());
        int32_t hh[2];
        TSVD_TRY_CUDA(cudaMemcpyAsync(hh, hinfo, sizeof(hh), cudaMemcpyDeviceToHost, st));
        TSVD_TRY_CUDA(cudaStreamSynchronize(st));
        if (hh[0] > 0) {
            int64_t P = 1;
            while (P < hh[1]) P <<= 1;
            const int64_t half_p = P / 2;
            const unsigned gx = (unsigned)((half_p + 255) / 256 < 1024 ? (half_p + 255) / 256 : 1024);
            for (int64_t k = 2; k <= P; k <<= 1) {
                for (int64_t j = k >> 1; j > 0; j >>= 1) {
                    h->launches++;
                    seg_sort_global_stage<T><<<dim3(gx, (unsigned)hh[0]), 256, 0, st>>>(
                        t_row_ptr, heavy, t_col_idx, t_val, (int)k, (int)j, half_p);
                }
            }
            TSVD_TRY_CUDA(cudaGetLastError());
        }
    }
    return TSVD_OK;
}

template int csr_transpose<double>(tsvd_handle*, int64_t, int64_t, int64_t, const int32_t*, const int32_t*,
                                   const double*, int32_t*, int32_t*, double*, Arena&, int*, cudaStream_t);
template int csr_transpose<float>(tsvd_handle*, int64_t, int64_t, int64_t, const int32_t*, const int32_t*,
                                  const float*, int32_t*, int32_t*, float*, Arena&, int*, cudaStream_t);

}  // namespace tsvd
