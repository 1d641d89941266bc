// Sparse kernels: CSR SpMM Y = A X with a tall-skinny dense block (Table 1 "SpMM",
// Alg. 1 S1/S3, Alg. 2 S2/S4) and the one-time build of CSR(A^T) that turns the
// A^T products into the same row-oriented kernel.
//
// FP64 on GB300 is bound by the FP64 pipe (2 DFMA/clk/SM), not by HBM: one
// warp owns one row, lanes own consecutive column pairs of the dense block
// (16-byte loads of each gathered X row), the row's (col, val) pairs are read
// 32 at a time cooperatively and broadcast with shuffles.  Every y_ij is
// accumulated in CSR order with FMA, so the result is deterministic.
#include <climits>

#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
    using type = double2;
};
template <>
struct Vec2<float> {
    using type = float2;
};

// NV = number of 2-element vectors per lane per column panel (panel width 64*NV).
template <typename T, int NV>
__global__ void __launch_bounds__(256) spmm_v2_kernel(int64_t m, int64_t n, const int32_t* __restrict__ rp,
                                                      const int32_t* __restrict__ ci,
                                                      const T* __restrict__ va, int w,
                                                      const T* __restrict__ X, int64_t ldx,
                                                      T* __restrict__ Y, int64_t ldy, int* status) {
    using V2 = typename Vec2<T>::type;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    const int beg = rp[row], end = rp[row + 1];
    for (int c0 = 0; c0 < w; c0 += 64 * NV) {
        T ax[NV], ay[NV];
#pragma unroll
        for (int t = 0; t < NV; ++t) ax[t] = ay[t] = T(0);
        for (int e0 = beg; e0 < end; e0 += 32) {
            const int e = e0 + lane;
            int myc = 0;
            T mya = T(0);
            if (e < end) {
                myc = ci[e];
                mya = va[e];
            }
            const int cnt = min(32, end - e0);
            for (int j = 0; j < cnt; ++j) {
                const int c = __shfl_sync(kFull, myc, j);
                const T a = __shfl_sync(kFull, mya, j);
                if ((uint64_t)(int64_t)c >= (uint64_t)n) {
                    if (lane == 0) atomicOr(&status[kStBadCsr], 1);
                    continue;
                }
                const T* xr = X + (int64_t)c * ldx + c0;
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    const int col = 2 * lane + 64 * t;
                    if (c0 + col + 1 < w) {
                        const V2 x = *reinterpret_cast<const V2*>(xr + col);
                        ax[t] = fma(a, x.x, ax[t]);
                        ay[t] = fma(a, x.y, ay[t]);
                    } else if (c0 + col < w) {
                        ax[t] = fma(a, xr[col], ax[t]);
                    }
                }
            }
        }
        T* yr = Y + row * ldy + c0;
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const int col = 2 * lane + 64 * t;
            if (c0 + col + 1 < w) {
                V2 v;
                v.x = ax[t];
                v.y = ay[t];
                *reinterpret_cast<V2*>(yr + col) = v;
            } else if (c0 + col < w) {
                yr[col] = ax[t];
            }
        }
    }
}

// Scalar variant for unaligned blocks: lane owns columns lane + 32 t.
template <typename T>
__global__ void __launch_bounds__(256) spmm_scalar_kernel(int64_t m, int64_t n, const int32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci,
                                                          const T* __restrict__ va, int w,
                                                          const T* __restrict__ X, int64_t ldx,
                                                          T* __restrict__ Y, int64_t ldy, int* status) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    const int beg = rp[row], end = rp[row + 1];
    for (int c0 = 0; c0 < w; c0 += 128) {
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int e0 = beg; e0 < end; e0 += 32) {
            const int e = e0 + lane;
            int myc = 0;
            T mya = T(0);
            if (e < end) {
                myc = ci[e];
                mya = va[e];
            }
            const int cnt = min(32, end - e0);
            for (int j = 0; j < cnt; ++j) {
                const int c = __shfl_sync(kFull, myc, j);
                const T a = __shfl_sync(kFull, mya, j);
                if ((uint64_t)(int64_t)c >= (uint64_t)n) {
                    if (lane == 0) atomicOr(&status[kStBadCsr], 1);
                    continue;
                }
                const T* xr = X + (int64_t)c * ldx + c0;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int col = lane + 32 * t;
                    if (c0 + col < w) acc[t] = fma(a, xr[col], acc[t]);
                }
            }
        }
        T* yr = Y + row * ldy + c0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int col = lane + 32 * t;
            if (c0 + col < w) yr[col] = acc[t];
        }
    }
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

template <typename T>
cudaError_t launch_spmm(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr,
                        const int32_t* col_idx, const T* val, int w, const T* X, int64_t ldx, T* Y,
                        int64_t ldy, int* status, cudaStream_t st) {
    if (m == 0 || w == 0) return cudaSuccess;
    // compulsory traffic: the CSR arrays, X and Y once each
    const double es = (double)sizeof(T);
    ProfScope prof(h, TSVD_K_APROD, 2.0 * nnz * w,
                   (4.0 + es) * nnz + 4.0 * (m + 1) + es * (double)n * w + es * (double)m * w, st);
    const unsigned blocks = (unsigned)((m + 7) / 8);
    const bool v2 = (ldx % 2 == 0) && (ldy % 2 == 0) && ((reinterpret_cast<uintptr_t>(X) & (2 * sizeof(T) - 1)) == 0) &&
                    ((reinterpret_cast<uintptr_t>(Y) & (2 * sizeof(T) - 1)) == 0);
    h->launches++;
    if (v2 && w <= 64) {
        spmm_v2_kernel<T, 1><<<blocks, 256, 0, st>>>(m, n, row_ptr, col_idx, val, w, X, ldx, Y, ldy, status);
    } else if (v2 && w <= 128) {
        spmm_v2_kernel<T, 2><<<blocks, 256, 0, st>>>(m, n, row_ptr, col_idx, val, w, X, ldx, Y, ldy, status);
    } else if (v2) {
        spmm_v2_kernel<T, 4><<<blocks, 256, 0, st>>>(m, n, row_ptr, col_idx, val, w, X, ldx, Y, ldy, status);
    } else {
        spmm_scalar_kernel<T><<<blocks, 256, 0, st>>>(m, n, row_ptr, col_idx, val, w, X, ldx, Y, ldy, status);
    }
    return cudaGetLastError();
}

template cudaError_t launch_spmm<double>(tsvd_handle*, int64_t, int64_t, int64_t, const int32_t*, const int32_t*,
                                         const double*, int, const double*, int64_t, double*, int64_t, int*,
                                         cudaStream_t);
template cudaError_t launch_spmm<float>(tsvd_handle*, int64_t, int64_t, int64_t, const int32_t*, const int32_t*,
                                        const float*, int, const float*, int64_t, float*, int64_t, int*,
                                        cudaStream_t);

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
