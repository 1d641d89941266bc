// Small SVD of the projected matrix (R_p of Alg. 1 S5, B_k of Alg. 2 S6) on the
// device: one-sided Jacobi (Hestenes 1958) on the columns of B, with the
// parallel round-robin ("tournament") pair ordering of Brent and Luk (1985) so
// that n/2 disjoint column pairs rotate at once.  The paper runs this step as
// LAPACK GESVD on the host; here it stays on the GPU so the iteration never
// leaves the device.
//
// Layout: G = B padded to an even number of columns with a zero column,
// column-major (ld = n rows); V = identity of order npad, column-major.  One
// warp owns one pair per round: it forms alpha = |g_p|^2, beta = |g_q|^2,
// gamma = g_p.g_q with a fixed shuffle tree, and if |gamma| > tol*sqrt(alpha*beta)
// applies the rotation with t = sign(zeta)/(|zeta| + hypot(1, zeta)),
// zeta = (beta - alpha)/(2 gamma) (Rutishauser's formulas) to both G and V.
// Rounds are separated by a grid barrier whose spin is bounded: on timeout it
// raises the status word and every CTA returns.  Sweeps repeat until one sweep
// rotates nothing (or kMaxSweeps).  Then sigma_j = |g_j|, columns are sorted by
// (sigma descending, index ascending), Ubar_j = g_j / sigma_j, Vbar_j = v_j, and
// each pair is sign-flipped so the largest-magnitude entry of Vbar_j is positive.
#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxSweeps = 40;
constexpr long long kMaxSpins = 1LL << 24;  // ~1 s with 64 ns naps

enum Ctl : int { kCtlCount = 0, kCtlGen = 1, kCtlErr = 2, kCtlSweeps = 3, kCtlRot = 8 };
constexpr int kCtlWords = kCtlRot + kMaxSweeps;

__device__ inline unsigned vload(const unsigned* p) { return *reinterpret_cast<const volatile unsigned*>(p); }

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).
// Returns false once any CTA has timed out.
__device__ bool grid_sync(unsigned* ctl) {
    if (gridDim.x == 1) {
        __syncthreads();
        return true;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = vload(&ctl[kCtlGen]);
        __threadfence();
        const unsigned prev = atomicAdd(&ctl[kCtlCount], 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(&ctl[kCtlCount], 0u);
            __threadfence();
            atomicAdd(&ctl[kCtlGen], 1u);
        } else {
            long long spins = 0;
            while (vload(&ctl[kCtlGen]) == g) {
                if (++spins > kMaxSpins) {
                    atomicOr(&ctl[kCtlErr], 1u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return vload(&ctl[kCtlErr]) == 0u;
}

__device__ inline double warp_sum(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

// Player at seat `seat` in round `rnd` of the round-robin on npad players.
__device__ inline int rr_player(int seat, int rnd, int npad) {
    return seat == 0 ? 0 : ((seat - 1 + rnd) % (npad - 1)) + 1;
}

__global__ void jacobi_init_kernel(int n, int npad, const double* __restrict__ B, int64_t ldb,
                                   double* __restrict__ G, double* __restrict__ V) {
    const int64_t tot = (int64_t)npad * npad;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / npad), r = (int)(idx % npad);
        V[idx] = (c == r) ? 1.0 : 0.0;
        if (r < n) G[(int64_t)c * n + r] = (c < n) ? B[(int64_t)r * ldb + c] : 0.0;
    }
}

__global__ void jacobi_sweep_kernel(int n, int npad, double* __restrict__ G, double* __restrict__ V,
                                    unsigned* ctl, double tol) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
    const int total_w = gridDim.x * wpb;
    const int npairs = npad / 2;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        bool rotated = false;
        for (int rnd = 0; rnd < npad - 1; ++rnd) {
            for (int pi = gw; pi < npairs; pi += total_w) {
                const int a = rr_player(pi, rnd, npad), bq = rr_player(npad - 1 - pi, rnd, npad);
                const int p = min(a, bq), q = max(a, bq);
                double* gp = G + (int64_t)p * n;
                double* gq = G + (int64_t)q * n;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int r = lane; r < n; r += 32) {
                    const double x = gp[r], y = gq[r];
                    al = fma(x, x, al);
                    be = fma(y, y, be);
                    ga = fma(x, y, ga);
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (ga != 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
                    const double zeta = (be - al) / (2.0 * ga);
                    const double t = copysign(1.0, zeta) / (fabs(zeta) + hypot(1.0, zeta));
                    const double c = 1.0 / sqrt(fma(t, t, 1.0));
                    const double s = c * t;
                    for (int r = lane; r < n; r += 32) {
                        const double x = gp[r], y = gq[r];
                        gp[r] = fma(c, x, -s * y);
                        gq[r] = fma(s, x, c * y);
                    }
                    double* vp = V + (int64_t)p * npad;
                    double* vq = V + (int64_t)q * npad;
                    for (int r = lane; r < npad; r += 32) {
                        const double x = vp[r], y = vq[r];
                        vp[r] = fma(c, x, -s * y);
                        vq[r] = fma(s, x, c * y);
                    }
                    rotated = true;
                }
            }
            if (!grid_sync(ctl)) return;
        }
        if (rotated && lane == 0) atomicAdd(&ctl[kCtlRot + sweep], 1u);
        if (!grid_sync(ctl)) return;
        if (vload(&ctl[kCtlRot + sweep]) == 0u) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl[kCtlSweeps] = (unsigned)(sweep + 1);
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl[kCtlSweeps] = (unsigned)kMaxSweeps;
}

// One CTA (1024 threads): column norms, then a bitonic sort of (sigma desc, index asc).
__global__ void __launch_bounds__(1024) jacobi_sort_kernel(int n, int npad, const double* __restrict__ G,
                                                           double* __restrict__ sig, int* __restrict__ perm,
                                                           const unsigned* ctl, int* status) {
    __shared__ double sk[TSVD_MAX_SMALL_SVD];
    __shared__ int si[TSVD_MAX_SMALL_SVD];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = warp; c < npad; c += 32) {
        const double* g = G + (int64_t)c * n;
        double acc = 0.0;
        for (int r = lane; r < n; r += 32) acc = fma(g[r], g[r], acc);
        acc = warp_sum(acc);
        if (lane == 0) {
            const double s = sqrt(acc);
            sk[c] = s;
            si[c] = c;
            if (!isfinite(s)) atomicOr(&status[kStNonfinite], 1);
        }
    }
    int P = 1;
    while (P < npad) P <<= 1;
    for (int c = npad + threadIdx.x; c < P; c += blockDim.x) {
        sk[c] = -1.0;
        si[c] = c;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int p = (j == (k >> 1)) ? (i ^ (k - 1)) : (i ^ j);
                if (p > i) {
                    // element p should come first if it is larger, or equal with a smaller index
                    const bool swap = sk[p] > sk[i] || (sk[p] == sk[i] && si[p] < si[i]);
                    if (swap) {
                        const double tk = sk[i];
                        sk[i] = sk[p];
                        sk[p] = tk;
                        const int ti = si[i];
                        si[i] = si[p];
                        si[p] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int c = threadIdx.x; c < npad; c += blockDim.x) {
        sig[c] = sk[c];
        perm[c] = si[c];
    }
    if (threadIdx.x == 0) {
        status[kStSweeps] = (int)ctl[kCtlSweeps];
        if (ctl[kCtlErr]) atomicOr(&status[kStTimeout], 1);
    }
}

// CTA per output column j < n: sign convention and the row-major outputs.
__global__ void __launch_bounds__(128) jacobi_out_kernel(int n, int npad, const double* __restrict__ G,
                                                         const double* __restrict__ V,
                                                         const double* __restrict__ sig, const int* __restrict__ perm,
                                                         double* __restrict__ Ubar, double* __restrict__ sigma,
                                                         double* __restrict__ Vbar) {
    __shared__ double bv[128];
    __shared__ int bi[128];
    const int j = blockIdx.x;
    const int src = perm[j];
    const double* v = V + (int64_t)src * npad;
    double best = -1.0;
    int besti = 0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double a = fabs(v[r]);
        if (a > best) {
            best = a;
            besti = r;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int d = 64; d > 0; d >>= 1) {
        if (threadIdx.x < d) {
            const double ob = bv[threadIdx.x + d];
            const int oi = bi[threadIdx.x + d];
            if (ob > bv[threadIdx.x] || (ob == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = ob;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const double sgn = v[bi[0]] < 0.0 ? -1.0 : 1.0;
    const double sj = sig[j];
    const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
    const double* g = G + (int64_t)src * n;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        Ubar[(int64_t)r * n + j] = sgn * (g[r] * inv);
        Vbar[(int64_t)r * n + j] = sgn * v[r];
    }
    if (threadIdx.x == 0) sigma[j] = sj;
}

}  // namespace

size_t small_svd_ws(int n) {
    const int npad = n + (n & 1);
    Arena ar;
    ar.take<double>((size_t)n * npad);
    ar.take<double>((size_t)npad * npad);
    ar.take<double>(npad);
    ar.take<int>(npad);
    ar.take<unsigned>(kCtlWords);
    return ar.off;
}

int small_svd(tsvd_handle* h, int n, const double* B, int64_t ldb, double* Ubar, double* sigma, double* Vbar,
              Arena& ar, int* status, cudaStream_t st) {
    if (n < 1 || n > TSVD_MAX_SMALL_SVD) return TSVD_ERR_UNSUPPORTED;
    const int npad = n + (n & 1);
    double* G = ar.take<double>((size_t)n * npad);
    double* V = ar.take<double>((size_t)npad * npad);
    double* sig = ar.take<double>(npad);
    int* perm = ar.take<int>(npad);
    unsigned* ctl = ar.take<unsigned>(kCtlWords);
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    ProfScope prof(h, TSVD_K_SVD, 0.0, 0.0, st);
    TSVD_TRY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(unsigned) * kCtlWords, st));
    const int64_t tot = (int64_t)npad * npad;
    h->launches += 4;
    jacobi_init_kernel<<<(unsigned)((tot + 255) / 256 < 4096 ? (tot + 255) / 256 : 4096), 256, 0, st>>>(
        n, npad, B, ldb, G, V);
    TSVD_TRY_CUDA(cudaGetLastError());
    const int npairs = npad / 2;
    const double tol = (double)(n > 16 ? n : 16) * kEps;
    if (npad <= 64) {
        jacobi_sweep_kernel<<<1, 32 * npairs, 0, st>>>(n, npad, G, V, ctl, tol);
        TSVD_TRY_CUDA(cudaGetLastError());
    } else {
        int nblocks = npairs < h->jacobi_coop_blocks ? npairs : h->jacobi_coop_blocks;
        if (nblocks < 1) return TSVD_ERR_UNSUPPORTED;
        void* args[] = {(void*)&n, (void*)&npad, (void*)&G, (void*)&V, (void*)&ctl, (void*)&tol};
        TSVD_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_sweep_kernel, dim3(nblocks), dim3(32), args,
                                                  0, st));
    }
    jacobi_sort_kernel<<<1, 1024, 0, st>>>(n, npad, G, sig, perm, ctl, status);
    jacobi_out_kernel<<<n, 128, 0, st>>>(n, npad, G, V, sig, perm, Ubar, sigma, Vbar);
    TSVD_TRY_CUDA(cudaGetLastError());
    return TSVD_OK;
}

// Occupancy of the cooperative sweep kernel (called once per handle).
int jacobi_coop_capacity(int device, int sm_count) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_sweep_kernel, 32, 0) != cudaSuccess) return 0;
    (void)device;
    return per_sm * sm_count;
}

}  // namespace tsvd
