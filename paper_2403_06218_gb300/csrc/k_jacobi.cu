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

constexpr int kJWarps = 4;     // warps per CTA when several CTAs share the sweep
constexpr int kMaxSlots = 64;  // column pairs one CTA owns per round

// One-sided Jacobi sweeps.  CTA b owns the round's pairs [b*ppb, (b+1)*ppb).
// Per round: (A) each warp forms gamma = g_p.g_q for its pairs; (B) one lane per
// pair turns (alpha, beta, gamma) into the rotation (c, s) and updates the squared
// column norms alpha - t*gamma, beta + t*gamma (exact consequences of the rotation;
// recomputed exactly at every sweep start); (C) the warps apply the rotations to
// G (and to V when it is accumulated).  Scalar FP64 work (sqrt, division) is thus
// done once per pair instead of once per lane.
__global__ void jacobi_sweep_kernel(int n, int npad, double* __restrict__ G, double* __restrict__ V,
                                    double* __restrict__ nrm, unsigned* ctl, double tol, int ppb) {
    __shared__ double s_gam[kMaxSlots], s_c[kMaxSlots], s_s[kMaxSlots];
    __shared__ int s_rot[kMaxSlots];
    __shared__ int s_any;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int npairs = npad / 2;
    const int base = blockIdx.x * ppb;
    const int cnt = max(0, min(ppb, npairs - base));
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        // exact squared column norms at the start of the sweep
        for (int c = blockIdx.x * wpb + warp; c < npad; c += gridDim.x * wpb) {
            const double* g = G + (int64_t)c * n;
            double acc = 0.0;
            for (int r = lane; r < n; r += 32) acc = fma(g[r], g[r], acc);
            acc = warp_sum(acc);
            if (lane == 0) nrm[c] = acc;
        }
        if (threadIdx.x == 0) s_any = 0;
        if (!grid_sync(ctl)) return;
        for (int rnd = 0; rnd < npad - 1; ++rnd) {
            for (int slot = warp; slot < cnt; slot += wpb) {                     // (A)
                const int pi = base + slot;
                const int a = rr_player(pi, rnd, npad), bq = rr_player(npad - 1 - pi, rnd, npad);
                const double* gp = G + (int64_t)min(a, bq) * n;
                const double* gq = G + (int64_t)max(a, bq) * n;
                double ga = 0.0;
                for (int r = lane; r < n; r += 32) ga = fma(gp[r], gq[r], ga);
                ga = warp_sum(ga);
                if (lane == 0) s_gam[slot] = ga;
            }
            __syncthreads();
            if (warp == 0) {                                                      // (B)
                for (int slot = lane; slot < cnt; slot += 32) {
                    const int pi = base + slot;
                    const int a = rr_player(pi, rnd, npad), bq = rr_player(npad - 1 - pi, rnd, npad);
                    const int p = min(a, bq), q = max(a, bq);
                    const double al = nrm[p], be = nrm[q], ga = s_gam[slot];
                    int rot = 0;
                    if (ga != 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
                        const double zeta = (be - al) / (2.0 * ga);
                        const double t = copysign(1.0, zeta) / (fabs(zeta) + hypot(1.0, zeta));
                        const double c = 1.0 / sqrt(fma(t, t, 1.0));
                        s_c[slot] = c;
                        s_s[slot] = c * t;
                        nrm[p] = fma(-t, ga, al);
                        nrm[q] = fma(t, ga, be);
                        rot = 1;
                        s_any = 1;
                    }
                    s_rot[slot] = rot;
                }
            }
            __syncthreads();
            for (int slot = warp; slot < cnt; slot += wpb) {                     // (C)
                if (!s_rot[slot]) continue;
                const int pi = base + slot;
                const int a = rr_player(pi, rnd, npad), bq = rr_player(npad - 1 - pi, rnd, npad);
                const int p = min(a, bq), q = max(a, bq);
                const double c = s_c[slot], sn = s_s[slot];
                double* gp = G + (int64_t)p * n;
                double* gq = G + (int64_t)q * n;
                for (int r = lane; r < n; r += 32) {
                    const double x = gp[r], y = gq[r];
                    gp[r] = fma(c, x, -sn * y);
                    gq[r] = fma(sn, x, c * y);
                }
                if (V != nullptr) {
                    double* vp = V + (int64_t)p * npad;
                    double* vq = V + (int64_t)q * npad;
                    for (int r = lane; r < npad; r += 32) {
                        const double x = vp[r], y = vq[r];
                        vp[r] = fma(c, x, -sn * y);
                        vq[r] = fma(sn, x, c * y);
                    }
                }
            }
            if (!grid_sync(ctl)) return;
        }
        if (threadIdx.x == 0 && s_any) atomicAdd(&ctl[kCtlRot + sweep], 1u);
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

// CTA per output column j < n.  With V accumulated: the sign convention and the
// row-major Ubar, Vbar.  Without V: Ubar = G / sigma only (the sign is fixed
// later, together with the Vbar columns recovered from B^T Ubar).
__global__ void __launch_bounds__(128) jacobi_out_kernel(int n, int npad, const double* __restrict__ G,
                                                         const double* __restrict__ V,
                                                         const double* __restrict__ sig, const int* __restrict__ perm,
                                                         double* __restrict__ Ubar, double* __restrict__ sigma,
                                                         double* __restrict__ Vbar) {
    __shared__ double bv[128];
    __shared__ int bi[128];
    const int j = blockIdx.x;
    const int src = perm[j];
    double sgn = 1.0;
    const double* v = V ? V + (int64_t)src * npad : nullptr;
    if (v) {
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
        sgn = v[bi[0]] < 0.0 ? -1.0 : 1.0;
    }
    const double sj = sig[j];
    const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
    const double* g = G + (int64_t)src * n;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        Ubar[(int64_t)r * n + j] = sgn * (g[r] * inv);
        if (v) Vbar[(int64_t)r * n + j] = sgn * v[r];
    }
    if (threadIdx.x == 0) sigma[j] = sj;
}

// Vbar[:, j] (held unscaled as B^T ubar_j) /= sigma_j, then the pair (ubar_j, vbar_j)
// is flipped so the largest-magnitude entry of vbar_j (first on ties) is positive.
__global__ void __launch_bounds__(128) jacobi_vfix_kernel(int n, const double* __restrict__ sigma,
                                                          double* __restrict__ Ubar, double* __restrict__ Vbar) {
    __shared__ double bv[128];
    __shared__ int bi[128];
    const int j = blockIdx.x;
    const double sj = sigma[j];
    const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
    double best = -1.0;
    int besti = 0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double a = fabs(Vbar[(int64_t)r * n + j] * inv);
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
    const double sgn = (Vbar[(int64_t)bi[0] * n + j] * inv) < 0.0 ? -1.0 : 1.0;
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        Vbar[(int64_t)r * n + j] = sgn * (Vbar[(int64_t)r * n + j] * inv);
        Ubar[(int64_t)r * n + j] = sgn * Ubar[(int64_t)r * n + j];
    }
}

}  // namespace

size_t small_svd_ws(int n) {
    const int npad = n + (n & 1);
    Arena ar;
    ar.take<double>((size_t)n * npad);
    ar.take<double>((size_t)npad * npad);
    ar.take<double>(npad);
    ar.take<double>(npad);
    ar.take<int>(npad);
    ar.take<unsigned>(kCtlWords);
    size_t part = 0;
    for (int nv = 1; nv <= n; ++nv) {
        const size_t v = gemm_tn_ws(nullptr, n, n, nv, false);
        if (v > part) part = v;
    }
    ar.take<char>(part + sizeof(double));
    return ar.off;
}

static int jacobi_grid(const tsvd_handle* h, int npairs, int& block) {
    if (npairs <= 32) {  // one CTA, one warp per pair, __syncthreads between rounds
        block = 32 * npairs;
        return 1;
    }
    block = 32 * kJWarps;
    int nb = (npairs + kJWarps - 1) / kJWarps;
    if (nb > h->sm_count) nb = h->sm_count;
    const int min_nb = (npairs + kMaxSlots - 1) / kMaxSlots;
    if (nb < min_nb) nb = min_nb;
    if (nb > h->jacobi_coop_blocks) return 0;
    return nb;
}

int small_svd(tsvd_handle* h, int n, const double* B, int64_t ldb, double* Ubar, double* sigma, double* Vbar, int nv,
              Arena& ar, int* status, cudaStream_t st) {
    if (n < 1 || n > TSVD_MAX_SMALL_SVD) return TSVD_ERR_UNSUPPORTED;
    if (nv < 0 || nv > n) return TSVD_ERR_INVALID_ARG;
    const int npad = n + (n & 1);
    const bool accumulate = (nv == n);
    double* G = ar.take<double>((size_t)n * npad);
    double* V = ar.take<double>((size_t)npad * npad);
    double* nrm = ar.take<double>(npad);
    double* sig = ar.take<double>(npad);
    int* perm = ar.take<int>(npad);
    unsigned* ctl = ar.take<unsigned>(kCtlWords);
    double* part = ar.take<double>(gemm_tn_ws(h, n, n, nv > 0 ? nv : 1, false) / sizeof(double) + 1);
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    const int npairs = npad / 2;
    int block = 0;
    const int nblocks = jacobi_grid(h, npairs, block);
    if (nblocks < 1) return TSVD_ERR_UNSUPPORTED;
    const int ppb = (npairs + nblocks - 1) / nblocks;
    ProfScope prof(h, TSVD_K_SVD, 0.0, 0.0, st);
    TSVD_TRY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(unsigned) * kCtlWords, st));
    const int64_t tot = (int64_t)npad * npad;
    h->launches += 4;
    jacobi_init_kernel<<<(unsigned)((tot + 255) / 256 < 4096 ? (tot + 255) / 256 : 4096), 256, 0, st>>>(
        n, npad, B, ldb, G, V);
    TSVD_TRY_CUDA(cudaGetLastError());
    const double tol = (double)(n > 16 ? n : 16) * kEps;
    double* Vacc = accumulate ? V : nullptr;
    if (nblocks == 1) {
        jacobi_sweep_kernel<<<1, block, 0, st>>>(n, npad, G, Vacc, nrm, ctl, tol, ppb);
        TSVD_TRY_CUDA(cudaGetLastError());
    } else {
        int nn = n, np = npad, pp = ppb;
        double t = tol;
        void* args[] = {(void*)&nn, (void*)&np, (void*)&G, (void*)&Vacc, (void*)&nrm, (void*)&ctl, (void*)&t,
                        (void*)&pp};
        TSVD_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_sweep_kernel, dim3(nblocks), dim3(block), args,
                                                  0, st));
    }
    jacobi_sort_kernel<<<1, 1024, 0, st>>>(n, npad, G, sig, perm, ctl, status);
    jacobi_out_kernel<<<n, 128, 0, st>>>(n, npad, G, Vacc, sig, perm, Ubar, sigma, Vbar);
    TSVD_TRY_CUDA(cudaGetLastError());
    if (!accumulate && nv > 0) {
        // right vectors of the leading nv triplets: vbar_j = B^T ubar_j / sigma_j
        TSVD_TRY_CUDA(gemm_tn(h, n, n, nv, B, ldb, Ubar, n, Vbar, n, false, part, st));
        h->launches++;
        jacobi_vfix_kernel<<<nv, 128, 0, st>>>(n, sigma, Ubar, Vbar);
        TSVD_TRY_CUDA(cudaGetLastError());
    }
    return TSVD_OK;
}

// Co-resident CTAs of the cooperative sweep kernel at its multi-CTA block size.
int jacobi_coop_capacity(int device, int sm_count) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_sweep_kernel, 32 * kJWarps, 0) != cudaSuccess)
        return 0;
    (void)device;
    return per_sm * sm_count;
}

}  // namespace tsvd
