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
// Rounds are separated by a grid barrier whose wait is bounded (clock64, ~1 s):
// on timeout it raises the status word and every CTA returns.  Sweeps repeat until one sweep
// rotates nothing (or kMaxSweeps).  Then sigma_j = |g_j|, columns are sorted by
// (sigma descending, index ascending), Ubar_j = g_j / sigma_j, Vbar_j = v_j, and
// each pair is sign-flipped so the largest-magnitude entry of Vbar_j is positive.
#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxSweeps = 40;
constexpr long long kMaxWaitCycles = 2000000000LL;  // bound of one barrier wait, ~1 s

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
            // busy-wait (naps wake late), bounded by the SM clock: ~1 s at 2 GHz
            const long long t0 = clock64();
            while (vload(&ctl[kCtlGen]) == g) {
                if (clock64() - t0 > kMaxWaitCycles) {
                    atomicOr(&ctl[kCtlErr], 1u);
                    break;
                }
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
// G (and to V when it is accumulated).  A warp-wide FP64 instruction costs the
// 2-lane FP64 pipe the same whatever its active lanes, so the scalar work of (B)
// is done once per pair, and its divide and square roots run in FP32 (see (B)).
__global__ void jacobi_sweep_kernel(int n, int npad, double* __restrict__ G, double* __restrict__ V,
                                    double* __restrict__ nrm, unsigned* ctl, double tol, int ppb) {
    const double tol2 = tol * tol;
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
                    const double big = fmax(al, be);
                    if (ga != 0.0 && big > 0.0) {
                        // scale by a power of two so the test and the FP32 ratio cannot over/underflow
                        const int e = ilogb(big);
                        const double as = scalbn(al, -e), bs = scalbn(be, -e), gs = scalbn(ga, -e);
                        if (gs * gs > tol2 * as * bs) {
                            // zeta = (beta - alpha) / (2 gamma): the difference in FP64 (it may cancel),
                            // the ratio and t in FP32 (relative accuracy 1e-7 keeps the convergence
                            // quadratic); c = 1/sqrt(1 + t^2), s = c t in FP64 so that c^2 + s^2 = 1
                            // to FP64 rounding and the rotation stays orthogonal
                            const float zf = (float)(bs - as) / (2.0f * (float)gs);
                            const float az = fabsf(zf);
                            const float tf = az > 1e18f ? 0.5f / zf
                                                        : copysignf(1.0f, zf) / (az + sqrtf(fmaf(az, az, 1.0f)));
                            const double t = (double)tf;
                            const double c = rsqrt(fma(t, t, 1.0));
                            s_c[slot] = c;
                            s_s[slot] = c * t;
                            nrm[p] = fma(-t, ga, al);
                            nrm[q] = fma(t, ga, be);
                            rot = 1;
                            s_any = 1;
                        }
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

// Block variant (right vectors not accumulated).  The npad columns form nblk
// blocks of w columns; in each round of a round-robin over blocks, CTA c owns one
// pair of blocks (I, J), copies their 2w columns into shared memory, applies all
// w*w rotations between I and J (w mini-rounds of w disjoint pairs, one warp per
// pair) -- plus, in the first round of a sweep, the rotations inside I and inside
// J -- and writes the columns back.  Every column pair meets once per sweep, so a
// sweep is still a full cyclic sweep, but it needs nblk - 1 grid barriers instead
// of npad - 1 and the rotations of a block pair stay on chip.
constexpr int kJGroup = 4;  // warps per column pair (disjoint row ranges)

// Rotations of npair_local disjoint column pairs held in shared memory.  Each pair
// is served by kJGroup warps over interleaved rows, so every SMSP holds several
// warps to hide the FP64 latency; the group's partial dot products are summed in
// a fixed order (bitwise reproducible).
__device__ inline void block_pair_rotations(double* cols, double* snrm, int n, int npair_local, const int* pp,
                                            const int* pq, double tol2, double (*s_part)[kJGroup], double* s_c,
                                            double* s_s, int* s_rot, int* s_any) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int stride = 32 * kJGroup;
    for (int slot = warp; slot < npair_local * kJGroup; slot += nw) {  // (A) partial gamma
        const int k = slot / kJGroup, sub = slot % kJGroup;
        const double* gp = cols + (size_t)pp[k] * n;
        const double* gq = cols + (size_t)pq[k] * n;
        double g0 = 0.0, g1 = 0.0;
        int r = sub * 32 + lane;
        for (; r + stride < n; r += 2 * stride) {
            g0 = fma(gp[r], gq[r], g0);
            g1 = fma(gp[r + stride], gq[r + stride], g1);
        }
        if (r < n) g0 = fma(gp[r], gq[r], g0);
        const double ga = warp_sum(g0 + g1);
        if (lane == 0) s_part[k][sub] = ga;
    }
    __syncthreads();
    if (warp == 0) {  // (B) rotation parameters, one lane per pair
        for (int k = lane; k < npair_local; k += 32) {
            double ga = 0.0;
#pragma unroll
            for (int t = 0; t < kJGroup; ++t) ga += s_part[k][t];
            const double al = snrm[pp[k]], be = snrm[pq[k]];
            int rot = 0;
            const double big = fmax(al, be);
            if (ga != 0.0 && big > 0.0) {
                const int e = ilogb(big);
                const double as = scalbn(al, -e), bs = scalbn(be, -e), gs = scalbn(ga, -e);
                if (gs * gs > tol2 * as * bs) {
                    const float zf = (float)(bs - as) / (2.0f * (float)gs);
                    const float az = fabsf(zf);
                    const float tf = az > 1e18f ? 0.5f / zf : copysignf(1.0f, zf) / (az + sqrtf(fmaf(az, az, 1.0f)));
                    const double t = (double)tf;
                    const double c = rsqrt(fma(t, t, 1.0));
                    s_c[k] = c;
                    s_s[k] = c * t;
                    snrm[pp[k]] = fma(-t, ga, al);
                    snrm[pq[k]] = fma(t, ga, be);
                    rot = 1;
                    *s_any = 1;
                }
            }
            s_rot[k] = rot;
        }
    }
    __syncthreads();
    for (int slot = warp; slot < npair_local * kJGroup; slot += nw) {  // (C) rotate
        const int k = slot / kJGroup, sub = slot % kJGroup;
        if (!s_rot[k]) continue;
        const double c = s_c[k], sn = s_s[k];
        double* gp = cols + (size_t)pp[k] * n;
        double* gq = cols + (size_t)pq[k] * n;
        for (int r = sub * 32 + lane; r < n; r += stride) {
            const double x = gp[r], y = gq[r];
            gp[r] = fma(c, x, -sn * y);
            gq[r] = fma(sn, x, c * y);
        }
    }
    __syncthreads();
}

constexpr int kJBlkMaxW = 8;

__global__ void jacobi_block_kernel(int n, int npad, int w, double* __restrict__ G, double* __restrict__ nrm,
                                    unsigned* ctl, double tol) {
    extern __shared__ double jsm[];
    double* cols = jsm;                         // 2w columns of n
    double* snrm = jsm + (size_t)2 * w * n;     // their squared norms
    __shared__ double s_part[kJBlkMaxW][kJGroup], s_c[kJBlkMaxW], s_s[kJBlkMaxW];
    __shared__ int s_rot[kJBlkMaxW], s_pp[kJBlkMaxW], s_pq[kJBlkMaxW];
    __shared__ int s_any;
    const double tol2 = tol * tol;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nblk = npad / w;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        for (int c = blockIdx.x * nw + warp; c < npad; c += gridDim.x * nw) {  // exact norms
            const double* g = G + (int64_t)c * n;
            double acc = 0.0;
            for (int r = lane; r < n; r += 32) acc = fma(g[r], g[r], acc);
            acc = warp_sum(acc);
            if (lane == 0) nrm[c] = acc;
        }
        if (threadIdx.x == 0) s_any = 0;
        if (!grid_sync(ctl)) return;
        for (int rnd = 0; rnd < nblk - 1; ++rnd) {
            const int bi = rr_player(blockIdx.x, rnd, nblk), bj = rr_player(nblk - 1 - blockIdx.x, rnd, nblk);
            // load the 2w columns (I first, then J) and their norms
            for (int idx = threadIdx.x; idx < 2 * w * n; idx += blockDim.x) {
                const int lc = idx / n, r = idx % n;
                const int gc = lc < w ? bi * w + lc : bj * w + (lc - w);
                cols[idx] = G[(int64_t)gc * n + r];
            }
            for (int lc = threadIdx.x; lc < 2 * w; lc += blockDim.x)
                snrm[lc] = nrm[lc < w ? bi * w + lc : bj * w + (lc - w)];
            __syncthreads();
            if (rnd == 0) {
                // rotations inside I and inside J: round-robin on w players, w/2 pairs per block
                for (int mr = 0; mr < w - 1; ++mr) {
                    if (threadIdx.x < w) {
                        const int k = threadIdx.x, blk = k / (w / 2), seat = k % (w / 2);
                        const int a = rr_player(seat, mr, w), b2 = rr_player(w - 1 - seat, mr, w);
                        s_pp[k] = blk * w + min(a, b2);
                        s_pq[k] = blk * w + max(a, b2);
                    }
                    __syncthreads();
                    block_pair_rotations(cols, snrm, n, w, s_pp, s_pq, tol2, s_part, s_c, s_s, s_rot, &s_any);
                }
            }
            for (int mr = 0; mr < w; ++mr) {  // rotations between I and J
                if (threadIdx.x < w) {
                    s_pp[threadIdx.x] = threadIdx.x;
                    s_pq[threadIdx.x] = w + (threadIdx.x + mr) % w;
                }
                __syncthreads();
                block_pair_rotations(cols, snrm, n, w, s_pp, s_pq, tol2, s_part, s_c, s_s, s_rot, &s_any);
            }
            for (int idx = threadIdx.x; idx < 2 * w * n; idx += blockDim.x) {
                const int lc = idx / n, r = idx % n;
                const int gc = lc < w ? bi * w + lc : bj * w + (lc - w);
                G[(int64_t)gc * n + r] = cols[idx];
            }
            for (int lc = threadIdx.x; lc < 2 * w; lc += blockDim.x)
                nrm[lc < w ? bi * w + lc : bj * w + (lc - w)] = snrm[lc];
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
    const int npad = n + 2 * kJBlkMaxW;
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
    // re-orthonormalisation of the computed right vectors (block CGS-QR, blocks of 128)
    const int bw = n < TSVD_MAX_BLOCK ? n : TSVD_MAX_BLOCK;
    ar.take<double>((size_t)n * n);
    ar.take<double>((size_t)(n - bw) * bw);
    ar.take<char>(orth_ws(nullptr, n, n - bw, bw));
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

// Block width of the block-Jacobi kernel for an order-n SVD without V, or 0 when
// the per-pair kernel is used (small n, or V accumulated).
static int block_width(int n) {
    if (n <= 64 || n > 1024) return 0;
    int w = 1;
    while (w < kJBlkMaxW && (n + 2 * w - 1) / (2 * w) * 2 > 256) w *= 2;  // at most 256 blocks -> 128 CTAs
    return w;
}

static size_t block_smem(int n, int w) { return sizeof(double) * ((size_t)2 * w * n + 2 * w); }

int small_svd(tsvd_handle* h, int n, const double* B, int64_t ldb, double* Ubar, double* sigma, double* Vbar, int nv,
              Arena& ar, int* status, cudaStream_t st) {
    if (n < 1 || n > TSVD_MAX_SMALL_SVD) return TSVD_ERR_UNSUPPORTED;
    if (nv < 0 || nv > n) return TSVD_ERR_INVALID_ARG;
    const bool accumulate = (nv == n);
    const int w = accumulate ? 0 : block_width(n);
    const int npad = w ? (n + 2 * w - 1) / (2 * w) * (2 * w) : n + (n & 1);
    double* G = ar.take<double>((size_t)n * npad);
    double* V = ar.take<double>((size_t)npad * npad);
    double* nrm = ar.take<double>(npad);
    double* sig = ar.take<double>(npad);
    int* perm = ar.take<int>(npad);
    unsigned* ctl = ar.take<unsigned>(kCtlWords);
    double* part = ar.take<double>(gemm_tn_ws(h, n, n, nv > 0 ? nv : 1, false) / sizeof(double) + 1);
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    {  // the Jacobi sweeps (the right-vector products below are timed as products)
        ProfScope prof(h, TSVD_K_SVD, 0.0, 0.0, st);
        TSVD_TRY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(unsigned) * kCtlWords, st));
        const int64_t tot = (int64_t)npad * npad;
        h->launches += 4;
        jacobi_init_kernel<<<(unsigned)((tot + 255) / 256 < 4096 ? (tot + 255) / 256 : 4096), 256, 0, st>>>(
            n, npad, B, ldb, G, V);
        TSVD_TRY_CUDA(cudaGetLastError());
        const double tol = (double)(n > 16 ? n : 16) * kEps;
        double* Vacc = accumulate ? V : nullptr;
        if (w > 0) {
            const int nblk = npad / w;
            const int nb = nblk / 2;
            const size_t smem = block_smem(n, w);
            static thread_local int configured = -1;
            if (configured != h->device) {
                TSVD_TRY_CUDA(cudaFuncSetAttribute(jacobi_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)block_smem(1024, kJBlkMaxW)));
                configured = h->device;
            }
            int per_sm = 0;
            TSVD_TRY_CUDA(
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_block_kernel, 32 * w * kJGroup, smem));
            if (per_sm * h->sm_count < nb) return TSVD_ERR_UNSUPPORTED;
            int nn = n, np = npad, ww = w;
            double t = tol;
            void* args[] = {(void*)&nn, (void*)&np, (void*)&ww, (void*)&G, (void*)&nrm, (void*)&ctl, (void*)&t};
            TSVD_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_block_kernel, dim3(nb), dim3(32 * w * kJGroup),
                                                      args, smem, st));
        } else {
            const int npairs = npad / 2;
            int block = 0;
            const int nblocks = jacobi_grid(h, npairs, block);
            if (nblocks < 1) return TSVD_ERR_UNSUPPORTED;
            const int ppb = (npairs + nblocks - 1) / nblocks;
            if (nblocks == 1) {
                jacobi_sweep_kernel<<<1, block, 0, st>>>(n, npad, G, Vacc, nrm, ctl, tol, ppb);
                TSVD_TRY_CUDA(cudaGetLastError());
            } else {
                int nn = n, np = npad, pp = ppb;
                double t = tol;
                void* args[] = {(void*)&nn, (void*)&np, (void*)&G, (void*)&Vacc, (void*)&nrm, (void*)&ctl, (void*)&t,
                                (void*)&pp};
                TSVD_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_sweep_kernel, dim3(nblocks), dim3(block),
                                                          args, 0, st));
            }
        }
        jacobi_sort_kernel<<<1, 1024, 0, st>>>(n, npad, G, sig, perm, ctl, status);
        jacobi_out_kernel<<<n, 128, 0, st>>>(n, npad, G, Vacc, sig, perm, Ubar, sigma, Vbar);
        TSVD_TRY_CUDA(cudaGetLastError());
    }
    if (!accumulate && nv > 0) {
        // right vectors of the leading nv triplets: vbar_j = B^T ubar_j / sigma_j
        TSVD_TRY_CUDA(gemm_tn(h, n, n, nv, B, ldb, Ubar, n, Vbar, n, false, part, st));
        h->launches++;
        jacobi_vfix_kernel<<<nv, 128, 0, st>>>(n, sigma, Ubar, Vbar);
        TSVD_TRY_CUDA(cudaGetLastError());
        // The columns of Ubar are orthonormal to the sweep tolerance tau, those of
        // B^T Ubar Sigma^-1 only to tau sigma_1 / sigma_j: one block CGS-QR (Alg. 3)
        // pass restores orthonormal right vectors (R = I + O(tau sigma_1 / sigma_nv)).
        OrthCtx vctx;
        vctx.seed = 0x5eedULL;
        double* Rv = ar.take<double>((size_t)nv * nv);
        if (!ar.fits()) return TSVD_ERR_WORKSPACE;
        TSVD_TRY(cgs_qr<double>(h, n, nv, nv < TSVD_MAX_BLOCK ? nv : TSVD_MAX_BLOCK, Vbar, n, Rv, vctx, ar, status,
                                st));
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
