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
#include <algorithm>

#include "tsvd_internal.cuh"

namespace tsvd {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxSweeps = 40;

enum Ctl : int { kCtlCount = 0, kCtlGen = 1, kCtlErr = 2, kCtlSweeps = 3, kCtlRot = 8 };
constexpr int kCtlWords = kCtlRot + kMaxSweeps;

__device__ inline unsigned vload(const unsigned* p) { return *reinterpret_cast<const volatile unsigned*>(p); }

// Grid-wide barrier for a cooperative launch (all CTAs co-resident); one wait
// gives up after max_wait SM clock cycles (the handle's limit, about 1 s by
// default).  Returns false once any CTA has timed out; the answer is read once
// per CTA (by thread 0, through shared memory), so every thread of a CTA takes
// the same branch and none is left at a later __syncthreads.
__device__ bool grid_sync(unsigned* ctl, long long max_wait) {
    if (gridDim.x == 1) {
        __syncthreads();
        return true;
    }
    __shared__ int s_ok;
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
            // busy-wait (naps wake late), bounded by the SM clock
            const long long t0 = clock64();
            while (vload(&ctl[kCtlGen]) == g) {
                if (clock64() - t0 > max_wait) {
                    atomicOr(&ctl[kCtlErr], 1u);
                    break;
                }
            }
        }
        __threadfence();
        s_ok = vload(&ctl[kCtlErr]) == 0u ? 1 : 0;
    }
    __syncthreads();
    return s_ok != 0;
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
                                    double* __restrict__ nrm, unsigned* ctl, double tol, int ppb,
                                    long long max_wait) {
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
        if (!grid_sync(ctl, max_wait)) return;
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
            if (!grid_sync(ctl, max_wait)) return;
        }
        if (threadIdx.x == 0 && s_any) atomicAdd(&ctl[kCtlRot + sweep], 1u);
        if (!grid_sync(ctl, max_wait)) return;
        if (vload(&ctl[kCtlRot + sweep]) == 0u) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl[kCtlSweeps] = (unsigned)(sweep + 1);
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl[kCtlSweeps] = (unsigned)kMaxSweeps;
}

// Block variant (right vectors not accumulated): the block one-sided method of
// Hari and Veselic with the rotations of a block pair done on its Gram matrix.
// The npad columns form nblk blocks of W columns; in each round of a
// round-robin over blocks, CTA c owns one pair of blocks (I, J).  It copies their
// 2W columns C into shared memory and forms M = C^T C from them; one warp then
// runs the round's rotations (the W mini-rounds of W disjoint pairs between I
// and J, and in the first round of a sweep the W - 1 mini-rounds inside I and
// inside J) two-sided on M, M <- R^T M R, accumulating Z = R_1 R_2 ...; finally
// C Z replaces the columns.  Each rotation is computed from the same
// alpha = |g_p|^2, beta = |g_q|^2, gamma = g_p.g_q as in the one-sided method
// (M holds exactly the Gram matrix of the rotated columns, to rounding, and a
// rotation's update of M has errors relative to the norms of the columns it
// mixes, so the relative accuracy is that of the one-sided method).  Every column
// pair meets once per sweep, as in a cyclic sweep; the n-length work of a round
// is two small dense products (the Gram matrix and C Z) over all the CTA's
// threads, and the sequential rotations touch only the 2W x 2W matrices of one
// warp, so a sweep costs nblk - 1 grid barriers and about n warp-local
// mini-rounds instead of n CTA-wide ones.
constexpr int kJGThreads = 256;  // threads of the block kernel

// Rotation parameters of one column pair from alpha = |g_p|^2, beta = |g_q|^2 and
// gamma = g_p.g_q (Rutishauser's formulas); false when |gamma| <= tol sqrt(alpha beta).
// FP64: zeta = (beta - alpha) / (2 gamma) with the difference in FP64 (it may cancel),
// the ratio and t in FP32 (relative accuracy 1e-7 keeps the convergence quadratic),
// c = 1/sqrt(1 + t^2) and s = c t in FP64 so that c^2 + s^2 = 1 to FP64 rounding and
// the rotation stays orthogonal.  FP32 (the preconditioning sweeps): all in FP32.
__device__ inline bool rot_params(double al, double be, double ga, double tol2, double& c, double& sn, double& t) {
    const double big = fmax(al, be);
    if (!(ga != 0.0 && big > 0.0)) return false;
    // scale by a power of two so the test and the FP32 ratio cannot over/underflow
    const int e = ilogb(big);
    const double as = scalbn(al, -e), bs = scalbn(be, -e), gs = scalbn(ga, -e);
    if (!(gs * gs > tol2 * as * bs)) return false;
    const float zf = (float)(bs - as) / (2.0f * (float)gs);
    const float az = fabsf(zf);
    const float tf = az > 1e18f ? 0.5f / zf : copysignf(1.0f, zf) / (az + sqrtf(fmaf(az, az, 1.0f)));
    t = (double)tf;
    c = rsqrt(fma(t, t, 1.0));
    sn = c * t;
    return true;
}
__device__ inline bool rot_params(float al, float be, float ga, float tol2, float& c, float& sn, float& t) {
    const float big = fmaxf(al, be);
    if (!(ga != 0.0f && big > 0.0f)) return false;
    const int e = ilogbf(big);
    const float as = scalbnf(al, -e), bs = scalbnf(be, -e), gs = scalbnf(ga, -e);
    if (!(gs * gs > tol2 * as * bs)) return false;
    const float zf = (bs - as) / (2.0f * gs);
    const float az = fabsf(zf);
    t = az > 1e18f ? 0.5f / zf : copysignf(1.0f, zf) / (az + sqrtf(fmaf(az, az, 1.0f)));
    c = rsqrtf(fmaf(t, t, 1.0f));
    sn = c * t;
    return true;
}

template <typename T>
__device__ inline T warp_sum_t(T v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

// Column stride (elements) of the block's columns in shared memory: odd, so that
// the same row of different columns falls in different banks.
__host__ __device__ inline int gram_ld(int n) { return n | 1; }

template <typename T, int W>
__host__ __device__ constexpr size_t gram_smem(int n) {
    return sizeof(T) * (size_t)(2 * W) * (size_t)gram_ld(n);
}

// M = C^T C for the 2W columns in shared memory (stride ld): the tiles on and
// above the diagonal of TM x TM register tiles (the others mirrored), each tile's
// rows split over S interleaved lane slices that a shuffle tree sums in a fixed
// order.  A diagonal tile is symmetric bit for bit (x_a x_b = x_b x_a in every fma).
template <typename T, int W>
__device__ inline void gram_form(const T* cols, int n, int ld, T (*M)[2 * W + 1]) {
    constexpr int W2 = 2 * W;
    constexpr int TM = W2 >= 32 ? 8 : (W2 >= 8 ? 4 : 2);
    constexpr int NTS = W2 / TM;
    constexpr int NT = NTS * (NTS + 1) / 2;
    constexpr int S0 = kJGThreads / NT;
    constexpr int S = S0 >= 32 ? 32 : (S0 >= 16 ? 16 : (S0 >= 8 ? 8 : (S0 >= 4 ? 4 : (S0 >= 2 ? 2 : 1))));
    static_assert(NT * S <= kJGThreads, "Gram tiling exceeds the block");
    const int t = threadIdx.x;
    int u = t / S;
    const int s = t % S;
    // lanes of one warp share their tile group: a warp is wholly in or out when S
    // divides 32; with S < 32 the last warp may be partly idle, so idle lanes run the
    // loop on tile 0 and drop their sums (the shuffles need every lane)
    const bool live = u < NT;
    if (!live) u = 0;
    if ((t & ~31) >= NT * S) return;  // whole idle warps
    int ti = 0;
    while (u >= NTS - ti) {
        u -= NTS - ti;
        ++ti;
    }
    const int tj = ti + u;
    T acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
    const T* ca = cols + (size_t)(ti * TM) * ld;
    const T* cb = cols + (size_t)(tj * TM) * ld;
    for (int r = s; r < n; r += S) {
        T x[TM], y[TM];
#pragma unroll
        for (int a = 0; a < TM; ++a) {
            x[a] = ca[(size_t)a * ld + r];
            y[a] = cb[(size_t)a * ld + r];
        }
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TM; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) {
            T v = acc[a][b];
#pragma unroll
            for (int d = S / 2; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
            if (s == 0 && live) {
                M[ti * TM + a][tj * TM + b] = v;
                M[tj * TM + b][ti * TM + a] = v;
            }
        }
}

// Row stride of Z: 16-byte rows, so that the C Z products read a row of Z four
// floats (two doubles) at a time.
template <typename T, int W>
__host__ __device__ constexpr int gram_zs() {
    return 2 * W + (int)(16 / sizeof(T));
}

// acc[j] += x Z_k[j] for j < W2, Z_k a 16-byte aligned row (vector loads, broadcast
// to the warp).
template <typename T, int W2>
__device__ inline void gram_axpy_row(T x, const T* zk, T* acc) {
    if constexpr (sizeof(T) == 4 && W2 % 4 == 0) {
#pragma unroll
        for (int j = 0; j < W2; j += 4) {
            const float4 z = *reinterpret_cast<const float4*>(zk + j);
            acc[j] = fma(x, (T)z.x, acc[j]);
            acc[j + 1] = fma(x, (T)z.y, acc[j + 1]);
            acc[j + 2] = fma(x, (T)z.z, acc[j + 2]);
            acc[j + 3] = fma(x, (T)z.w, acc[j + 3]);
        }
    } else if constexpr (sizeof(T) == 8 && W2 % 2 == 0) {
#pragma unroll
        for (int j = 0; j < W2; j += 2) {
            const double2 z = *reinterpret_cast<const double2*>(zk + j);
            acc[j] = fma(x, (T)z.x, acc[j]);
            acc[j + 1] = fma(x, (T)z.y, acc[j + 1]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < W2; ++j) acc[j] = fma(x, zk[j], acc[j]);
    }
}

// One mini-round on the block's Gram matrix by warp 0: npr disjoint pairs
// (pp[k], pq[k]) rotated at once; M <- R^T M R and Z <- Z R.  Returns whether any
// pair rotated (warp-uniform).
template <typename T, int W>
__device__ inline bool gram_mini_round(T (*M)[2 * W + 1], T (*Z)[gram_zs<T, W>()], const int* pp, const int* pq,
                                       int npr,
                                       T tol2, T* s_c, T* s_s, int* s_rot) {
    constexpr int W2 = 2 * W;
    const int lane = threadIdx.x & 31;
    int rot = 0;
    if (lane < npr) {
        const int p = pp[lane], q = pq[lane];
        T c = T(1), sn = T(0), t = T(0);
        rot = rot_params(M[p][p], M[q][q], M[p][q], tol2, c, sn, t) ? 1 : 0;
        s_c[lane] = c;
        s_s[lane] = sn;
        s_rot[lane] = rot;
    }
    const bool any = __any_sync(kFull, rot != 0);
    if (!any) return false;
    __syncwarp();
    if (lane < W2) {  // columns: lane = row of M and of Z
        for (int k = 0; k < npr; ++k) {
            if (!s_rot[k]) continue;
            const int p = pp[k], q = pq[k];
            const T c = s_c[k], sn = s_s[k];
            const T x = M[lane][p], y = M[lane][q];
            M[lane][p] = fma(c, x, -sn * y);
            M[lane][q] = fma(sn, x, c * y);
            const T u = Z[lane][p], v = Z[lane][q];
            Z[lane][p] = fma(c, u, -sn * v);
            Z[lane][q] = fma(sn, u, c * v);
        }
    }
    __syncwarp();
    if (lane < W2) {  // rows: lane = column of M
        for (int k = 0; k < npr; ++k) {
            if (!s_rot[k]) continue;
            const int p = pp[k], q = pq[k];
            const T c = s_c[k], sn = s_s[k];
            const T x = M[p][lane], y = M[q][lane];
            M[p][lane] = fma(c, x, -sn * y);
            M[q][lane] = fma(sn, x, c * y);
        }
    }
    __syncwarp();
    return true;
}

// The W mini-rounds between the blocks (pairs (k, W + (k + mr) mod W)) by warp 0
// with the block's Gram matrix in registers: lane r < 2W holds row r of M and of
// Z, the J half of each row stored cyclically shifted by mr (position k holds
// column W + (k + mr) mod W), so that pair k always meets positions k and k of a
// row and no register is indexed at run time.  A rotation acts on the columns of
// M and Z within each lane, and on the rows of M between lane k and its partner
// lane by shuffles.  M and Z enter and leave in shared memory.  Returns whether
// any pair rotated (warp-uniform).
template <typename T, int W>
__device__ inline bool gram_rounds_ij(T (*M)[2 * W + 1], T (*Z)[gram_zs<T, W>()], T tol2) {
    constexpr int W2 = 2 * W;
    const int lane = threadIdx.x & 31;
    const int r = lane < W2 ? lane : 0;  // lanes past 2W mirror row 0 (their results are dropped)
    T A[W], J[W], ZA[W], ZJ[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
        A[j] = M[r][j];
        J[j] = M[r][W + j];
        ZA[j] = Z[r][j];
        ZJ[j] = Z[r][W + j];
    }
    bool any = false;
    for (int mr = 0; mr < W; ++mr) {
        // own diagonal entry: column r sits at A[r] (r < W) or at J[(r - W - mr) mod W]
        const int jpos = r < W ? r : (r - W - mr + 2 * W) % W;
        T d = T(0), g = T(0);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            if (j == jpos) d = r < W ? A[j] : J[j];
            if (j == r) g = J[j];  // M[k][q_k] for the pair's I lane k = r
        }
        const int partner = r < W ? W + (r + mr) % W : jpos;
        const T dq = __shfl_sync(kFull, d, partner);
        T c = T(1), sn = T(0), t = T(0);
        int rot = 0;
        if (lane < W) rot = rot_params(d, dq, g, tol2, c, sn, t) ? 1 : 0;
        if (!rot) {
            c = T(1);
            sn = T(0);
        }
        if (!__any_sync(kFull, rot != 0)) {
            // no pair rotates: only the shift of the J halves
        } else {
            any = true;
            // columns (p, q) = (k, W + (k + mr) mod W) of this lane's rows of M and Z
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const T ck = __shfl_sync(kFull, c, k), sk = __shfl_sync(kFull, sn, k);
                const T x = A[k], y = J[k];
                A[k] = fma(ck, x, -sk * y);
                J[k] = fma(sk, x, ck * y);
                const T u = ZA[k], v = ZJ[k];
                ZA[k] = fma(ck, u, -sk * v);
                ZJ[k] = fma(sk, u, ck * v);
            }
            // rows p and q of M: lane p (r < W) and lane q exchange their rows
            const int pair = r < W ? r : jpos;
            const T cp = __shfl_sync(kFull, c, pair), sp = __shfl_sync(kFull, sn, pair);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const T oa = __shfl_sync(kFull, A[k], partner), oj = __shfl_sync(kFull, J[k], partner);
                if (r < W) {
                    A[k] = fma(cp, A[k], -sp * oa);
                    J[k] = fma(cp, J[k], -sp * oj);
                } else {
                    A[k] = fma(sp, oa, cp * A[k]);
                    J[k] = fma(sp, oj, cp * J[k]);
                }
            }
        }
        // next mini-round: position k of the J halves moves to column W + (k + mr + 1) mod W
        const T j0 = J[0], z0 = ZJ[0];
#pragma unroll
        for (int k = 0; k < W - 1; ++k) {
            J[k] = J[k + 1];
            ZJ[k] = ZJ[k + 1];
        }
        J[W - 1] = j0;
        ZJ[W - 1] = z0;
    }
    __syncwarp();
    if (lane < W2) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            M[r][j] = A[j];
            M[r][W + j] = J[j];
            Z[r][j] = ZA[j];
            Z[r][W + j] = ZJ[j];
        }
    }
    __syncwarp();
    return any;
}

template <typename T, int W>
__global__ void __launch_bounds__(kJGThreads, 1) jacobi_gram_kernel(int n, int npad, T* __restrict__ G,
                                                                 T* __restrict__ V, unsigned* ctl, T tol,
                                                                 long long max_wait) {
    constexpr int W2 = 2 * W;
    static_assert(W2 <= 32 && (W == 1 || W % 2 == 0), "block width: 1 or even, at most 16");
    extern __shared__ __align__(16) unsigned char jsm_raw[];
    T* cols = reinterpret_cast<T*>(jsm_raw);  // 2W columns, stride ld
    __shared__ T M[W2][W2 + 1];
    __shared__ __align__(16) T Z[W2][gram_zs<T, W>()];
    __shared__ T s_c[W], s_s[W];
    __shared__ int s_rot[W], s_pp[W], s_pq[W];
    __shared__ int s_any, s_rnd;
    const T tol2 = tol * tol;
    const int ld = gram_ld(n);
    const int nblk = npad / W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        if (threadIdx.x == 0) s_any = 0;
        for (int rnd = 0; rnd < nblk - 1; ++rnd) {
            const int bi = rr_player(blockIdx.x, rnd, nblk), bj = rr_player(nblk - 1 - blockIdx.x, rnd, nblk);
            for (int r = threadIdx.x; r < n; r += blockDim.x) {  // all 2W loads in flight at once
                T v[W2];
#pragma unroll
                for (int k = 0; k < W2; ++k) v[k] = G[(int64_t)(k < W ? bi * W + k : bj * W + (k - W)) * n + r];
#pragma unroll
                for (int k = 0; k < W2; ++k) cols[(size_t)k * ld + r] = v[k];
            }
            __syncthreads();
            gram_form<T, W>(cols, n, ld, M);
            __syncthreads();
            if (warp == 0) {
                for (int e = lane; e < W2 * W2; e += 32) Z[e / W2][e % W2] = (e / W2 == e % W2) ? T(1) : T(0);
                __syncwarp();
                bool any = false;
                if (rnd == 0) {
                    // rotations inside I and inside J: round-robin on W players, W/2 pairs per block
                    for (int mr = 0; mr < W - 1; ++mr) {
                        if (lane < W) {
                            const int blk = lane / (W / 2), seat = lane % (W / 2);
                            const int a = rr_player(seat, mr, W), b2 = rr_player(W - 1 - seat, mr, W);
                            s_pp[lane] = blk * W + min(a, b2);
                            s_pq[lane] = blk * W + max(a, b2);
                        }
                        __syncwarp();
                        any |= gram_mini_round<T, W>(M, Z, s_pp, s_pq, W, tol2, s_c, s_s, s_rot);
                        __syncwarp();
                    }
                }
                any |= gram_rounds_ij<T, W>(M, Z, tol2);  // rotations between I and J
                if (lane == 0) {
                    s_rnd = any ? 1 : 0;
                    if (any) s_any = 1;
                }
            }
            __syncthreads();
            if (s_rnd) {
                // C Z: thread r computes row r of the 2W rotated columns (2W independent sums)
                for (int r = threadIdx.x; r < n; r += blockDim.x) {
                    T acc[W2];
#pragma unroll
                    for (int j = 0; j < W2; ++j) acc[j] = T(0);
#pragma unroll 2
                    for (int k = 0; k < W2; ++k) {
                        const T x = cols[(size_t)k * ld + r];
                        gram_axpy_row<T, W2>(x, Z[k], acc);
                    }
#pragma unroll
                    for (int j = 0; j < W2; ++j) G[(int64_t)(j < W ? bi * W + j : bj * W + (j - W)) * n + r] = acc[j];
                }
                if (V) {
                    // accumulated rotations (npad x npad, column-major): V <- V Z on the
                    // block pair's columns, read from global memory row by row
                    for (int r = threadIdx.x; r < npad; r += blockDim.x) {
                        T acc[W2];
#pragma unroll
                        for (int j = 0; j < W2; ++j) acc[j] = T(0);
#pragma unroll 4
                        for (int k = 0; k < W2; ++k) {
                            const T x = V[(int64_t)(k < W ? bi * W + k : bj * W + (k - W)) * npad + r];
                            gram_axpy_row<T, W2>(x, Z[k], acc);
                        }
#pragma unroll
                        for (int j = 0; j < W2; ++j)
                            V[(int64_t)(j < W ? bi * W + j : bj * W + (j - W)) * npad + r] = acc[j];
                    }
                }
            }
            if (!grid_sync(ctl, max_wait)) return;
        }
        if (threadIdx.x == 0 && s_any) atomicAdd(&ctl[kCtlRot + sweep], 1u);
        if (!grid_sync(ctl, max_wait)) return;
        if (vload(&ctl[kCtlRot + sweep]) == 0u) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl[kCtlSweeps] = (unsigned)(sweep + 1);
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl[kCtlSweeps] = (unsigned)kMaxSweeps;
}


// FP32 copy of B in the Jacobi layout: column c of G32 (ld n) = column c of B
// (B row-major), padded columns zero; V32 (npad x npad, column-major) = I.
__global__ void jacobi_init32_kernel(int n, int npad, const double* __restrict__ B, int64_t ldb,
                                     float* __restrict__ G, float* __restrict__ V) {
    const int64_t tot = (int64_t)npad * n, totv = (int64_t)npad * npad;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot + totv;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < tot) {
            const int c = (int)(idx / n), r = (int)(idx % n);
            G[idx] = c < n ? (float)B[(int64_t)r * ldb + c] : 0.0f;
        } else {
            const int64_t k = idx - tot;
            V[k] = (k / npad == k % npad) ? 1.0f : 0.0f;
        }
    }
}

// V (n x n row-major, FP64) = the leading n x n block of the accumulated FP32
// rotations V32 (the right singular directions of B to FP32 accuracy).  Also hands
// a timeout of the FP32 sweeps to the status words.
__global__ void jacobi_vinit_kernel(int n, int npad, const float* __restrict__ V32, double* __restrict__ V,
                                    const unsigned* ctl32, int* status) {
    const int64_t tot = (int64_t)n * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / n), c = (int)(idx % n);
        V[idx] = (double)V32[(int64_t)c * npad + r];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && ctl32[kCtlErr]) atomicOr(&status[kStTimeout], 1);
}

// After the polar iterations: if V^T V (in T) is not the identity to 1e-12, V = I
// (the FP64 sweeps then start from B itself).  One CTA.
__global__ void __launch_bounds__(1024) jacobi_vcheck_kernel(int n, const double* __restrict__ Tm,
                                                             double* __restrict__ V) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += blockDim.x) {
        const int i = (int)(idx / n), j = (int)(idx % n);
        const double d = Tm[idx] - (i == j ? 1.0 : 0.0);
        if (!(fabs(d) <= 1e-12)) bad = 1;
    }
    __syncthreads();
    if (!bad) return;
    for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += blockDim.x)
        V[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
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

// Breakdown, non-finite and timeout words of a private status block OR-ed into the caller's.
__global__ void fold_status_kernel(const int* __restrict__ from, int* __restrict__ to) {
    const int w = threadIdx.x;
    if ((w == kStBreakdown || w == kStNonfinite || w == kStTimeout) && from[w]) atomicOr(&to[w], 1);
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

// Block width of the FP64 block-Jacobi kernel for an order-n SVD without V (at most
// one wave of 152 CTAs, each owning a pair of blocks), or 0 when the per-pair kernel
// is used (small n, or V accumulated).
static int block_width(int n) {
    if (n <= 64 || n > 1024) return 0;
    int w = 1;
    while (w < 8 && (n + 2 * w - 1) / (2 * w) > 152) w *= 2;
    return w;
}
// Block width of the FP32 preconditioning sweeps: the widest blocks (fewest rounds;
// FP32 work is cheap next to the rounds' latency).
constexpr int kJW32 = 16;

static int pad_to(int n, int w) { return (n + 2 * w - 1) / (2 * w) * (2 * w); }

// Buffers of one small SVD, carved identically by the sizing and the run.
struct SvdBufs {
    double *G, *V, *nrm, *sig, *part;
    int* perm;
    unsigned *ctl, *ctl32;
    float *G32, *V32;
    double *Vp, *Tm, *Y;  // preconditioner: V, V^T V, B V (n x n row-major)
    void* oz;
    size_t oz_bytes;
};

static SvdBufs carve_svd(Arena& ar, int n, int npad, int nv, bool precond) {
    SvdBufs b{};
    b.G = ar.take<double>((size_t)n * npad);
    b.V = ar.take<double>((size_t)npad * npad);
    b.nrm = ar.take<double>(npad);
    b.sig = ar.take<double>(npad);
    b.perm = ar.take<int>(npad);
    b.ctl = ar.take<unsigned>(kCtlWords);
    b.part = ar.take<double>(gemm_tn_ws(nullptr, n, n, nv > 0 ? nv : 1, false) / sizeof(double) + 1);
    if (precond) {
        const int np32 = pad_to(n, kJW32);
        b.ctl32 = ar.take<unsigned>(kCtlWords);
        b.G32 = ar.take<float>((size_t)n * np32);
        b.V32 = ar.take<float>((size_t)np32 * np32);
        b.Vp = ar.take<double>((size_t)n * n);
        b.Tm = ar.take<double>((size_t)n * n);
        b.Y = ar.take<double>((size_t)n * n);
        b.oz_bytes = std::max(oz_tn_ws(n, n, n, true), oz_nn_ws(n, n, n));
        b.oz = ar.take<char>(b.oz_bytes);
    }
    return b;
}

size_t small_svd_ws(int n) {
    size_t best = 0;
    for (int nv : {n, n - 1}) {
        if (nv < 0) continue;
        const bool acc = nv == n;
        const int w = acc ? 0 : block_width(n);
        const int npad = w ? pad_to(n, w) : n + (n & 1);
        Arena ar;
        carve_svd(ar, n, npad, n, w > 0);
        // re-orthonormalisation of the computed right vectors (block CGS-QR, blocks of 128)
        const int bw = n < TSVD_MAX_BLOCK ? n : TSVD_MAX_BLOCK;
        ar.take<double>((size_t)n * n);
        ar.take<int>(kStCount);
        ar.take<double>((size_t)(n - bw) * bw);
        ar.take<char>(orth_ws(nullptr, n, n - bw, bw));
        best = std::max(best, ar.off);
    }
    return best;
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

// Cooperative launch of the block-Jacobi sweeps on G (n x npad, column-major) in T
// with blocks of W columns.
template <typename T, int W>
static int launch_gram(tsvd_handle* h, int n, int npad, T* G, unsigned* ctl, T tol, cudaStream_t st, T* V) {
    const int nb = npad / W / 2;
    const size_t smem = gram_smem<T, W>(n);
    static thread_local int configured = -1;
    if (configured != h->device) {
        TSVD_TRY_CUDA(cudaFuncSetAttribute(jacobi_gram_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)gram_smem<T, W>(1024)));
        configured = h->device;
    }
    int per_sm = 0;
    TSVD_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_gram_kernel<T, W>, kJGThreads, smem));
    if (per_sm * h->sm_count < nb) return TSVD_ERR_UNSUPPORTED;
    int nn = n, np = npad;
    T t = tol;
    long long mw = h->max_wait;
    void* args[] = {(void*)&nn, (void*)&np, (void*)&G, (void*)&V, (void*)&ctl, (void*)&t, (void*)&mw};
    h->launches++;
    TSVD_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_gram_kernel<T, W>, dim3(nb), dim3(kJGThreads), args,
                                              smem, st));
    return TSVD_OK;
}

template <typename T>
static int run_block_sweeps(tsvd_handle* h, int n, int npad, int w, T* G, unsigned* ctl, T tol, cudaStream_t st,
                            T* V = nullptr) {
    switch (w) {
        case 1: return launch_gram<T, 1>(h, n, npad, G, ctl, tol, st, V);
        case 2: return launch_gram<T, 2>(h, n, npad, G, ctl, tol, st, V);
        case 4: return launch_gram<T, 4>(h, n, npad, G, ctl, tol, st, V);
        case 8: return launch_gram<T, 8>(h, n, npad, G, ctl, tol, st, V);
        default: return TSVD_ERR_UNSUPPORTED;
    }
}
template <>
int run_block_sweeps<float>(tsvd_handle* h, int n, int npad, int w, float* G, unsigned* ctl, float tol,
                            cudaStream_t st, float* V) {
    if (w != kJW32) return TSVD_ERR_UNSUPPORTED;
    return launch_gram<float, kJW32>(h, n, npad, G, ctl, tol, st, V);
}

int small_svd(tsvd_handle* h, int n, const double* B, int64_t ldb, double* Ubar, double* sigma, double* Vbar, int nv,
              Arena& ar, int* status, cudaStream_t st, bool deferred, double target) {
    if (n < 1 || n > TSVD_MAX_SMALL_SVD) return TSVD_ERR_UNSUPPORTED;
    if (nv < 0 || nv > n) return TSVD_ERR_INVALID_ARG;
    const bool accumulate = (nv == n);
    const int w = accumulate ? 0 : block_width(n);
    const int npad = w ? pad_to(n, w) : n + (n & 1);
    const SvdBufs bf = carve_svd(ar, n, npad, nv, w > 0);
    if (!ar.fits()) return TSVD_ERR_WORKSPACE;
    double* G = bf.G;
    double* V = bf.V;
    {  // the Jacobi sweeps (the right-vector products below are timed as products)
        ProfScope prof(h, TSVD_K_SVD, 0.0, 0.0, st);
        TSVD_TRY_CUDA(cudaMemsetAsync(bf.ctl, 0, sizeof(unsigned) * kCtlWords, st));
        const int64_t tot = (int64_t)npad * npad;
        const unsigned ib = (unsigned)((tot + 255) / 256 < 4096 ? (tot + 255) / 256 : 4096);
        // Sweep tolerance tau (columns p, q count as orthogonal once |g_p.g_q| <=
        // tau |g_p||g_q|): max(n, 16) eps by default.  Ritz pairs built on the result
        // have residuals of a small multiple of tau sigma_1: couplings below tau are
        // never rotated away, and with thick restart the converged kept Ritz vectors
        // enter B with exactly such couplings (their columns are then not rotated at
        // all, and the last block rows of their singular vectors stay zero).  A caller
        // that needs residuals below 1e3 n eps (or as small as they get, target 0)
        // gets tau = sqrt(n) eps, the level to which a computed coupling (an n-term
        // FP64 dot product) is itself known.
        double tol = (double)(n > 16 ? n : 16) * kEps;
        if (target >= 0.0 && target < 1e3 * tol) tol = std::sqrt((double)(n > 16 ? n : 16)) * kEps;
        double* Vacc = accumulate ? V : nullptr;
        if (w > 0) {
            // (1) FP32 block-Jacobi sweeps on B with the rotations accumulated in V32: the
            //     right singular directions of B, orthogonal to FP32 rounding (so B V has
            //     columns orthogonal to about eps32 sigma_1 / sigma_j, where the right
            //     vectors from the orthogonalised columns of B^T would leave couplings of
            //     eps32 (sigma_1 / sigma_j)^2 and more FP64 sweeps)
            const int np32 = pad_to(n, kJW32);
            TSVD_TRY_CUDA(cudaMemsetAsync(bf.ctl32, 0, sizeof(unsigned) * kCtlWords, st));
            h->launches += 2;
            jacobi_init32_kernel<<<(unsigned)std::min<int64_t>(4096, ((int64_t)(n + np32) * np32 + 255) / 256), 256, 0,
                                   st>>>(n, np32, B, ldb, bf.G32, bf.V32);
            TSVD_TRY_CUDA(cudaGetLastError());
            const float tol32 = (float)(n > 16 ? n : 16) * 5.9604645e-08f;  // n 2^-24
            TSVD_TRY(run_block_sweeps<float>(h, n, np32, kJW32, bf.G32, bf.ctl32, tol32, st, bf.V32));
            jacobi_vinit_kernel<<<(unsigned)std::min<int64_t>(4096, ((int64_t)n * n + 255) / 256), 256, 0, st>>>(
                n, np32, bf.V32, bf.Vp, bf.ctl32, status);
            TSVD_TRY_CUDA(cudaGetLastError());
            // (2) V orthogonal to FP64 rounding: two polar (Newton-Schulz) steps
            //     V <- V (3 I - V^T V) / 2 with FP64-accurate tensor-core products, then a
            //     check that falls back to V = I if V^T V is not the identity to 1e-12
            for (int itn = 0; itn < 2; ++itn) {
                TSVD_TRY(oz_gemm_tn(h, n, n, n, bf.Vp, n, bf.Vp, n, bf.Tm, n, true, bf.oz, bf.oz_bytes, status, st));
                TSVD_TRY(oz_gemm_nn(h, n, n, n, -0.5, bf.Vp, n, bf.Tm, n, 1.5, bf.Vp, n, false, bf.oz, bf.oz_bytes,
                                    status, st));
            }
            TSVD_TRY(oz_gemm_tn(h, n, n, n, bf.Vp, n, bf.Vp, n, bf.Tm, n, true, bf.oz, bf.oz_bytes, status, st));
            h->launches++;
            jacobi_vcheck_kernel<<<1, 1024, 0, st>>>(n, bf.Tm, bf.Vp);
            TSVD_TRY_CUDA(cudaGetLastError());
            // (3) FP64 sweeps on B V: the SVD of B V is that of B with the right vectors
            //     rotated by V, and its columns start orthogonal to FP32 accuracy
            TSVD_TRY(oz_gemm_nn(h, n, n, n, 1.0, B, ldb, bf.Vp, n, 0.0, bf.Y, n, false, bf.oz, bf.oz_bytes, status,
                                st));
            h->launches++;
            jacobi_init_kernel<<<ib, 256, 0, st>>>(n, npad, bf.Y, n, G, V);
            TSVD_TRY_CUDA(cudaGetLastError());
            TSVD_TRY(run_block_sweeps<double>(h, n, npad, w, G, bf.ctl, tol, st));
        } else {
            h->launches++;
            jacobi_init_kernel<<<ib, 256, 0, st>>>(n, npad, B, ldb, G, V);
            TSVD_TRY_CUDA(cudaGetLastError());
            const int npairs = npad / 2;
            int block = 0;
            const int nblocks = jacobi_grid(h, npairs, block);
            if (nblocks < 1) return TSVD_ERR_UNSUPPORTED;
            const int ppb = (npairs + nblocks - 1) / nblocks;
            h->launches++;
            if (nblocks == 1) {
                jacobi_sweep_kernel<<<1, block, 0, st>>>(n, npad, G, Vacc, bf.nrm, bf.ctl, tol, ppb, h->max_wait);
                TSVD_TRY_CUDA(cudaGetLastError());
            } else {
                int nn = n, np = npad, pp = ppb;
                double t = tol;
                double* nrm = bf.nrm;
                unsigned* ctl = bf.ctl;
                long long mw = h->max_wait;
                void* args[] = {(void*)&nn, (void*)&np, (void*)&G, (void*)&Vacc, (void*)&nrm, (void*)&ctl, (void*)&t,
                                (void*)&pp, (void*)&mw};
                TSVD_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_sweep_kernel, dim3(nblocks), dim3(block),
                                                          args, 0, st));
            }
        }
        h->launches += 2;
        jacobi_sort_kernel<<<1, 1024, 0, st>>>(n, npad, G, bf.sig, bf.perm, bf.ctl, status);
        jacobi_out_kernel<<<n, 128, 0, st>>>(n, npad, G, Vacc, bf.sig, bf.perm, Ubar, sigma, Vbar);
        TSVD_TRY_CUDA(cudaGetLastError());
    }
    if (!accumulate && nv > 0) {
        // right vectors of the leading nv triplets: vbar_j = B^T ubar_j / sigma_j
        TSVD_TRY_CUDA(gemm_tn(h, n, n, nv, B, ldb, Ubar, n, Vbar, n, false, bf.part, st));
        h->launches++;
        jacobi_vfix_kernel<<<nv, 128, 0, st>>>(n, sigma, Ubar, Vbar);
        TSVD_TRY_CUDA(cudaGetLastError());
        // The columns of Ubar are orthonormal to the sweep tolerance tau, those of
        // B^T Ubar Sigma^-1 only to tau sigma_1 / sigma_j: one block CGS-QR (Alg. 3)
        // pass restores orthonormal right vectors (R = I + O(tau sigma_1 / sigma_nv)).
        // It reports to status words of its own, so that it never consumes the caller's
        // pending breakdown flag; deferred: unsynchronised, its breakdown folded into the
        // caller's flag (the caller then redoes its work checked).
        OrthCtx vctx;
        vctx.seed = 0x5eedULL;
        vctx.deferred = deferred;
        double* Rv = ar.take<double>((size_t)nv * nv);
        int* vst = ar.take<int>(kStCount);
        if (!ar.fits()) return TSVD_ERR_WORKSPACE;
        TSVD_TRY_CUDA(cudaMemsetAsync(vst, 0, sizeof(int) * kStCount, st));
        TSVD_TRY(cgs_qr<double>(h, n, nv, nv < TSVD_MAX_BLOCK ? nv : TSVD_MAX_BLOCK, Vbar, n, Rv, vctx, ar, vst, st));
        h->launches++;
        fold_status_kernel<<<1, 32, 0, st>>>(vst, status);
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
