// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "tsvd.h"

namespace tsvd {
// A matrix whose BF16 digit planes (the FP64-accurate tensor-core product's input
// form) are kept for many products: a Lanczos basis, or a dense A.  Rows layout:
// one stored row per row, one exponent per row (K = the columns); cols layout: one
// stored row per column, one exponent per column (K = the rows); planes in the
// K-block-major layout of k_oz.cu.  Columns [0, valid) are current; the owner slices
// columns as it writes them (oz_cache_slice).
struct OzCache {
    const double* src = nullptr;
    int64_t ld = 0, rows = 0, cols = 0;
    bool cols_layout = false;
    int fixed_exp = 0;  // rows layout of an orthonormal basis: every row's exponent
    __nv_bfloat16* planes = nullptr;
    int* exps = nullptr;
    int64_t valid = 0;
};
constexpr int kOzNoFixedExp = -(1 << 30);
}  // namespace tsvd

// CUDA-event timing per kernel class (TSVD_FLAG_PROFILE).
struct tsvd_prof_rec {
    int cls;
    cudaEvent_t e0, e1;
    double flops, bytes;
};

struct tsvd_handle {
    int device;
    int sm_count;
    int jacobi_coop_blocks;  // co-resident CTAs of the cooperative Jacobi kernel
    int64_t launches;        // kernels enqueued through this handle (running total)
    bool profiling = false;
    int prof_class = -1;     // when >= 0, the class every ProfScope records (see ProfClass)
    std::vector<tsvd_prof_rec> recs;
    std::vector<cudaEvent_t> pool;
    // Scratch of the FP64-accurate tensor-core products for the current call
    // (carved from the caller's workspace by the entry point; null: the FP64
    // products run on the FP64 pipe), and the status words its kernels report to.
    void* oz_ws = nullptr;
    size_t oz_bytes = 0;
    int* oz_status = nullptr;
    // operands whose digit planes are kept for the current call (owned by the caller)
    std::vector<const tsvd::OzCache*> oz_caches;
    // set by OzFreshRows: products slice their left operand afresh instead of
    // reading a rows-layout basis cache
    bool oz_fresh_rows = false;
    // limit, in SM clock cycles, of one bounded wait of the pipelined product kernels
    // and of the Jacobi grid barrier (2e9, about 1 s; tsvd_set_wait_limit lowers it)
    long long max_wait = 2000000000LL;
    // row partition (tsvd_set_row_partition): this process holds rows
    // [part_row0, part_row0 + m) of a part_rows x n matrix; part_fn sums host buffers
    // over the processes of the partition
    tsvd_allreduce_fn part_fn = nullptr;
    void* part_ctx = nullptr;
    int64_t part_row0 = 0, part_rows = 0;
    std::vector<double> part_host;
};

namespace tsvd {

constexpr double kEps = 2.220446049250313e-16;  // 2^-52

// Device status words live at the front of every workspace; kernels set them,
// the host reads them back after a stream synchronisation.
enum StatusWord : int {
    kStBreakdown = 0,    // Cholesky pivot at/below the breakdown threshold
    kStNonfinite = 1,    // NaN/Inf met
    kStBadCsr = 2,       // CSR structure invalid
    kStTimeout = 3,      // a bounded device-side wait gave up
    kStSweeps = 4,       // Jacobi sweeps used
    kStCount = 16
};

#define TSVD_TRY_CUDA(expr)                                   \
    do {                                                      \
        cudaError_t tsvd_e_ = (expr);                         \
        if (tsvd_e_ != cudaSuccess) return TSVD_ERR_CUDA;     \
    } while (0)

#define TSVD_TRY(expr)                                        \
    do {                                                      \
        int tsvd_s_ = (expr);                                 \
        if (tsvd_s_ < 0) return tsvd_s_;                      \
    } while (0)

// Makes the handle's device current for the lifetime of the guard and restores
// the caller's current device afterwards (on every return path).
class DeviceGuard {
  public:
    explicit DeviceGuard(int device) {
        ok_ = cudaGetDevice(&prev_) == cudaSuccess;
        if (ok_ && prev_ != device) ok_ = cudaSetDevice(device) == cudaSuccess;
        switched_ = ok_;
        if (!ok_) prev_ = -1;
    }
    ~DeviceGuard() {
        if (switched_ && prev_ >= 0) cudaSetDevice(prev_);
    }
    bool ok() const { return ok_; }

  private:
    int prev_ = -1;
    bool ok_ = false, switched_ = false;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Brackets the launches of one kernel class with events on the launching stream.
class ProfScope {
  public:
    ProfScope(tsvd_handle* h, int cls, double flops, double bytes, cudaStream_t st)
        : h_(h && h->profiling ? h : nullptr), st_(st) {
        if (!h_) return;
        rec_.cls = h_->prof_class >= 0 ? h_->prof_class : cls;
        rec_.flops = flops;
        rec_.bytes = bytes;
        rec_.e0 = get();
        rec_.e1 = get();
        cudaEventRecord(rec_.e0, st_);
    }
    ~ProfScope() {
        if (!h_) return;
        cudaEventRecord(rec_.e1, st_);
        h_->recs.push_back(rec_);
    }

  private:
    cudaEvent_t get() {
        if (!h_->pool.empty()) {
            cudaEvent_t e = h_->pool.back();
            h_->pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    tsvd_handle* h_;
    cudaStream_t st_;
    tsvd_prof_rec rec_{};
};

// Files every launch in its lifetime under one class (products with A that
// reuse the GEMM kernels count as products with A).
struct ProfClass {
    tsvd_handle* h;
    int prev;
    ProfClass(tsvd_handle* hh, int cls) : h(hh), prev(hh->prof_class) { h->prof_class = cls; }
    ~ProfClass() { h->prof_class = prev; }
};

// Sets the flop count of the latest record of a class (work known only after
// the launch, e.g. the Jacobi sweeps).
inline void prof_set_last_flops(tsvd_handle* h, int cls, double flops) {
    if (!h->profiling) return;
    for (auto it = h->recs.rbegin(); it != h->recs.rend(); ++it)
        if (it->cls == cls) {
            it->flops = flops;
            return;
        }
}
inline double jacobi_flops(int n, int nv, int sweeps) {
    return (double)sweeps * (nv >= n ? 18.0 : 12.0) * n * (0.5 * n * (n - 1.0));
}

// Sums the recorded events into info->prof_* (the stream must be synchronised).
void prof_collect(tsvd_handle* h, tsvd_info* info);

// Bump allocator over caller-owned workspace.  With base == nullptr it only
// measures (sizing pass); the same carving code runs for both passes.
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += align256(count * sizeof(T));
        return p;
    }
    bool fits() const { return base == nullptr || off <= cap; }
};

inline int check_ws(const void* ws, size_t have, size_t need) {
    if (need == 0) return TSVD_OK;
    if (ws == nullptr || have < need) return TSVD_ERR_WORKSPACE;
    if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return TSVD_ERR_WORKSPACE;
    return TSVD_OK;
}

// Reads the status words back (synchronises the stream) and maps them to a code.
int read_status(cudaStream_t st, const int* d_status, int* h_status /* kStCount */);

// ---- kernel launchers (return cudaError_t of the launch) -------------------
// All matrices row-major with explicit leading dimensions.

// y = A x, CSR A (m rows), x (w columns, ldx), y (ldy).  Entries whose column
// is outside [0, n) are skipped and flag kStBadCsr.
// T = double (FP64 path) or float (mixed path: FP32 values and blocks).
// Split plan of a CSR matrix for SpMM: rows longer than kSpmmChunk entries are cut
// into chunks of kSpmmChunk (descriptor {row, chunk index in the row, chunks of
// the row, 0}, ordered by row), each summed by its own warp into `partial`.
constexpr int64_t kSpmmChunk = 1024;
inline int64_t spmm_max_chunks(int64_t nnz) { return 2 * (nnz / kSpmmChunk) + 1; }
inline int64_t spmm_partial_ld(int w) { return (w + 1) & ~1; }
struct SpmmPlan {
    int64_t nchunks = 0;  // host copy of the chunk count
    const int4* chunks = nullptr;
    void* partial = nullptr;  // (nchunks) x spmm_partial_ld(wmax) values of the SpMM type
    int wmax = 0;
};
size_t spmm_plan_ws(int64_t m, int64_t nnz, int wmax, size_t elem);
// Builds the plan of row_ptr (m rows, nnz entries) in `ar`; synchronises `st` once
// to read the chunk count.
int spmm_plan(tsvd_handle* h, int64_t m, int64_t nnz, const int32_t* rp, int wmax, size_t elem, Arena& ar,
              SpmmPlan* plan, cudaStream_t st);
template <typename T>
cudaError_t launch_spmm(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr,
                        const int32_t* col_idx, const T* val, int w, const T* X,
                        int64_t ldx, T* Y, int64_t ldy, int* status, cudaStream_t st,
                        const SpmmPlan* plan = nullptr);

size_t csr_transpose_ws(int64_t m, int64_t n, int64_t nnz);
template <typename T>
int csr_transpose(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr,
                  const int32_t* col_idx, const T* val, int32_t* t_row_ptr,
                  int32_t* t_col_idx, T* t_val, Arena& ar, int* status, cudaStream_t st);

// y[i] = (float)x[i]
cudaError_t convert_to_float(tsvd_handle* h, int64_t n, const double* x, float* y, cudaStream_t st);

// C (s x b, ldc) = X^T Z over q rows; X (q x s, ldx), Z (q x b, ldz).
// symmetric: X == Z and s == b; only the upper half is computed and mirrored.
// TI in {double, float} is the input and in-slab accumulation type; split-K
// partial sums are FP64; TC is the output type.
// Split-K scratch of gemm_tn for inputs of elem_bytes (8: FP64 inputs, 4: FP32 inputs).
size_t gemm_tn_ws(tsvd_handle* h, int64_t q, int64_t s, int64_t b, bool symmetric, int elem_bytes = 8);
// Register-tiled FP32 kernels (k_f32.cu) behind gemm_tn<float, *> and gemm_nn<float, *, *>.
template <typename TW>
cudaError_t launch_gemm_tn_f32(dim3 grid, cudaStream_t st, int64_t q, int64_t s, int64_t b, const float* X,
                               int64_t ldx, const float* Z, int64_t ldz, TW* out, int64_t ldo, int64_t slab_stride,
                               int64_t slab_rows, int symmetric, int nreg_s, int nreg_b);
// Split-BF16 tensor-core products (k_tc.cu).  Pieces of a rows x cols matrix are
// stored [3][rows][bf16x3_ld(cols)] as BF16.
int64_t bf16x3_ld(int64_t cols);
size_t bf16x3_bytes(int64_t rows, int64_t cols);
// Pieces of S (rows x cols) or, with trans, of S^T.
template <typename T>
cudaError_t bf16x3_split(tsvd_handle* h, int64_t rows, int64_t cols, const T* S, int64_t lds, bool trans, void* out,
                         cudaStream_t st);
// Y (rows x w, FP32) = P X, P given by its pieces (rows x cols), X cols x w (FP32).
size_t tc_mm_ws(int64_t rows, int64_t cols, int w);
cudaError_t tc_mm(tsvd_handle* h, int64_t rows, int64_t cols, const void* pieces, int w, const float* X, int64_t ldx,
                  float* Y, int64_t ldy, void* ws, int* status, cudaStream_t st);
template <typename TM, typename TY>
cudaError_t launch_gemm_nn_f32(cudaStream_t st, int64_t q, int64_t s, int64_t b, double alpha, const float* X,
                               int64_t ldx, const TM* M, int64_t ldm, double beta, TY* Y, int64_t ldy, bool upper);
// Fused update + Gram of FP32 blocks (k_f32.cu kernel, k_dense.cu host side):
//   Y (q x b, ldy) = beta Y + alpha X M  (X q x s FP32, M s x b FP64; upper as in gemm_nn),
//   W (b x b, ld b, FP64, both halves) = Y^T Y of the updated Y,
// in one pass over the rows; Y may alias X (s == b, ldx == ldy).  b <= 128.
// Partial Gram sums per row slab go to `partial` (update_gram_ws bytes) and are
// reduced in a fixed order.
size_t update_gram_ws(int64_t q, int64_t b);
cudaError_t update_gram(tsvd_handle* h, int64_t q, int64_t s, int64_t b, double alpha, const float* X, int64_t ldx,
                        const double* M, int64_t ldm, double beta, float* Y, int64_t ldy, bool upper, double* W,
                        double* partial, cudaStream_t st);
template <typename TM>
cudaError_t launch_update_gram_f32(cudaStream_t st, int slabs, int64_t slab_rows, int64_t q, int64_t s, int64_t b,
                                   double alpha, const float* X, int64_t ldx, const TM* M, int64_t ldm, double beta,
                                   float* Y, int64_t ldy, bool upper, double* partial);
template <typename TI, typename TC>
cudaError_t gemm_tn(tsvd_handle* h, int64_t q, int64_t s, int64_t b, const TI* X, int64_t ldx,
                    const TI* Z, int64_t ldz, TC* C, int64_t ldc, bool symmetric,
                    double* partial_ws, cudaStream_t st);

// ---- FP64-accurate tensor-core products (k_oz.cu) -------------------------------
// Worth running on the tensor cores rather than the FP64 pipe (M x N outputs, K deep).
bool oz_worth(int64_t M, int64_t N, int64_t K);
// Scratch of C = X^T Z (q rows; s x b outputs) and of Y = X M (q x s times s x b);
// cached_x: the planes of X come from a cache.
size_t oz_tn_ws(int64_t q, int64_t s, int64_t b, bool symmetric, bool cached_x = false);
size_t oz_nn_ws(int64_t q, int64_t s, int64_t b, bool cached_x = false);
// Scratch that covers every product with q <= qmax, s <= smax, b <= bmax (and s, b swapped).
size_t oz_ws_bound(int64_t qmax, int64_t smax, int64_t bmax);
// C (s x b, ldc) = X^T Z, X (q x s, ldx), Z (q x b, ldz); symmetric: Z == X, C mirrored.
// xc: cached planes of X (cols layout, s <= xc->valid) instead of slicing X.
int oz_gemm_tn(tsvd_handle* h, int64_t q, int64_t s, int64_t b, const double* X, int64_t ldx, const double* Z,
               int64_t ldz, double* C, int64_t ldc, bool symmetric, void* ws, size_t ws_bytes, int* status,
               cudaStream_t st, const OzCache* xc = nullptr);
// Y (q x b, ldy) = beta Y + alpha X M; upper: M upper triangular (entries below its
// diagonal are not read).  Y may alias X.
// xc: cached planes of X (rows layout, s <= xc->valid).
int oz_gemm_nn(tsvd_handle* h, int64_t q, int64_t s, int64_t b, double alpha, const double* X, int64_t ldx,
               const double* Mm, int64_t ldm, double beta, double* Y, int64_t ldy, bool upper, void* ws,
               size_t ws_bytes, int* status, cudaStream_t st, const OzCache* xc = nullptr);
// Caches: bytes, carving (no device work), slicing of columns [c0, c1) (c0 <= valid;
// then valid = c1), and the lookup the products use.
size_t oz_cache_bytes(int64_t rows, int64_t cols, bool cols_layout);
void oz_cache_carve(OzCache& c, Arena& ar, const double* src, int64_t ld, int64_t rows, int64_t cols,
                    bool cols_layout, int fixed_exp);
int oz_cache_slice(tsvd_handle* h, OzCache& c, int64_t c0, int64_t c1, cudaStream_t st);
// Columns from v on are about to be rewritten: valid = min(valid, v).
int oz_cache_truncate(tsvd_handle* h, OzCache& c, int64_t v, cudaStream_t st);
const OzCache* oz_find_cache(const tsvd_handle* h, const double* X, int64_t ldx, int64_t rows, int64_t s,
                             bool cols_layout);
// Registers caches with the handle for its lifetime.
struct OzCacheScope {
    tsvd_handle* h;
    size_t n0;
    explicit OzCacheScope(tsvd_handle* hh) : h(hh), n0(hh->oz_caches.size()) {}
    void add(const OzCache* c) { h->oz_caches.push_back(c); }
    ~OzCacheScope() { h->oz_caches.resize(n0); }
};

// Within its lifetime the FP64 products slice their left operand afresh, with one
// exponent per row, instead of reading the rows-layout planes of a basis cache.
// Those planes give every row the fixed exponent of an orthonormal basis (entries
// below 2), so a basis of n rows, with entries near n^-1/2, keeps about log2(n)/2
// bits fewer than FP64 there.  The cache serves the CGS-CQR2 updates, whose
// coefficients are computed from the same planes; the restart and Ritz products,
// whose results the next cycle takes as exact Ritz vectors, slice afresh.
struct OzFreshRows {
    tsvd_handle* h;
    bool prev;
    explicit OzFreshRows(tsvd_handle* hh) : h(hh), prev(hh->oz_fresh_rows) { h->oz_fresh_rows = true; }
    ~OzFreshRows() { h->oz_fresh_rows = prev; }
};

// Makes the FP64 products of one call run on the tensor cores with `bytes` of
// scratch at `ws` (restores the handle's previous setting on destruction).
struct OzScope {
    tsvd_handle* h;
    void* prev_ws;
    size_t prev_bytes;
    int* prev_status;
    OzScope(tsvd_handle* hh, void* ws, size_t bytes, int* status)
        : h(hh), prev_ws(hh->oz_ws), prev_bytes(hh->oz_bytes), prev_status(hh->oz_status) {
        h->oz_ws = ws;
        h->oz_bytes = bytes;
        h->oz_status = status;
    }
    ~OzScope() {
        h->oz_ws = prev_ws;
        h->oz_bytes = prev_bytes;
        h->oz_status = prev_status;
    }
};

// Y (q x b, ldy) = beta Y + alpha X M; X (q x s, ldx), M (s x b, ldm).
// upper: M is upper triangular (entries below the diagonal are not read).
// Y may alias X (in place) when s == b and ldx == ldy.
// Accumulates in TX; M is converted to TX.
template <typename TX, typename TM, typename TY>
cudaError_t gemm_nn(tsvd_handle* h, int64_t q, int64_t s, int64_t b, double alpha, const TX* X,
                    int64_t ldx, const TM* M, int64_t ldm, double beta, TY* Y, int64_t ldy,
                    bool upper, cudaStream_t st);

// Cholesky W = L L^T of a b x b SPD matrix (ld b) in one CTA; writes
// Lt = L^T and Mt = L^{-T} (both upper, ld b).  Sets kStBreakdown on a pivot
// <= b*eps*max_i W_ii, kStNonfinite on NaN/Inf.
cudaError_t chol_inv(tsvd_handle* h, int b, const double* W, double* Lt, double* Mt, int* status,
                     cudaStream_t st);

// out = A U where A, U are b x b upper triangular (ld b); trans writes out^T.
cudaError_t trmm_upper(tsvd_handle* h, int b, const double* A, const double* U, double* out,
                       int64_t ldo, bool trans, cudaStream_t st);

// rows x cols of the N(0,1) block of the given seed and stream, starting at global
// row row0 (a row slice of the same global block, whichever process draws it).
cudaError_t gaussian(tsvd_handle* h, int64_t rows, int64_t cols, uint64_t seed, uint32_t stream_id,
                     double* out, int64_t ld, cudaStream_t st, int64_t row0 = 0);

// Small SVD by one-sided Jacobi.  nv == n accumulates every right vector; nv < n
// recovers only the leading nv right vectors as B^T ubar_j / sigma_j (columns
// j >= nv of Vbar are left undefined and those of Ubar carry no sign convention).
size_t small_svd_ws(int n);
// deferred: the re-orthonormalisation of the recovered right vectors runs unsynchronised
// and a breakdown there only sets the caller's breakdown flag.
// target >= 0: the relative residual the caller needs from Ritz pairs built on the
// result (0: as small as it gets); a small target tightens the sweep tolerance (see
// k_jacobi.cu).  target < 0: the default tolerance.
int small_svd(tsvd_handle* h, int n, const double* B, int64_t ldb, double* Ubar, double* sigma,
              double* Vbar, int nv, Arena& ar, int* status, cudaStream_t st, bool deferred = false,
              double target = -1.0);

// out[j] = sum_i (Y[i,j] - U[i,j] * sigma[j])^2 for j < k  (deterministic).
size_t colres_ws(int64_t q, int k);
cudaError_t col_residual_sq(tsvd_handle* h, int64_t q, int k, const double* Y, int64_t ldy,
                            const double* U, int64_t ldu, const double* sigma, double* out,
                            double* partial, cudaStream_t st);

// rho[j] = || Rr * Vlast[:, j] ||_2, Rr b x b upper (ld b), Vlast b rows of Vbar (ld ldv), j < k.
// ---- backward kernels (backward.cu) -----------------------------------------
int svd_backward_run(tsvd_handle* h, const tsvd_matrix* A, int k, const double* sigma, const double* U,
                     const double* V, const double* sb, const double* Ub, const double* Vb, double* grad,
                     const tsvd_backward_opts* o, char* ws, size_t ws_bytes, size_t* sizing,
                     tsvd_backward_info* info);
size_t coldot_ws(int64_t rows, int k);
// out[j] = sum_i X[i][j] Y[i][j] (fixed order); partial: coldot_ws bytes.
cudaError_t coldot(tsvd_handle* h, int64_t rows, int k, const double* X, int64_t ldx, const double* Y, int64_t ldy,
                   double* out, double* partial, cudaStream_t st);
cudaError_t cg_alpha(tsvd_handle* h, int k, const double* rr, const double* pap, const double* bb, double tol2,
                     double* alpha, cudaStream_t st);
cudaError_t cg_beta(tsvd_handle* h, int k, double* rr, const double* rr_new, const double* alpha, double* beta,
                    cudaStream_t st);
cudaError_t cg_xr(tsvd_handle* h, int64_t rows, int k, const double* alpha, const double* p, const double* Ap,
                  double* x, double* r, cudaStream_t st);
cudaError_t cg_p(tsvd_handle* h, int64_t rows, int k, const double* alpha, const double* beta, const double* r,
                 double* p, cudaStream_t st);
cudaError_t shifted(tsvd_handle* h, int64_t rows, int k, const double* s, const double* p, const double* q,
                    double* out, cudaStream_t st);
cudaError_t add_scaled_cols(tsvd_handle* h, int64_t rows, int k, const double* Y, const double* s, double* out,
                            int64_t ldo, cudaStream_t st);
cudaError_t coupling(tsvd_handle* h, int k, const double* s, const double* sb, const double* J, const double* K,
                     double* C, cudaStream_t st);
cudaError_t sddmm(tsvd_handle* h, int64_t m, int64_t nnz, const int32_t* rp, const int32_t* ci, int kk,
                  const double* Lf, int64_t ldl, const double* Rf, int64_t ldr, double* grad, cudaStream_t st);

// D (cols x rows, ld ldd) = H^T for H rows x cols (ld ldh).
cudaError_t put_transposed(tsvd_handle* h, int rows, int cols, const double* H, int64_t ldh, double* D, int64_t ldd,
                           cudaStream_t st);
// B[i][i] = sig[i], i < s.
cudaError_t put_diagonal(tsvd_handle* h, int s, const double* sig, double* B, int64_t ldb, cudaStream_t st);
cudaError_t lanczos_rho(tsvd_handle* h, int b, int k, const double* Rr, const double* Vlast,
                        int64_t ldv, double* rho, cudaStream_t st);

// Flip (u_j, v_j) so that the largest-magnitude entry of v_j (first on ties) is positive.
size_t sign_fix_ws(int64_t n, int k);
cudaError_t sign_fix(tsvd_handle* h, int64_t n, int64_t m, int k, double* V, int64_t ldv,
                     double* U, int64_t ldu, void* ws, cudaStream_t st);

// Strided 2-D copy of a rows x cols block (device to device).
template <typename T>
inline cudaError_t copy_block(const T* src, int64_t lds, T* dst, int64_t ldd, int64_t rows, int64_t cols,
                              cudaStream_t st) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    return cudaMemcpy2DAsync(dst, ldd * sizeof(T), src, lds * sizeof(T), cols * sizeof(T), rows,
                             cudaMemcpyDeviceToDevice, st);
}

// ---- orthogonalisation (orth.cu) -------------------------------------------
struct OrthCtx {
    uint64_t seed = 0;
    int replacements = 0;  // Philox replacement columns drawn (stream 0x100 + t)
    int fallbacks = 0;     // Cholesky breakdowns sent to the CGS2 fallback
    // Deferred: do not synchronise after each orthogonalisation; a breakdown only
    // leaves the sticky status word set, and the caller redoes the whole cycle
    // with deferred = false so that the fallback runs where it is needed.
    bool deferred = false;
    // the tall dimension is this process's rows of a row-partitioned block: every
    // product that sums over it (Gram matrices, projections, norms) is summed over the
    // partition before use, and replacement columns are drawn at the global rows
    // starting at row0
    bool reduce = false;
    int64_t row0 = 0;
};

// Sums the rows x cols block d (ld doubles, device) over the row partition of the
// handle, in place (a no-op without one).  TSVD_ERR_COMM when the exchange fails.
int part_sum(tsvd_handle* h, double* d, int64_t rows, int64_t cols, int64_t ld, cudaStream_t st);

// Workspace of one orthogonalisation (sized for double blocks, which covers float).
size_t orth_ws(tsvd_handle* h, int64_t q, int64_t s, int b);
// Y (q x b) <- Q; R (b x b, ld ldr, trans: write R^T); H (s x b, ld b) optional.
// T = double or float (storage of P and Y); H and R are FP64.
template <typename T>
int cgs_cqr2(tsvd_handle* h, int64_t q, int64_t s, int b, const T* P, int64_t ldp,
             T* Y, int64_t ldy, double* H, double* R, int64_t ldr, bool r_trans,
             OrthCtx& ctx, Arena ar, int* status, cudaStream_t st);
template <typename T>
int cgs_qr(tsvd_handle* h, int64_t q, int r, int b, T* Y, int64_t ldy, double* R,
           OrthCtx& ctx, Arena ar, int* status, cudaStream_t st);

}  // namespace tsvd
