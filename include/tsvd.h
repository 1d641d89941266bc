/*
 * tsvd.h -- C ABI of a truncated-SVD library for one NVIDIA GB300 (sm_103a).
 *
 * Methods (Tomas, Quintana-Orti, Anzt, "Fast Truncated SVD of Sparse and Dense
 * Matrices on Graphics Processors"):
 *   - RandSVD, randomized subspace iteration (Sec. 2.1, Alg. 1);
 *   - LancSVD, block Golub-Kahan-Lanczos bidiagonalisation with full two-sided
 *     block re-orthogonalisation and basic restart (Sec. 2.2, Alg. 2), or a
 *     thick restart that keeps Ritz pairs (tsvd_opts.restart_keep);
 * their building blocks: CGS-QR (Alg. 3), CholeskyQR2 (Alg. 4),
 * CGS-CQR2 (Alg. 5), the sparse/dense block products with A and A^T (Table 1),
 * the small SVD of the projected matrix (Alg. 1 S5, Alg. 2 S6) and the
 * Gaussian start block (Sec. 4); a mixed-precision form of both methods
 * (TSVD_PREC_MIXED); and the gradient of a loss on the k leading triplets
 * with respect to A (tsvd_svd_backward).
 *
 * Conventions shared by every entry point
 *   - Dense blocks are ROW-MAJOR: element (i, j) of a block with leading
 *     dimension ld is at p[i * ld + j].  ld >= number of columns.
 *   - Arithmetic and floating-point outputs are FP64, except where an entry
 *     point says otherwise: the *_f32 and BF16-piece products, and the FP32
 *     blocks and products of the mixed form (TSVD_PREC_MIXED), whose returned
 *     triplets are still FP64.
 *   - Pointers are CUDA device pointers unless a descriptor field says
 *     TSVD_HOST.  The caller owns every buffer; the library keeps no pointer
 *     after a call returns and never allocates device memory: scratch comes
 *     from the caller's workspace, sized by the matching *_workspace_size call.
 *     Workspace pointers must be 256-byte aligned.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it; every entry point synchronises that stream before it
 *     returns (the status words it reports are read back from the device).
 *   - Return value: TSVD_OK (0), TSVD_NOT_CONVERGED (1, a warning: outputs
 *     hold the best triplets found), or a negative error code.  On an error the
 *     outputs are unspecified; no exception or abort crosses the ABI.
 *   - Integers describing sizes are int64_t; CSR indices are int32_t.
 */
#ifndef TSVD_H_
#define TSVD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define TSVD_OK                 0
#define TSVD_NOT_CONVERGED      1   /* warning: tolerance not met within max_restarts */
#define TSVD_ERR_INVALID_ARG   (-1) /* bad size, parameter, pointer, or CSR structure  */
#define TSVD_ERR_NONFINITE     (-2) /* NaN/Inf met in the data or a Gram diagonal     */
#define TSVD_ERR_CUDA          (-3) /* a CUDA runtime call failed                       */
#define TSVD_ERR_WORKSPACE     (-4) /* workspace missing, too small or misaligned       */
#define TSVD_ERR_TIMEOUT       (-5) /* a bounded device-side wait gave up               */
#define TSVD_ERR_UNSUPPORTED   (-6) /* a size beyond this build's kernel limits         */
#define TSVD_ERR_COMM          (-7) /* the row partition's reduction callback failed   */

/* ---- enumerations ------------------------------------------------------ */
#define TSVD_DENSE   0   /* tsvd_matrix.format: row-major dense                    */
#define TSVD_CSR     1   /* tsvd_matrix.format: compressed sparse row              */
#define TSVD_F64     0   /* tsvd_matrix.dtype: FP64 values                         */
#define TSVD_F32     1   /* tsvd_matrix.dtype: FP32 values (widened exactly where FP64 is needed) */
#define TSVD_DEVICE  0   /* memory location of a buffer                            */
#define TSVD_HOST    1

#define TSVD_METHOD_RSVD      0
#define TSVD_METHOD_BLANCZOS  1

/* tsvd_opts.precision */
#define TSVD_PREC_FP64   0   /* every step in FP64 (the paper's method)                      */
#define TSVD_PREC_MIXED  1   /* FP32 blocks, bases and products (sparse A: FP32 values;
                                dense A: split-BF16 tensor-core products of FP32 accuracy);
                                FP64 Gram reductions, Cholesky, R, B, small SVD, and a final
                                FP64 Rayleigh-Ritz step on the Ritz vectors with the FP64 A
                                (k <= TSVD_MAX_BLOCK) */

/* Largest block width of one Cholesky factorisation (CholeskyQR2 / CGS-CQR2);
 * CGS-QR splits wider blocks (Alg. 3).  Largest small-SVD order. */
#define TSVD_MAX_BLOCK      128
#define TSVD_MAX_SMALL_SVD  2048

/* The matrix A (m x n).  Dense: `val` points to m*ld values (dtype), row-major.
 * CSR: row_ptr[m+1] (row_ptr[0] = 0, non-decreasing, row_ptr[m] = nnz),
 * col_idx[nnz] in [0, n), val[nnz] (dtype); columns within a row in any order. */
typedef struct tsvd_matrix {
    int64_t m, n;
    int32_t format;          /* TSVD_DENSE or TSVD_CSR                     */
    int32_t dtype;           /* TSVD_F64 or TSVD_F32 (values widened exactly
                                wherever FP64 is needed)                   */
    int32_t location;        /* TSVD_DEVICE or TSVD_HOST (copied in)       */
    int32_t reserved;        /* set to 0                                   */
    const void* val;
    int64_t ld;              /* dense only                                 */
    const int32_t* row_ptr;  /* CSR only                                   */
    const int32_t* col_idx;  /* CSR only                                   */
    int64_t nnz;             /* CSR only                                   */
} tsvd_matrix;

/* tsvd_opts.flags bits */
#define TSVD_FLAG_PROFILE  1   /* time every kernel class with CUDA events (tsvd_info.prof_*) */
#define TSVD_FLAG_ROW_PARTITION 2 /* A is one process's row block (tsvd_set_row_partition):
                                     never transposed; size the workspace with it too */

/* Kernel classes reported by TSVD_FLAG_PROFILE (index into tsvd_info.prof_*). */
#define TSVD_K_APROD    0   /* products with A or A^T: CSR SpMM (Table 1 SpMM), dense GEMM
                               with A, split-BF16 tensor-core products                    */
#define TSVD_K_SPMM     TSVD_K_APROD
#define TSVD_K_GEMM_TN  1   /* X^T Z: Gram matrices and projections P^T Q (Algs. 4, 5)    */
#define TSVD_K_GEMM_NN  2   /* X M: updates Q - P H, Q L^{-T}, Ritz/restart products      */
#define TSVD_K_CHOL     3   /* Cholesky + triangular inverse of a Gram matrix             */
#define TSVD_K_SVD      4   /* small Jacobi SVD (flops: 12 n per rotation, 18 n with V,
                               n(n-1)/2 rotations a sweep, times the sweeps it took)    */
#define TSVD_K_OTHER    5   /* start block, transpose build, residuals, copies            */
#define TSVD_K_UPD_GRAM 6   /* fused update + Gram of FP32 blocks (mixed form): Q - P H or
                               Q L^{-T} together with the Gram matrix of the result       */
#define TSVD_K_COUNT    7

/* Options; fill with tsvd_default_opts() and override fields. */
typedef struct tsvd_opts {
    double tol;              /* LancSVD stops when the residual of every returned triplet,
                                max(||A v_j - s_j u_j||, ||A^T u_j - s_j v_j||), is <= tol * s_1
                                (default 1e-6) */
    int32_t max_restarts;    /* LancSVD restarts allowed after the first cycle (default 50) */
    int32_t qr_block;        /* RandSVD CGS-QR block width; 0 = min(k+p, TSVD_MAX_BLOCK) */
    int32_t output_location; /* TSVD_DEVICE or TSVD_HOST for sigma/U/V (default device) */
    int32_t flags;           /* TSVD_FLAG_* bits (default 0) */
    const double* start_block; /* optional device block replacing the Philox draw:
                                  RandSVD n' x (k+p), LancSVD m' x b, row-major, ld = cols,
                                  where m' >= n' are the dimensions after the m<n transpose */
    void* stream;            /* cudaStream_t */
    int32_t precision;       /* TSVD_PREC_FP64 (default) or TSVD_PREC_MIXED */
    int32_t restart_keep;    /* LancSVD restart: 0 (default) = the paper's basic restart from the
                                b leading left Ritz vectors; s > 0 = thick restart keeping the s
                                leading Ritz pairs (k <= s, s + b <= r b) and continuing from
                                the residual block, with (r b - s) / b new blocks per cycle;
                                in the mixed form the kept vectors have FP64 master copies (the
                                bases hold their FP32 rounding) */
} tsvd_opts;

/* Per-call report.  Phase times are CUDA-event milliseconds on `stream`. */
typedef struct tsvd_info {
    int32_t iterations;      /* RandSVD loop trips (q+1); LancSVD restart cycles run */
    int32_t restarts;        /* LancSVD restarts taken                              */
    int32_t breakdowns;      /* Cholesky breakdowns sent to the CGS2 fallback       */
    int32_t converged;       /* 1 if resid_max <= tol (LancSVD)                      */
    int32_t transposed;      /* 1 if m < n and the method ran on A^T                 */
    int32_t svd_sweeps;      /* Jacobi sweeps of the last small SVD                   */
    double resid_max;        /* max over j of ||A v_j - s_j u_j||_2 and ||A^T u_j - s_j v_j||_2,
                                divided by s_1, for the returned triplets */
    double rho_last;         /* last Lanczos residual estimate / s_1                  */
    double ms_total;         /* whole call, including the CSR transpose build         */
    double ms_transpose;     /* CSR(A^T) build                                         */
    int64_t kernel_launches; /* kernels this call enqueued                             */
    /* With TSVD_FLAG_PROFILE: per kernel class, the launches, their summed
     * CUDA-event time on `stream`, and the algorithmic flops and compulsory
     * bytes they were asked to do (Table 1 cost model, symmetric Gram counted
     * as its upper half).  Zero otherwise. */
    int64_t prof_launches[TSVD_K_COUNT];
    double prof_ms[TSVD_K_COUNT];
    double prof_flops[TSVD_K_COUNT];
    double prof_bytes[TSVD_K_COUNT];
} tsvd_info;

typedef struct tsvd_handle tsvd_handle;

/* Sums count doubles at buf (host memory) over the processes of a row partition, in
 * place; returns 0 on success.  Called by the library on the thread that made the
 * solver call, in the same order on every process. */
typedef int (*tsvd_allreduce_fn)(void* ctx, double* buf, int64_t count);

/* ---- lifetime ----------------------------------------------------------- */

/* Fills *opts with the defaults listed above. */
void tsvd_default_opts(tsvd_opts* opts);

/* Creates a handle bound to CUDA device `device` (queries its SM count and
 * kernel occupancy; allocates only the host-side struct).  *out = NULL on error. */
int tsvd_create(tsvd_handle** out, int device);

/* Frees the handle (host memory only).  NULL is accepted. */
int tsvd_destroy(tsvd_handle* h);

/* Sets the limit, in SM clock cycles, of every bounded device-side wait of the
 * kernels this handle launches afterwards: the mbarrier waits of the pipelined
 * tensor-core products (tsvd_mm_bf16x6, tsvd_dense_mm_f64tc and the solvers'
 * products) and the grid barrier of the block Jacobi SVD.  cycles <= 0 restores
 * the default of 2e9 cycles (about 1 s).  A wait that reaches the limit gives
 * up, the kernel stops its pipeline (copies and products already issued are
 * waited for with the default limit, tensor memory is freed) and the call
 * returns TSVD_ERR_TIMEOUT; the outputs are then undefined and the context stays
 * usable.  This is a test hook (a short limit makes the waits run out without
 * any fault); the paper has no counterpart.  TSVD_ERR_INVALID_ARG for a NULL
 * handle. */
int tsvd_set_wait_limit(tsvd_handle* h, long long cycles);

/* Row-partitioned LancSVD (Alg. 2 with the rows of A, and of the left basis Pbar,
 * split over processes; Sec. 3.2's CholeskyQR2 exchanges only b x b Gram matrices).
 * After this call tsvd_blanczos on this handle treats its matrix argument A (m x n,
 * CSR or dense, FP64, device) as rows [row0, row0 + m) of a rows_total x n matrix
 * whose other rows the other processes hold, with rows_total >= n:
 *   - the right basis P (n-side) is replicated: every process computes it, from the
 *     sum over processes of A_local^T Qbar_local (one n x b reduction per block);
 *   - the left blocks stay local; their Gram matrices, projection coefficients and
 *     norms are summed over the processes (b x b and s x b reductions);
 *   - B, its SVD and the stopping test are replicated, so every process takes the
 *     same path; the start block is rows [row0, row0 + m) of the one the whole
 *     matrix would get with the same seed;
 *   - outputs: sigma and V (n x k) replicated, U (m x k) this process's rows.
 * Each reduction is a call fn(ctx, buf, count) on a host buffer (the library copies
 * the device data to it and back), so any transport serves (MPI, a socket, a
 * torch.distributed group); every process must make the same solver calls in the
 * same order.  fn == NULL ends the partition.  Precision FP64 only; tsvd_rsvd and
 * the mixed form return TSVD_ERR_UNSUPPORTED on a partitioned handle.  The solve and
 * its tsvd_workspace_size call carry TSVD_FLAG_ROW_PARTITION in tsvd_opts.flags
 * (TSVD_ERR_INVALID_ARG when the flag and the handle disagree).  A failed
 * reduction gives TSVD_ERR_COMM.  The paper runs one GPU; this is the data-parallel
 * split of its method. */
int tsvd_set_row_partition(tsvd_handle* h, int64_t row0, int64_t rows_total, tsvd_allreduce_fn fn, void* ctx);

/* Static text for a status code. */
const char* tsvd_status_string(int status);

/* ---- drivers ------------------------------------------------------------ */

/* Workspace bytes for tsvd_rsvd (method TSVD_METHOD_RSVD, a = p, c = q) or
 * tsvd_blanczos (TSVD_METHOD_BLANCZOS, a = b, c = r) on A with k triplets. */
int tsvd_workspace_size(const tsvd_matrix* A, int method, int k, int a, int c,
                        const tsvd_opts* opts, size_t* bytes);

/* RandSVD, Alg. 1 (Sec. 2.1): block width l = k + p, q + 1 trips of S1-S4
 * (q power steps), then the SVD of R (S5) and the Ritz vectors (S6, S7).
 * The start block is N(0,1) Philox4x32-10 (key = seed, stream 1) unless
 * opts->start_block is given.  If m < n the method runs on A^T (Sec. 2).
 * Outputs: sigma[k] descending; U (m x k), V (n x k) row-major, ld = k; the
 * largest-magnitude entry of each v_j is positive.
 * Requires 1 <= k <= k + p <= min(m, n). */
int tsvd_rsvd(tsvd_handle* h, const tsvd_matrix* A, int k, int p, int q, uint64_t seed,
              const tsvd_opts* opts, void* ws, size_t ws_bytes,
              double* sigma, double* U, double* V, tsvd_info* info);

/* LancSVD, Alg. 2 (Sec. 2.2): blocks of width b, r blocks per cycle (Krylov
 * dimension r*b), full block re-orthogonalisation on both sides (Alg. 5),
 * basic restart with the b leading Ritz vectors (or the thick restart of
 * opts->restart_keep), repeated until the residual of every returned triplet
 * (tsvd_opts.tol) is <= opts->tol * s_1, or opts->max_restarts.  The explicit
 * residual is computed only at the end of a cycle whose Lanczos estimate
 * rho_j = ||R_r vbar_j[last b rows]|| has passed; it confirms the stop.
 * The start block is N(0,1) Philox4x32-10 (key = seed, stream 2),
 * orthonormalised by CholeskyQR2 (S1), unless opts->start_block is given.
 * Outputs as tsvd_rsvd.  Requires 1 <= b <= TSVD_MAX_BLOCK, r >= 1,
 * 1 <= k <= r*b <= min(m, n), r*b <= TSVD_MAX_SMALL_SVD.
 * Returns TSVD_NOT_CONVERGED if the tolerance was not met. */
int tsvd_blanczos(tsvd_handle* h, const tsvd_matrix* A, int k, int b, int r, uint64_t seed,
                  const tsvd_opts* opts, void* ws, size_t ws_bytes,
                  double* sigma, double* U, double* V, tsvd_info* info);

/* ---- building blocks ---------------------------------------------------- */

/* Start block (Sec. 4: N(0,1) start vectors): out[i*ld + j], i < rows, j < cols.
 * Element e = i*cols + j uses Philox4x32-10 (Salmon et al., SC'11) at counter
 * (e/2 mod 2^32, e/2 >> 32, stream_id, 0), key (seed mod 2^32, seed >> 32);
 * uniforms u = ((w_a >> 5) 2^26 + (w_b >> 6) + 1) 2^-53 from words (w0,w1), (w2,w3);
 * Box-Muller gives sqrt(-2 ln u1) cos(2 pi u2) (even e) or sin(...) (odd e). */
int tsvd_gaussian_block(int64_t rows, int64_t cols, uint64_t seed, uint32_t stream_id,
                        double* out, int64_t ld, void* stream);

/* CSR(A^T) of an m x n CSR matrix (needed by the A^T products, Table 1 S3 of
 * Alg. 1 and S2 of Alg. 2).  Outputs t_row_ptr[n+1], t_col_idx[nnz],
 * t_val[nnz]; within each row of A^T the entries are in increasing original
 * row order, so the output is deterministic.  Validates the input CSR on the
 * device (TSVD_ERR_INVALID_ARG on a bad structure). */
int tsvd_csr_transpose_workspace(int64_t m, int64_t n, int64_t nnz, size_t* bytes);
int tsvd_csr_transpose(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz,
                       const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                       int32_t* t_row_ptr, int32_t* t_col_idx, double* t_val,
                       void* ws, size_t ws_bytes, void* stream);

/* Y = A X for CSR A (m x n): X is n x w (ldx), Y is m x w (ldy), Table 1 SpMM.
 * Each y_i sums its row's entries in CSR order; a row longer than 1024 entries
 * is summed in chunks of 1024 whose partial sums are added in chunk order
 * (deterministic).  ws (tsvd_spmm_workspace bytes) holds the status words and
 * the chunk plan; an entry whose column lies outside [0, n) is skipped and
 * reported as TSVD_ERR_INVALID_ARG.  row_ptr must be a valid CSR row pointer
 * (row_ptr[0] = 0, non-decreasing, row_ptr[m] = nnz): the product reads each
 * row's extent from it unchecked, as sparse BLAS libraries do (tsvd_csr_transpose
 * and both methods validate the structure before their first product). */
int tsvd_spmm_workspace(int64_t m, int64_t nnz, int w, size_t* bytes);
int tsvd_spmm(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz,
              const int32_t* row_ptr, const int32_t* col_idx, const double* val,
              int w, const double* X, int64_t ldx, double* Y, int64_t ldy,
              void* ws, size_t ws_bytes, void* stream);
/* The same product in FP32 (values, X and Y float32; the mixed form's SpMM), with
 * the workspace tsvd_spmm_workspace reports. */
int tsvd_spmm_f32(tsvd_handle* h, int64_t m, int64_t n, int64_t nnz,
                  const int32_t* row_ptr, const int32_t* col_idx, const float* val,
                  int w, const float* X, int64_t ldx, float* Y, int64_t ldy,
                  void* ws, size_t ws_bytes, void* stream);

/* Y = op(A) X for dense row-major A (m x n, lda): trans = 0 gives A X
 * (X n x w, Y m x w); trans = 1 gives A^T X (X m x w, Y n x w).
 * The dense GEMM of Table 1 (the products marked * there). */
int tsvd_dense_mm_workspace(int trans, int64_t m, int64_t n, int w, size_t* bytes);
int tsvd_dense_mm(tsvd_handle* h, int trans, int64_t m, int64_t n, const double* A, int64_t lda,
                  int w, const double* X, int64_t ldx, double* Y, int64_t ldy,
                  void* ws, size_t ws_bytes, void* stream);

/* The same products, FP64-accurate, on the tensor cores (what the FP64 methods
 * run for their Gram, projection, update and Ritz products when the shape is
 * large enough; the dense GEMM rows of Table 1).  Each row of the left operand
 * and each column of the right operand is scaled by its own power of two and
 * split into 7 signed 8-bit digits held exactly in BF16 (exponent-aligned
 * slicing: Ozaki, Ogita, Oishi, Rump 2012; Ootomo, Ozaki, Yokota 2024); the 28
 * digit products of weight >= 2^-48 are summed as exact integers (BF16 MMAs with
 * FP32 accumulation over 128 terms, then 64-bit integers) and scaled back in
 * FP64.  With 2^ea_i, 2^eb_j the powers of two just above max_k |a_ik| and
 * max_k |x_kj| (K = the inner dimension):
 *   |Y - op(A) X|_ij <= 2^-56 (2^ea_i sum_k |x_kj| + sum_k |a_ik| 2^eb_j)
 *                       + 6.2 K 2^(ea_i + eb_j - 56) + 2^-52 P sum_k |a_ik x_kj|
 * (normwise FP64 accuracy; the middle term, the dropped digit products, is a
 * sum of mean-zero terms and in practice near sqrt(K) of that; P is the number
 * of FP64 partial sums the K range is cut into: one per CTA share of it and per
 * 8,192 k within a share, 1 when K <= 8,192 and the output has at least 152
 * tiles of 128 x 64).  Inf or NaN in
 * a row of op(A) or a column of X gives
 * NaN in the corresponding row (column) of Y.  Deterministic (fixed split and
 * summation order).  Workspace from tsvd_dense_mm_f64tc_workspace (planes of
 * both operands and split-K partial sums, 256-byte aligned).  Synchronises
 * `stream` before returning; a device wait that gives up returns
 * TSVD_ERR_TIMEOUT. */
int tsvd_dense_mm_f64tc_workspace(int trans, int64_t m, int64_t n, int w, size_t* bytes);
int tsvd_dense_mm_f64tc(tsvd_handle* h, int trans, int64_t m, int64_t n, const double* A, int64_t lda,
                        int w, const double* X, int64_t ldx, double* Y, int64_t ldy,
                        void* ws, size_t ws_bytes, void* stream);

/* The same products in FP32 (the mixed-precision form's kernels): A, X and Y
 * float32, products accumulated in FP32 within a row slab, and for trans = 1
 * the slabs' partial sums added in FP64 in a fixed order.  The workspace is
 * the one tsvd_dense_mm_workspace reports (it covers both element types). */
int tsvd_dense_mm_f32(tsvd_handle* h, int trans, int64_t m, int64_t n, const float* A, int64_t lda,
                      int w, const float* X, int64_t ldx, float* Y, int64_t ldy,
                      void* ws, size_t ws_bytes, void* stream);

/* ---- gradient of a loss on the k leading triplets (differentiation; the paper
 * has no backward pass) ----------------------------------------------------
 * Given the k leading triplets (sigma, U, V) of A, as tsvd_blanczos / tsvd_rsvd
 * return them, and the adjoints of a scalar loss L, sigma_bar = dL/dsigma (k),
 * U_bar = dL/dU (m x k), V_bar = dL/dV (n x k) (each may be NULL = 0), computes
 * dL/dA for the truncated SVD exactly (the other singular values of A need not
 * be zero):
 *   dL/dA = U C V^T + Y S V^T + U (A^T Y)^T + U S Z^T + (A Z) V^T,
 *   C = (F o (J - J^T)) S + diag(sigma_bar) + S (F o (K - K^T)),
 *   J = U^T U_bar, K = V^T V_bar, F_ij = 1/(s_j^2 - s_i^2) (i != j), S = diag(sigma),
 * with y_j, z_j the solutions of (s_j^2 I - A A^T) y_j = (I - UU^T) u_bar_j and
 * (s_j^2 I - A^T A) z_j = (I - VV^T) v_bar_j on the complements of span(U), span(V)
 * (conjugate gradients, one shift per column; positive definite there when
 * sigma_k > sigma_{k+1}).  Requires distinct sigma_1..sigma_k.
 *   grad: CSR A: nnz values on A's pattern, in CSR order (an SDDMM of the rank-2k
 *         factors); dense A: m x n row-major (ld n).  Device memory.
 *   All inputs are device FP64 row-major (U ld k, V ld k); A as for the solvers
 *   (FP64 or FP32 values, device or host).
 * Returns TSVD_NOT_CONVERGED (with the gradient of the last CG iterate) if a
 * solve did not reach cg_tol within cg_max_iter iterations. */
typedef struct tsvd_backward_opts {
    double cg_tol;           /* relative residual of every complement solve (default 1e-12) */
    int32_t cg_max_iter;     /* per side (default 20000) */
    int32_t check_every;     /* CG iterations between convergence reads (default 10) */
    void* stream;            /* cudaStream_t */
} tsvd_backward_opts;

typedef struct tsvd_backward_info {
    int32_t cg_iters_u;      /* CG iterations of the U-side (A A^T) solves */
    int32_t cg_iters_v;      /* CG iterations of the V-side (A^T A) solves */
    double cg_resid_u;       /* largest final relative residual, U side */
    double cg_resid_v;       /* same, V side */
    double ms_total;         /* device time of the call (CUDA events) */
} tsvd_backward_info;

void tsvd_default_backward_opts(tsvd_backward_opts* opts);
int tsvd_svd_backward_workspace(const tsvd_matrix* A, int k, const tsvd_backward_opts* opts, size_t* bytes);
int tsvd_svd_backward(tsvd_handle* h, const tsvd_matrix* A, int k, const double* sigma, const double* U,
                      const double* V, const double* sigma_bar, const double* U_bar, const double* V_bar,
                      double* grad, const tsvd_backward_opts* opts, void* ws, size_t ws_bytes,
                      tsvd_backward_info* info);

/* Tensor-core products of the mixed form for dense A.  A (or A^T) is stored
 * once as three BF16 pieces, A = A0 + A1 + A2 to 24 significant bits, and the
 * block X as three pieces too; Y = sum of the six terms A_i X_j with i + j <= 2
 * computed by tcgen05 BF16 MMAs with FP32 accumulation.  The dropped terms are
 * O(2^-24) relative, so Y is as accurate as an FP32 product of the same values
 * (|Y - P X| <= c u |P| |X| with u = 2^-24 and c a small multiple of the inner
 * dimension).  These are the products A Q and A^T Q of Alg. 1 S1/S3 and Alg. 2
 * S2/S4 in the mixed form; the paper itself computes them in FP64.
 *   tsvd_bf16x3_bytes: bytes of the pieces of a rows x cols matrix (layout
 *     [3][rows][ld] BF16, ld = cols rounded up to a multiple of 8).
 *   tsvd_bf16x3_split: pieces of A (trans = 0; rows = m, cols = n) or of A^T
 *     (trans = 1; rows = n, cols = m) for FP64 A (m x n, lda) into `pieces`
 *     (device, caller-owned, tsvd_bf16x3_bytes(rows, cols) bytes).
 *   tsvd_mm_bf16x6: Y (rows x w, ldy, FP32) = P X with P given by its pieces
 *     (rows x cols) and X (cols x w, ldx, FP32).  Any w >= 0 (done in panels of
 *     128 columns).  Returns TSVD_ERR_TIMEOUT if a bounded wait in the kernel
 *     gave up (Y is then undefined).  Synchronises `stream` before returning. */
int tsvd_bf16x3_bytes(int64_t rows, int64_t cols, size_t* bytes);
int tsvd_bf16x3_split(tsvd_handle* h, int trans, int64_t m, int64_t n, const double* A, int64_t lda,
                      void* pieces, void* stream);
int tsvd_mm_bf16x6_workspace(int64_t rows, int64_t cols, int w, size_t* bytes);
int tsvd_mm_bf16x6(tsvd_handle* h, int64_t rows, int64_t cols, const void* pieces, int w,
                   const float* X, int64_t ldx, float* Y, int64_t ldy,
                   void* ws, size_t ws_bytes, void* stream);

/* Workspace bytes for the orthogonalisation entry points below on a q-row
 * block of width b against s earlier columns. */
int tsvd_orth_workspace(int64_t q, int64_t s, int b, size_t* bytes);

/* CholeskyQR2, Alg. 4 (Sec. 3.2): in place Y (q x b, ldy) <- Q with Q^T Q = I and
 * R (b x b, row-major, ld = b, upper triangular, positive diagonal) with
 * Y_in = Q R, R = Lbar^T L^T.  On a Cholesky breakdown (pivot <= b*eps*max W_ii)
 * the block is redone by column-wise classical Gram-Schmidt with
 * re-orthogonalisation (Sec. 3.2); columns found numerically dependent are
 * replaced by Philox columns (key = seed, stream 0x100 + t, t = *replacements,
 * which is advanced).  *breakdowns (may be NULL) is incremented per fallback.
 * Requires 1 <= b <= TSVD_MAX_BLOCK, q >= b. */
int tsvd_cholqr2(tsvd_handle* h, int64_t q, int b, double* Y, int64_t ldy, double* R,
                 uint64_t seed, int* replacements, int* breakdowns,
                 void* ws, size_t ws_bytes, void* stream);

/* CGS-CQR2, Alg. 5 (Sec. 3.3): orthogonalises Y (q x b) in place against the
 * orthonormal columns of P (q x s, ldp), two passes of block classical
 * Gram-Schmidt each followed by a CholeskyQR step: Y_in = P H + Q R with
 * P^T Q = 0, Q^T Q = I.  H (s x b, ld = b) may be NULL when not wanted; it is
 * H + Hbar L^T (the exact sum of the two passes).  R as tsvd_cholqr2.
 * s = 0 reduces to tsvd_cholqr2. */
int tsvd_cgs_cqr2(tsvd_handle* h, int64_t q, int64_t s, int b, const double* P, int64_t ldp,
                  double* Y, int64_t ldy, double* H, double* R,
                  uint64_t seed, int* replacements, int* breakdowns,
                  void* ws, size_t ws_bytes, void* stream);

/* CGS-CQR2 (Alg. 5; s = 0: CholeskyQR2, Alg. 4) on FP32 blocks, as the
 * mixed-precision form runs it: P (q x s, ldp) and Y (q x b, ldy) FP32 (device);
 * H (s x b, ld = b, may be NULL) and R (b x b, ld = b) FP64, with the meaning,
 * breakdown fallback and seed/replacement rules of tsvd_cgs_cqr2.  The products
 * read FP32 blocks and accumulate in FP32 within a row slab; Gram matrices,
 * projection coefficients, Cholesky factors, H and R are FP64.  Each update
 * (Y - P H, and with s = 0 the first Y L^{-T}) runs as one fused pass with the
 * Gram matrix of its result (tsvd_update_gram_f32).  Workspace:
 * tsvd_orth_workspace(q, s, b).  Synchronises `stream` before returning. */
int tsvd_cgs_cqr2_f32(tsvd_handle* h, int64_t q, int64_t s, int b, const float* P, int64_t ldp,
                      float* Y, int64_t ldy, double* H, double* R,
                      uint64_t seed, int* replacements, int* breakdowns,
                      void* ws, size_t ws_bytes, void* stream);

/* Fused update + Gram of an FP32 block (the update of Alg. 5 S2/S7, Y - P H, or
 * the Y L^{-T} of Alg. 4, together with the Gram matrix that the next CholeskyQR
 * step factors, Sec. 3.2-3.3), in one pass over the rows of Y:
 *   Y (q x b, ldy, FP32) <- beta Y + alpha X M,   X (q x s, ldx, FP32),
 *                                                  M (s x b, ldm, FP64, rounded to FP32),
 *   W (b x b, ld = b, FP64, both halves) = Y^T Y of the updated Y.
 * upper != 0: M is upper triangular (entries below its diagonal are not read).
 * Y may be X itself (s == b, ldx == ldy): the update is done in place.  Y gets the
 * same bits as the unfused FP32 product; W sums FP32 products over a row slab and
 * the slabs in FP64 in a fixed order (bitwise reproducible).  1 <= b <= 128,
 * s >= 1.  All pointers are device memory owned by the caller; ws holds
 * tsvd_update_gram_f32_workspace(q, b) bytes.  Asynchronous on `stream`. */
int tsvd_update_gram_f32_workspace(int64_t q, int b, size_t* bytes);
int tsvd_update_gram_f32(tsvd_handle* h, int64_t q, int64_t s, int b, double alpha, const float* X, int64_t ldx,
                         const double* M, int64_t ldm, double beta, float* Y, int64_t ldy, int upper,
                         double* W, void* ws, size_t ws_bytes, void* stream);

/* CGS-QR, Alg. 3 (Sec. 3.1): QR of Y (q x r) by column blocks of width b
 * (the last one narrower if b does not divide r): Y <- Q in place, R (r x r,
 * ld = r) upper triangular assembled from [H_j; R_j].  1 <= b <= TSVD_MAX_BLOCK. */
int tsvd_cgs_qr(tsvd_handle* h, int64_t q, int r, int b, double* Y, int64_t ldy, double* R,
                uint64_t seed, int* replacements, int* breakdowns,
                void* ws, size_t ws_bytes, void* stream);

/* Small SVD (Alg. 1 S5, Alg. 2 S6) of the n x n matrix B (ldb) by one-sided
 * Jacobi (Hestenes) with a parallel round-robin ordering:
 * B = Ubar diag(sigma) Vbar^T, sigma descending, Ubar and Vbar n x n
 * row-major (ld = n).  nv = n accumulates every right vector; 0 <= nv < n
 * computes only the leading nv columns of Vbar, as B^T ubar_j / sigma_j (the
 * other columns of Vbar are left undefined, and only the leading nv columns of
 * Ubar follow the sign convention); this is what the methods use, and for
 * 64 < n <= 1024 it runs the block-Jacobi kernel.  Sign convention: the
 * largest-magnitude entry of each defined Vbar column is positive.
 * *sweeps (may be NULL) receives the sweep count.
 * Requires 1 <= n <= TSVD_MAX_SMALL_SVD. */
int tsvd_small_svd_workspace(int n, size_t* bytes);
int tsvd_small_svd(tsvd_handle* h, int n, const double* B, int64_t ldb, int nv,
                   double* Ubar, double* sigma, double* Vbar, int* sweeps,
                   void* ws, size_t ws_bytes, void* stream);

/* ---- allocation-free variant ------------------------------------------- */

/* Y = A^T X exactly as tsvd_dense_mm with trans = 1 (same kernels, same split
 * of the sum, same result), but without a workspace: the split-K partial sums
 * live in one device array of TSVD_NOALLOC_SCRATCH_BYTES compiled into the
 * library.  The paper has no counterpart; this exists for callers that cannot
 * allocate device memory, e.g. code running inside an application whose own
 * memory pool already holds the whole device, or latency-critical code that
 * must never call cudaMalloc/cudaFree (they can synchronise the device).
 *   - A: m x n row-major (lda), X: m x w (ldx), Y: n x w (ldy), all device
 *     memory owned by the caller.
 *   - Shapes whose partial sums would exceed TSVD_NOALLOC_SCRATCH_BYTES return
 *     TSVD_ERR_UNSUPPORTED before any device work.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress)
 *     with the handle's device made current, and restores the caller's
 *     current device before returning.
 *   - Every call on a device shares the one array: calls whose work overlaps on
 *     the GPU (other streams, other threads) race on it and must be serialised
 *     by the caller.  Nothing in it needs to start at zero.
 *   - Each GPU that loads the library keeps the array until the process exits.
 *   - Synchronises `stream` before returning, so the call blocks the host
 *     until the product is done. */
#define TSVD_NOALLOC_SCRATCH_BYTES (4 * 1024 * 1024)
int tsvd_dense_mm_t_noalloc(tsvd_handle* h, int64_t m, int64_t n, const double* A, int64_t lda,
                            int w, const double* X, int64_t ldx, double* Y, int64_t ldy,
                            void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TSVD_H_ */
