// Allocation-free variant of the dense product Y = A^T X (tsvd_dense_mm with
// trans = 1).  Its split-K partial sums live in one fixed device array compiled
// into the library instead of in a caller workspace, so a caller that cannot
// obtain device memory can still run the product.
//
// Who needs this: code that runs inside a host application which has already
// reserved the whole device through its own memory pool (a new cudaMalloc would
// fail or fragment that pool), and latency-critical callers that must not call
// cudaMalloc/cudaFree at all, because those calls may synchronise the whole
// device and stall unrelated work.  Such callers still pass their own A, X and Y.
//
// Cost of the design: every GPU that loads the library reserves the array
// (kNoAllocScratchBytes) until the process exits, and all calls share it.
#include "tsvd_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = TSVD_NOALLOC_SCRATCH_BYTES;  // split-K partial sums

// The shared scratch.  In host code this name is only a stand-in for the device
// object: its device address must be fetched with cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double)];

// Device address of the scratch on the current device.  It is looked up on every
// call rather than cached: a cached address would go stale if the application
// reset the device or rebuilt its context between calls.
int scratch_address(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return TSVD_ERR_CUDA;
    *out = p;
    return TSVD_OK;
}

}  // namespace

extern "C" int tsvd_dense_mm_t_noalloc(tsvd_handle* h, int64_t m, int64_t n, const double* A, int64_t lda, int w,
                                       const double* X, int64_t ldx, double* Y, int64_t ldy, void* stream) {
    if (!h || m < 0 || n < 0 || w < 0 || lda < n || !A || !X || !Y || ldx < w || ldy < w)
        return TSVD_ERR_INVALID_ARG;
    const size_t need = tsvd::gemm_tn_ws(h, m, n, w, false);
    if (need > kNoAllocScratchBytes) return TSVD_ERR_UNSUPPORTED;
    tsvd::DeviceGuard dg(h->device);
    if (!dg.ok()) return TSVD_ERR_CUDA;
    void* scratch = nullptr;
    TSVD_TRY(scratch_address(&scratch));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Every partial-sum slot the reduction reads is written first by the same
    // call, so nothing in the scratch has to start at zero.
    TSVD_TRY_CUDA(tsvd::gemm_tn(h, m, n, w, A, lda, X, ldx, Y, ldy, false, static_cast<double*>(scratch), st));
    TSVD_TRY_CUDA(cudaStreamSynchronize(st));
    return TSVD_OK;
}
