// Inline-PTX helpers of the tcgen05 / TMA kernels (sm_103a): mbarriers with
// bounded waits, tiled TMA loads, tensor-memory allocation and loads, the
// shared-memory and instruction descriptors of kind::f16 MMAs, and the host-side
// tensor-map encoder.  Used by the split-BF16 product (k_tc.cu) and the
// FP64-accurate sliced product (k_oz.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace tsvd {
namespace tcx {

constexpr long long kMaxWait = 2000000000LL;  // clock64 cycles (about 1 s)

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ inline void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ inline void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ inline bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the completion of the phase with the given parity; false if the
// wait gave up (deadline, or another role raised the abort flag).
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                 long long max_wait = kMaxWait) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > max_wait) return false;
    }
    return true;
}
// The same with a short sleep between polls, for roles whose waits are long
// (frees issue slots for the warps that share the SM sub-partition).
__device__ inline bool mbar_wait_sleep(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                       long long max_wait = kMaxWait) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > max_wait) return false;
        __nanosleep(64);
    }
    return true;
}
// Bounded wait that ignores the abort flag (draining copies or products in flight).
__device__ inline void mbar_drain(uint32_t bar, uint32_t parity, long long max_wait = kMaxWait) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > max_wait) break;
}

__device__ inline void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ inline void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows of
// 64 bytes, 8-row groups 512 bytes apart (tile base 512-byte aligned).
__device__ inline uint64_t sdesc_sw64(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu)  // start address / 16
           | ((uint64_t)1 << 16)              // leading byte offset (unused for swizzled K-major)
           | ((uint64_t)(512 >> 4) << 32)     // stride byte offset: 8 rows x 64 B
           | ((uint64_t)1 << 46)              // descriptor version of tcgen05
           | ((uint64_t)4 << 61);             // swizzle mode: 64 B
}

// The same for rows of 32 bytes (16 BF16) with 32-byte swizzle: 8-row groups 256
// bytes apart (tile base 256-byte aligned); one K = 16 MMA covers a whole row.
__device__ inline uint64_t sdesc_sw32(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu)  // start address / 16
           | ((uint64_t)1 << 16)              // leading byte offset (unused for swizzled K-major)
           | ((uint64_t)(256 >> 4) << 32)     // stride byte offset: 8 rows x 32 B
           | ((uint64_t)1 << 46)              // descriptor version of tcgen05
           | ((uint64_t)6 << 61);             // swizzle mode: 32 B
}

// Instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ inline void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ inline void commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ inline void tmem_alloc(uint32_t dst_smem, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// 16 consecutive FP32 columns of the calling thread's TMEM lane.
__device__ inline void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 columns of the calling thread's TMEM lane: one load, one
// wait (the registers are defined only by the asm that also waits for them).
__device__ inline void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- host side ---------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
EncodeTiledFn encode_fn();

// 3-D map over `planes` BF16 matrices stored [planes][rows][ld] (ld in elements,
// a multiple of 8), K extent `cols`; box box_k (K) x box_rows x planes with a
// swizzle of 2 box_k bytes (box_k = 32: 64-byte swizzle, 16: 32-byte swizzle).
// Loads beyond `cols` or `rows` read zeros.
// pstride: elements between planes (default rows x ld).
bool make_plane_map(CUtensorMap* map, const void* base, int64_t cols, int64_t rows, int64_t ld, int box_rows,
                    int planes, int box_k = 32, int64_t pstride = -1);

}  // namespace tcx
}  // namespace tsvd
