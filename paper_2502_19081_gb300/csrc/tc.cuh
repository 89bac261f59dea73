// Fifth-generation tensor cores on sm_103a through inline PTX: tensor-memory
// (TMEM) allocation, shared-memory matrix descriptors, the bf16 x bf16 -> f32
// tcgen05.mma of one CTA, its completion through an mbarrier, and TMEM loads.
//
// Operands are built by the CTA's own threads in shared memory in the
// canonical K-major layout without swizzling: the matrix is cut into core
// matrices of 8 rows x 16 bytes (8 bf16 along K), each stored as 128
// contiguous bytes (row r of the core matrix at byte 16 r); `lbo` is the byte
// distance between core matrices adjacent along K, `sbo` between core matrices
// adjacent along M (or N).  One MMA instruction takes K = 16, i.e. two core
// matrices along K from its descriptor's start address.
//
// The accumulator D (M rows x N columns of f32) lives in TMEM, column j in
// column j of the allocation: for M = 128 row i in lane i, for M = 64 row i in
// lane 32 (i / 16) + i % 16 (the first 16 lanes of each quarter).  Warp w of
// the CTA may read lanes 32 (w % 4) .. 32 (w % 4) + 31 only.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace mixd {

// K strides of the operands of the expensive kernel's readout: A (Z rows, written
// by the warps) with 16 bytes of padding after each core matrix, so that the
// lanes of a warp storing one row spread over all banks; B (coefficients,
// built on the host) unpadded
constexpr int TC_LBO_A = 144;
constexpr int TC_LBO_B = 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (no swizzle, K-major, base offset 0)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the fifth-generation tensor cores
    return d;                 // layout type 0: no swizzle
}

// instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (+)= A B^T for one K = 16 slice; issued by one thread
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the mbarrier at `bar` receives one arrival once every MMA this thread issued
// before has completed
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// this thread's shared-memory writes become visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// one full warp: allocate ncols TMEM columns (a power of two >= 32), address to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive f32 columns of the warp's 32 lanes (thread t: lane base + t),
// waiting for the load inside the same statement
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// true once the phase of the given parity has completed; false after `limit`
// polls (each poll may suspend the thread for a short, hardware-defined time)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
    for (int i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// byte offset of element (row, k) in a K-major no-swizzle operand
__host__ __device__ __forceinline__ int tc_off(int row, int k, int lbo, int sbo) {
    return (row >> 3) * sbo + (k >> 3) * lbo + (row & 7) * 16 + (k & 7) * 2;
}

}  // namespace mixd
