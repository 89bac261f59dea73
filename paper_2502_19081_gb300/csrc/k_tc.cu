// Check of the tensor-core building block the expensive kernel's bf16 readout
// uses (tc.cuh): one CTA forms D = A B^T with M = 128 or 64, A [M][K] and
// B [N][K] bf16 (row-major in global memory, copied by the CTA's threads into
// the canonical K-major shared-memory layout with the same core-matrix strides
// as the readout), K / 16 tcgen05.mma instructions accumulating in TMEM, and
// all 128 TMEM lanes read back with tcgen05.ld by the four warps (lane l to
// row l of the output), so that the caller sees where each row of D lies.
#include "mix_launch.h"
#include "tc.cuh"

namespace mixd {

namespace {

__global__ void __launch_bounds__(128, 1) k_tc_selftest(const uint16_t* __restrict__ a, const uint16_t* __restrict__ b,
                                                        int m, int n, int k, float* __restrict__ d, int* status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ uint32_t tbase;
    unsigned char* sm = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int kc = k / 8;
    const int sbo_a = kc * TC_LBO_A, sbo_b = kc * TC_LBO_B;
    unsigned char* sa = sm;
    unsigned char* sb = sm + 16 * sbo_a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < m * k; e += blockDim.x) {
        const int r = e / k, c = e - r * k;
        *reinterpret_cast<uint16_t*>(sa + tc_off(r, c, TC_LBO_A, sbo_a)) = a[e];
    }
    for (int e = tid; e < n * k; e += blockDim.x) {
        const int r = e / k, c = e - r * k;
        *reinterpret_cast<uint16_t*>(sb + tc_off(r, c, TC_LBO_B, sbo_b)) = b[e];
    }
    uint32_t ncols = 32;
    while ((int)ncols < n) ncols <<= 1;
    if (warp == 0) tmem_alloc(smem_u32(&tbase), ncols);
    if (tid == 0) mbar_init(smem_u32(&bar), 1);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t t0 = tbase;
    if (tid == 0) {
        const uint32_t idesc = tc_idesc_bf16(m, n);
        for (int s = 0; s < k / 16; ++s) {
            const uint64_t ad = tc_desc(smem_u32(sa + s * 2 * TC_LBO_A), TC_LBO_A, sbo_a);
            const uint64_t bd = tc_desc(smem_u32(sb + s * 2 * TC_LBO_B), TC_LBO_B, sbo_b);
            tc_mma_bf16(t0, ad, bd, idesc, s > 0 ? 1u : 0u);
        }
        tc_commit(smem_u32(&bar));
    }
    const bool ok = mbar_wait(smem_u32(&bar), 0, 1 << 20);
    if (!ok && lane == 0) atomicOr(status, 1);
    tc_fence_after();
    const int row = 32 * warp + lane;
    for (int c0 = 0; c0 < n; c0 += 16) {
        float v[16];
        tmem_ld16(t0 + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) d[(size_t)row * n + c0 + j] = ok ? v[j] : __int_as_float(0x7fc00000);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(t0, ncols);
    }
}

}  // namespace

size_t tc_selftest_smem(int n, int k) { return (size_t)16 * (k / 8) * TC_LBO_A + (size_t)(n / 8) * (k / 8) * TC_LBO_B + 128; }

cudaError_t tc_selftest(const uint16_t* a, const uint16_t* b, int m, int n, int k, float* d, int* status,
                        cudaStream_t s) {
    const size_t smem = tc_selftest_smem(n, k);
    cudaError_t e = raise_smem_limit((const void*)k_tc_selftest, smem);
    if (e != cudaSuccess) return e;
    k_tc_selftest<<<1, 128, smem, s>>>(a, b, m, n, k, d, status);
    return cudaGetLastError();
}

}  // namespace mixd
