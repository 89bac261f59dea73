// Expensive potential with the nu = 3 readout on the tensor cores (float
// arithmetic elsewhere; the body is ace_group in k_ace.cuh with TCM != 0).
//
// A CTA of TC_ACE_WARPS = 4 warps takes groups of 4 consecutive atoms of the
// expensive list, a warp per atom as in the CUDA-core kernel, and three CTAs
// share an SM.  Per l-triple the warps write their atom's Z[m3][q1 n + q2]
// (bf16; with the hi/lo split also the remainders) into rows 16 w + m3 of a
// shared-memory A operand (the accumulator rows of an M = 64 product lie in
// TMEM lanes 32 (r / 16) + r % 16, so warp w's rows are in the lanes it may
// read), one thread issues kp / 16 tcgen05.mma (K = 16 each; three per slice
// with the split) against the triple's coefficients W as the B operand (16
// rows q3 x kp, streamed with the tile), accumulating V = Z W (64 x 16, f32)
// in 32 TMEM columns, and commits to an mbarrier; the warps take the Gaunt
// adjoints omega1 and omega2 meanwhile, wait (bounded), and read their rows
// of V: omega3 += mult3 V and E += sum A3 V.
// Shared memory: the A operand(s) (TC_M / 8 row groups x kp / 8 core matrices
// of TC_LBO_A bytes), then the tile buffers and the warp regions of AceLay.
#pragma once

#include <algorithm>

#include "k_ace.cuh"

namespace mixd {

template <int L, int NP, int TCM>
__global__ void __launch_bounds__(TC_ACE_WARPS * 32, TC_MIN_CTAS) k_ace_tc(Dev d, AceTab<float> tab, int nbuf) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ uint32_t s_tmem;
    // 128-byte aligned base, formed by pointer arithmetic on the shared array so
    // that the compiler keeps every access through it a shared-memory access
    unsigned char* sm = smem_tc + ((128u - (smem_u32(smem_tc) & 127u)) & 127u);
    const int tid = threadIdx.x, warp = tid >> 5;
    TcState tc;
    tc.kp = (tab.n * tab.n + 15) & ~15;
    tc.sbo = (tc.kp / 8) * TC_LBO_A;
    const int zbytes = (TC_M / 8) * tc.sbo;
    constexpr int NZ = TCM == 2 ? 2 : 1;
    tc.zhi = sm;
    tc.zlo = TCM == 2 ? sm + zbytes : nullptr;
    tc.nbuf = nbuf;
    tc.phase = 0u;
    tc.abort = 0;
    // the K padding of the A operand (columns n^2 .. kp - 1) stays zero
    for (int o = tid * 16; o < NZ * zbytes; o += blockDim.x * 16)
        *reinterpret_cast<uint4*>(sm + o) = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) tmem_alloc(smem_u32(&s_tmem), 32u);
    if (tid == 0) mbar_init(smem_u32(&s_bar), 1u);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tc.tmem = s_tmem;
    tc.bar = smem_u32(&s_bar);
    const int count = d.status[SW_NEXP];
    const int ng = (count + TC_ACE_WARPS - 1) / TC_ACE_WARPS;
    __shared__ int s_g;
    for (int g = ace_next_group(d, &s_g); g < ng; g = ace_next_group(d, &s_g))
        ace_group<float, L, NP, TCM>(d, tab, g * TC_ACE_WARPS, count, sm + NZ * zbytes, &tc);
    ace_groups_done(d);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tc.tmem, 32u);
    }
}

// dynamic shared memory of k_ace_tc (with 128 bytes for the base alignment)
inline size_t ace_tc_bytes(int tcm, int L, int NP, int n, int cap, int tile_max, int qb, int nbuf) {
    const int kp = (n * n + 15) & ~15;
    const size_t zbytes = (size_t)(TC_M / 8) * (kp / 8) * TC_LBO_A;
    const AceLay lay(tile_max, cap, n, qb, L, NP, 4, TC_ACE_WARPS, nbuf);
    return 128 + (size_t)(tcm == 2 ? 2 : 1) * zbytes + (size_t)lay.total;
}

// launch shape: one or two tile buffers, whichever lets more CTAs share an SM
// (two on a tie: the next tile then streams in during the current one); as
// many resident CTAs as fit (each holds 32 TMEM columns of 512)
template <int L, int NP, int TCM>
inline cudaError_t ace_tc_shape(int n, int cap, int tile_max, int qb, size_t* smem, int* grid, int* nbuf) {
    const void* kern = (const void*)k_ace_tc<L, NP, TCM>;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int best = 0, best_nb = 0;
    size_t best_bytes = 0;
    for (int nb = 2; nb >= 1; --nb) {
        const size_t bytes = ace_tc_bytes(TCM, L, NP, n, cap, tile_max, qb, nb);
        if (bytes + fa.sharedSizeBytes > (size_t)optin) continue;
        e = raise_smem_limit(kern, bytes);
        if (e != cudaSuccess) return e;
        // resident CTAs from the SM's registers, shared memory, threads and
        // TMEM (16 x 32 columns); the occupancy calculator reports a single CTA
        // for kernels that allocate tensor memory, whatever each allocates
        int smem_sm = 0, resv = 0;
        e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (e != cudaSuccess) return e;
        const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
        int per_sm = 65536 / (regs_warp * TC_ACE_WARPS);
        per_sm = std::min(per_sm, (int)((size_t)smem_sm / (bytes + fa.sharedSizeBytes + (size_t)resv)));
        per_sm = std::min(per_sm, 2048 / (TC_ACE_WARPS * 32));
        per_sm = std::min(per_sm, 16);
        if (per_sm > best) {
            best = per_sm;
            best_nb = nb;
            best_bytes = bytes;
        }
    }
    if (best < 1) return cudaErrorInvalidValue;
    e = raise_smem_limit(kern, best_bytes);
    if (e != cudaSuccess) return e;
    *smem = best_bytes;
    *grid = best * sm_count();
    *nbuf = best_nb;
    return cudaSuccess;
}

template <int NP, int TCM>
inline cudaError_t ace_tc_cfg_l(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid, int* nbuf) {
    switch (L) {
        case 0: return ace_tc_shape<0, NP, TCM>(n, cap, tile_max, qb, smem, grid, nbuf);
        case 1: return ace_tc_shape<1, NP, TCM>(n, cap, tile_max, qb, smem, grid, nbuf);
        case 2: return ace_tc_shape<2, NP, TCM>(n, cap, tile_max, qb, smem, grid, nbuf);
        case 3: return ace_tc_shape<3, NP, TCM>(n, cap, tile_max, qb, smem, grid, nbuf);
        case 4: return ace_tc_shape<4, NP, TCM>(n, cap, tile_max, qb, smem, grid, nbuf);
        case 5: return ace_tc_shape<5, NP, TCM>(n, cap, tile_max, qb, smem, grid, nbuf);
        case 6: return ace_tc_shape<6, NP, TCM>(n, cap, tile_max, qb, smem, grid, nbuf);
    }
    return cudaErrorInvalidValue;
}

template <int TCM>
inline cudaError_t ace_tc_cfg(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid, int* nbuf) {
    if (n <= 4) return ace_tc_cfg_l<4, TCM>(L, n, cap, tile_max, qb, smem, grid, nbuf);
    if (n <= 8) return ace_tc_cfg_l<8, TCM>(L, n, cap, tile_max, qb, smem, grid, nbuf);
    if (n <= 12) return ace_tc_cfg_l<12, TCM>(L, n, cap, tile_max, qb, smem, grid, nbuf);
    return ace_tc_cfg_l<16, TCM>(L, n, cap, tile_max, qb, smem, grid, nbuf);
}

template <int NP, int TCM>
inline void ace_tc_launch_l(const Dev& d, const AceTab<float>& tab, int L, size_t smem, int grid, int nbuf,
                            cudaStream_t s) {
    constexpr int T = TC_ACE_WARPS * 32;
    switch (L) {
        case 0: k_ace_tc<0, NP, TCM><<<grid, T, smem, s>>>(d, tab, nbuf); break;
        case 1: k_ace_tc<1, NP, TCM><<<grid, T, smem, s>>>(d, tab, nbuf); break;
        case 2: k_ace_tc<2, NP, TCM><<<grid, T, smem, s>>>(d, tab, nbuf); break;
        case 3: k_ace_tc<3, NP, TCM><<<grid, T, smem, s>>>(d, tab, nbuf); break;
        case 4: k_ace_tc<4, NP, TCM><<<grid, T, smem, s>>>(d, tab, nbuf); break;
        case 5: k_ace_tc<5, NP, TCM><<<grid, T, smem, s>>>(d, tab, nbuf); break;
        case 6: k_ace_tc<6, NP, TCM><<<grid, T, smem, s>>>(d, tab, nbuf); break;
    }
}

template <int TCM>
inline void ace_tc_launch(const Dev& d, const AceTab<float>& tab, int L, size_t smem, int grid, int nbuf,
                          cudaStream_t s) {
    if (tab.np == 4) ace_tc_launch_l<4, TCM>(d, tab, L, smem, grid, nbuf, s);
    else if (tab.np == 8) ace_tc_launch_l<8, TCM>(d, tab, L, smem, grid, nbuf, s);
    else if (tab.np == 12) ace_tc_launch_l<12, TCM>(d, tab, L, smem, grid, nbuf, s);
    else ace_tc_launch_l<16, TCM>(d, tab, L, smem, grid, nbuf, s);
}

}  // namespace mixd
