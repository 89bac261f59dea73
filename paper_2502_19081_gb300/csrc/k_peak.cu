// Fused multiply-add throughput microbenchmark (the arithmetic roofline used
// when stating the potential kernels' fraction of peak).  Each thread runs
// eight independent dependent chains x <- x * a + b; flops = 2 per FMA.
#include <algorithm>

#include "mix_launch.h"

namespace mixd {

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T* out, int iters, T a, T b) {
    T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x0 = fma(x0, a, b);
            x1 = fma(x1, a, b);
            x2 = fma(x2, a, b);
            x3 = fma(x3, a, b);
            x4 = fma(x4, a, b);
            x5 = fma(x5, a, b);
            x6 = fma(x6, a, b);
            x7 = fma(x7, a, b);
        }
    }
    const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == T(-12345.0)) out[blockIdx.x] = s;   // keeps the chains live
}

template <typename T>
static int fma_peak_t(cudaStream_t s, double* out) {
    T* sink = nullptr;
    const int blocks = sm_count() * 8, threads = 256;
    if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return MIX_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int iters = 256;
    double best = 0.0;
    for (int rep = 0; rep < 6; ++rep) {
        cudaEventRecord(e0, s);
        k_fma<T><<<blocks, threads, 0, s>>>(sink, iters, T(0.999999), T(1e-6));
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * 32.0 * iters * (double)blocks * threads;
        if (ms > 0) best = std::max(best, flops / (ms * 1e-3));
        if (ms < 20.f && iters < (1 << 24)) iters *= 4;   // grow until the launch is tens of ms
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (cudaGetLastError() != cudaSuccess || best <= 0) return MIX_ECUDA;
    *out = best;
    return MIX_OK;
}

int fma_peak(int precision, cudaStream_t s, double* out) {
    return precision == MIX_FP64 ? fma_peak_t<double>(s, out) : fma_peak_t<float>(s, out);
}

}  // namespace mixd
