// Host-side launchers of the library's kernels (one definition per .cu file).
#pragma once

#include "mix_dev.cuh"

namespace mixd {

// lists (k_lists.cu)
void launch_disp(const Dev& d, cudaStream_t s, int integrate, double dt, double h, int force_rebuild);
void launch_build(const Dev& d, cudaStream_t s);

// weights, sets, compaction (k_sets.cu)
void launch_sets(const Dev& d, const Regions& r, const SeedRule& sr, cudaStream_t s);
int sets_launches(const SeedRule& sr);   // kernels launch_sets enqueues

// expensive potential (k_ace.cuh, k_ace_f32.cu, k_ace_f64.cu); returns cudaSuccess or the launch error
cudaError_t ace_configure(int precision, int L, int n, int cap, size_t* smem, int* grid);
void launch_ace(const Dev& d, const void* tab, int precision, int L, size_t smem, int grid, cudaStream_t s);
cudaError_t ace_configure_f32(int L, int n, int cap, size_t* smem, int* grid);
cudaError_t ace_configure_f64(int L, int n, int cap, size_t* smem, int* grid);
void launch_ace_f32(const Dev& d, const void* tab, int L, size_t smem, int grid, cudaStream_t s);
void launch_ace_f64(const Dev& d, const void* tab, int L, size_t smem, int grid, cudaStream_t s);

// cheap potential (k_spline.cu)
cudaError_t spline_configure(int precision, int cap, size_t* smem, int* grid);
void launch_spline(const Dev& d, const void* tab, int precision, size_t smem, int grid, cudaStream_t s);

// gather + blend + second half-kick (k_gather.cu)
void launch_gather(const Dev& d, int precision, int integrate, double h, cudaStream_t s);

int sm_count();

// Raise (never lower) a kernel's dynamic shared-memory limit to `bytes`.  The
// limit belongs to the kernel, not to a context: contexts of different sizes
// share kernel instantiations, so one context must not shrink another's limit.
cudaError_t raise_smem_limit(const void* func, size_t bytes);

// FMA throughput microbenchmark (k_peak.cu)
int fma_peak(int precision, cudaStream_t s, double* flops_per_s);

}  // namespace mixd
