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

// expensive potential (k_ace.cuh, k_ace_f32.cu, k_ace_f64.cu); returns cudaSuccess or the launch error;
// wn: warps (atoms) a CTA, ACE_GROUP or ACE_MAX_WARPS
cudaError_t ace_configure(int precision, int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid,
                          int wn);
void launch_ace(const Dev& d, const void* tab, int precision, int L, size_t smem, int grid, int wn, cudaStream_t s);
cudaError_t ace_configure_f32(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid, int wn);
cudaError_t ace_configure_f64(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid, int wn);
void launch_ace_f32(const Dev& d, const void* tab, int L, size_t smem, int grid, int wn, cudaStream_t s);
void launch_ace_f64(const Dev& d, const void* tab, int L, size_t smem, int grid, int wn, cudaStream_t s);

// expensive potential with the tensor-core readout (k_ace_tc.cu; float tables
// with the bf16 operand sections): tcm 1 bf16, 2 bf16 hi/lo.  *nbuf: tile
// buffers that fit shared memory (2, else 1); cudaErrorInvalidValue when even
// one does not fit
cudaError_t ace_tc_configure(int tcm, int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid,
                             int* nbuf);
void launch_ace_tc(const Dev& d, const void* tab, int tcm, int L, size_t smem, int grid, int nbuf, cudaStream_t s);

// the Gaunt table of the float expensive kernels into the constant memory of
// every module that holds them, on the current device (k_ace_f64.cu dispatches)
cudaError_t ace_gaunt_upload(const void* ent_f, int n_ent, const int* rows, int n_rows);
cudaError_t ace_gaunt_upload_f32(const void* ent_f, int n_ent, const int* rows, int n_rows);
cudaError_t ace_gaunt_upload_tc1(const void* ent_f, int n_ent, const int* rows, int n_rows);
cudaError_t ace_gaunt_upload_tc2(const void* ent_f, int n_ent, const int* rows, int n_rows);

// tensor-core building block check (k_tc.cu)
cudaError_t tc_selftest(const uint16_t* a, const uint16_t* b, int m, int n, int k, float* d, int* status,
                        cudaStream_t s);

// cheap potential (k_spline.cu)
// lpa: lanes per evaluated atom (32, or 16 or 8 for atoms with few neighbours);
// spline_nb3(lpa): three-body neighbours an atom may have on chip with lpa lanes
cudaError_t spline_configure(int precision, int lpa, size_t* smem, int* grid);
int spline_nb3(int lpa);
void launch_spline(const Dev& d, const void* tab, int precision, int lpa, size_t smem, int grid, cudaStream_t s);

// gather + blend + second half-kick (k_gather.cu)
void launch_gather(const Dev& d, int precision, int integrate, double h, cudaStream_t s);

// ---------------------------------------------------------------------------
// multi-system step (batches of contexts sharing one stream)

// Block-table classes: every batched launch uses the table of its granularity.
enum BatchTabClass : int {
    BT_ATOM = 0,   // 256 threads, a thread per atom (grid-stride)
    BT_ONE,        // one block per system
    BT_NB,         // 4 warps, a warp per atom (list build)
    BT_REV,        // 8 warps, a warp per atom (reverse map)
    BT_WARP8,      // 8 warps of 32 atoms each (buffer scan)
    BT_SCAN,       // SCAN_BLOCK atoms per block, the system's own block count
    BT_GATHER,     // 8 warps of 32 atoms each (gather)
    BT_COUNT
};

struct FlatArgs {
    const Dev* devs;
    int nsys;
    int ngrp;
    const int* egroup;   // [nsys] expensive group (systems sharing T, L, NP)
    const int* elast;    // [nsys] 1 for the last system of its group
    const int* ebase;    // [ngrp] start of each group in list_e
    int2* list_e;        // {system, index in its expensive list}
    int2* list_c;        // {system, atom} for each entry of the systems' cheap lists
    int* counts;         // [ngrp + 1] expensive totals per group, cheap total
};

struct BatchPlan {
    BatchArgs ba[BT_COUNT];
    int nblk[BT_COUNT];
    const Regions* regions;   // [nsys]
    int capp2;                // largest power-of-two list capacity (build scratch)
    FlatArgs flat;
};

void launch_disp_batch(const BatchPlan& p, cudaStream_t s, int integrate, double dt, int force_rebuild);
void launch_build_batch(const BatchPlan& p, cudaStream_t s);
void launch_sets_batch(const BatchPlan& p, cudaStream_t s);
cudaError_t ace_batch_configure(int precision, int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid);
cudaError_t ace_batch_configure_f32(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid);
cudaError_t ace_batch_configure_f64(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid);
void launch_ace_batch(int precision, const Dev* devs, const void* tabs, const int2* list, const int* count, int n,
                      int L, size_t smem, int grid, cudaStream_t s);
void launch_ace_batch_f32(const Dev* devs, const void* tabs, const int2* list, const int* count, int n, int L,
                          size_t smem, int grid, cudaStream_t s);
void launch_ace_batch_f64(const Dev* devs, const void* tabs, const int2* list, const int* count, int n, int L,
                          size_t smem, int grid, cudaStream_t s);
cudaError_t spline_batch_configure(int precision, int lpa, size_t* smem, int* grid);
void launch_spline_batch(int precision, int lpa, const Dev* devs, const void* tabs, const int2* list,
                         const int* count, int uniform, size_t smem, int grid, cudaStream_t s);
void launch_gather_batch(const BatchPlan& p, int precision, int integrate, double dt, cudaStream_t s);

int sm_count();

// Raise (never lower) a kernel's dynamic shared-memory limit to `bytes`.  The
// limit belongs to the kernel, not to a context: contexts of different sizes
// share kernel instantiations, so one context must not shrink another's limit.
cudaError_t raise_smem_limit(const void* func, size_t bytes);

// FMA throughput microbenchmark (k_peak.cu)
int fma_peak(int precision, cudaStream_t s, double* flops_per_s);

}  // namespace mixd
