/*
 * mix.h - C ABI of the GB300 library for spatially mixed molecular dynamics
 * (force mixing of two local interatomic potentials, arXiv 2502.19081).
 *
 * One context holds one trajectory on one CUDA device.  Every step of the hot
 * path runs in the library's own sm_103a kernels: cell-list neighbour build,
 * blend weights lambda_i, evaluated sets with one-cutoff buffers, the expensive
 * many-body (linear cluster expansion) forces on lambda > 0 atoms plus buffer,
 * the cheap 2+3-body spline forces on lambda < 1 atoms plus buffer, the blend
 * F_i = w_i F_i^exp + (1 - w_i) F_i^cheap, and velocity-Verlet updates.
 *
 * Conventions for every call:
 *  - Return value: MIX_OK (0) or a negative MIX_E* code; no exceptions cross
 *    the boundary.  mix_strerror() names a code; mix_last_error() gives the
 *    context's last message.
 *  - Device work is enqueued asynchronously on the context's stream.  Errors
 *    detected by kernels (capacity overflow, non-finite values, an atom leaving
 *    a non-periodic box) surface at the next synchronising call: mix_sync(),
 *    the mix_get_* exports, mix_get_state() and the *_host entry points.
 *  - MIX_EOVERFLOW has two causes.  A neighbour row longer than the context's
 *    capacity is fatal for the context until it is re-created with a larger
 *    one.  A three-body neighbour count above what the cheap kernel's narrow
 *    lane groups hold (chosen at mix_init from the mean density) makes the
 *    context switch to a warp per atom for later evaluations; the forces of
 *    the failing evaluation are incomplete and the caller repeats it.
 *  - Ownership: positions, velocities, forces and the workspace are caller-owned
 *    device buffers that the library borrows from mix_bind() until the next
 *    mix_bind() or mix_destroy(); it never frees them.  Host arrays passed to
 *    mix_init() are copied.  A context allocates only host memory (plus pinned
 *    host memory for status reads); a batch's fused step and the serving layer
 *    allocate device memory of their own, described at their calls.
 *  - Layout: per-atom vectors are [N][4] float64 (x, y, z, unused), 32-byte rows,
 *    16-byte aligned or better.  Units: Angstrom, fs, eV, amu.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef MIX_H
#define MIX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MIX_OK 0
#define MIX_EINVAL (-1)     /* bad argument or unsupported configuration */
#define MIX_ENOMEM (-2)     /* workspace too small / host allocation failed */
#define MIX_ECUDA (-3)      /* a CUDA runtime call failed */
#define MIX_EOVERFLOW (-4)  /* a neighbour count exceeded its capacity */
#define MIX_ETIMEOUT (-5)   /* a bounded device wait gave up */
#define MIX_ENUMERIC (-6)   /* a non-finite position, force or energy */
#define MIX_ESTATE (-7)     /* call out of order (e.g. mix_forces before mix_bind) */
#define MIX_EBOX (-8)       /* an atom left the box in a non-periodic dimension */

/* arithmetic of the potential evaluations (integration, lambda and force
 * accumulation are always float64).  The bf16 modes are the float path with
 * the dense contraction of the nu = 3 product basis with the readout
 * coefficients (linear ACE readout, Sec. 2.1, Table 1), V = Z W with Z the
 * Gaunt-coupled product of two densities and W the coefficients, on the tensor
 * cores: bf16 operands, float accumulation; the site energy E = sum A3 V and
 * the adjoint omega3 = V follow from it, and each atom's energy is summed with
 * a compensation term.  MIX_BF16_SPLIT splits both operands into bf16 hi and
 * lo parts (x = hi + lo) and accumulates Zhi Whi + Zlo Whi + Zhi Wlo, about
 * 16 significant bits per product: the fallback when plain bf16 exceeds an
 * accuracy target.  A potential without nu = 3 terms runs the float path. */
#define MIX_FP64 0
#define MIX_FP32 1
#define MIX_BF16 2
#define MIX_BF16_SPLIT 3

/* region shapes (Sec. 4.4: core radius and blend width around a defect) */
#define MIX_REGION_SPHERE 0    /* distance to a centre point */
#define MIX_REGION_CYLINDER 1  /* distance to a line through centre along axis */

/* blend functions applied to the linear ramp (Sec. 4.4 names linear and cubic) */
#define MIX_BLEND_LINEAR 0
#define MIX_BLEND_CUBIC 1      /* w = lambda^2 (3 - 2 lambda) */

#define MIX_MAX_REGIONS 16
#define MIX_MAX_NRAD 16
#define MIX_MAX_LMAX 6

typedef struct mix_ctx mix_ctx;

/* The simulated system.  Periodic dimensions must have box_lo = 0 and at least
 * three cells of width >= max cutoff + skin, with box_len >= 2 (cutoff + skin)
 * (minimum image).  Non-periodic dimensions span [box_lo, box_lo + box_len);
 * an atom outside that range raises MIX_EBOX. */
typedef struct {
    int64_t n_atoms;
    double box_lo[3];
    double box_len[3];
    int periodic[3];
    double mass;            /* amu, single species */
} mix_system;

/* Expensive potential: a linear atomic cluster expansion (the paper's expensive
 * potentials are linear ACE, Sec. 2.1, Table 1).  Per site i,
 *   A_nlm = sum_{j: r_ij < r_cut} R_n(r_ij) Y_lm(r_ij / |r_ij|),
 *   R_n(r) = T_n(2 r / r_cut - 1) (1 - (r / r_cut)^2)^3  (Chebyshev T_n),
 *   Y_lm real orthonormal spherical harmonics without Condon-Shortley phase,
 *   E_i = 1/2 sum_j Vpair(r_ij) + sum_k c_k B_k(i)
 * with the product basis B of correlation order nu <= nu_max:
 *   nu = 1: A_n00;  nu = 2: sum_m A_n1lm A_n2lm (n1 <= n2);
 *   nu = 3: sum_{m1 m2 m3} G(l1 m1, l2 m2, l3 m3) A_n1l1m1 A_n2l2m2 A_n3l3m3,
 *   G = integral over the sphere of Y_l1m1 Y_l2m2 Y_l3m3, labels (l, n) sorted:
 *   l1 <= l2 <= l3, n1 <= n2 if l1 == l2, n2 <= n3 if l2 == l3,
 *   l1 + l2 + l3 even, l3 <= l1 + l2.
 * Coefficient tables (host, row-major, copied at mix_init):
 *   c1[n_rad], c2[l_max+1][n_rad][n_rad] (entries n1 <= n2 used),
 *   c3[l_max+1][l_max+1][l_max+1][n_rad][n_rad][n_rad] (sorted labels used; may
 *   be NULL when nu_max < 3), pair[16]: cubic B-spline pair coefficients on knots
 *   (a - 3) r_cut / 13 (NULL = no pair term). */
typedef struct {
    double r_cut;
    int n_rad;              /* 1 .. MIX_MAX_NRAD */
    int l_max;              /* 0 .. MIX_MAX_LMAX */
    int nu_max;             /* 1 .. 3 (body order - 1) */
    const double* c1;
    const double* c2;
    const double* c3;
    const double* pair;
} mix_ace;

/* Cheap potential: a 2+3-body cubic B-spline (the paper's UF3 family, Sec. 2.1):
 *   E_i = 1/2 sum_{j: r_ij < r_cut} V2(r_ij)
 *       + sum_{j<k: r_ij, r_ik < r_cut3} V3(r_ij, r_ik, r_jk),
 *   V2 = sum_{a<16} c2[a] B_a(r), knots (a - 3) r_cut / 13;
 *   V3 = sum_{a,b,c<8} c3[a][b][c] B_a(r_ij) B_b(r_ik) B_c(r_jk), knots
 *   (a - 3) r_cut3 / 5 for the first two arguments and (c - 3) 2 r_cut3 / 5 for
 *   the third; c3 must be symmetric in (a, b).  r_cut3 <= r_cut. */
typedef struct {
    double r_cut;
    double r_cut3;
    const double* c2;       /* [16] */
    const double* c3;       /* [8][8][8] */
} mix_spline;

typedef struct {
    int precision;          /* MIX_FP64, MIX_FP32, MIX_BF16 or MIX_BF16_SPLIT */
    double skin;            /* neighbour-list skin, Angstrom (> 0); lists rebuild
                               when an atom moved more than skin / 2 */
    int blend;              /* MIX_BLEND_* */
    double buffer_exp;      /* buffer radius of the expensive set; <= 0: its cutoff */
    double buffer_cheap;    /* buffer radius of the cheap set; <= 0: its cutoff */
    int nbr_cap;            /* neighbour slots per atom; 0: automatic */
    int no_graphs;          /* 0: mix_step replays each step as one captured CUDA
                               graph launch; nonzero: kernels are launched one by one */
    int potential_order;    /* how the two potential kernels of an evaluation share
                               the GPU (MIX_ORDER_*; mix_tune picks the fastest) */
} mix_options;

/* Orders of the two potential kernels (they write disjoint arrays, so every
 * order gives the same bits). */
enum {
    MIX_ORDER_CHEAP_FIRST = 0, /* two branches, the cheap kernel launched first, so
                                  that it fills the SMs a small expensive set leaves
                                  idle (default) */
    MIX_ORDER_EXP_FIRST = 1,   /* two branches, the expensive kernel launched first;
                                  the cheap one fills its last wave */
    MIX_ORDER_SERIAL = 2       /* one stream: the expensive kernel, then the cheap one,
                                  each with the whole GPU (their phase times are then
                                  their own durations) */
};

/* A core region.  d = distance of an atom from the shape (minimum image in
 * periodic dimensions); lambda = 1 for d < r_core, 1 - (d - r_core) / ramp for
 * d < r_core + ramp, else 0; the maximum over regions is taken (Alg. 2 takes
 * the maximum over core atoms; here the core is a geometric shape). */
typedef struct {
    int kind;               /* MIX_REGION_* */
    double centre[3];
    double axis[3];         /* cylinder direction (normalised by the library) */
    double r_core;
    double ramp;
} mix_region;

typedef struct {
    int64_t n_core;         /* lambda == 1 */
    int64_t n_ramp;         /* 0 < lambda < 1 */
    int64_t n_exp;          /* evaluated with the expensive potential (set + buffer) */
    int64_t n_cheap;        /* evaluated with the cheap potential (set + buffer) */
    int64_t rebuilds;       /* neighbour-list builds since mix_bind */
    int64_t steps;          /* velocity-Verlet steps since mix_bind */
    int max_neighbours;     /* largest list length seen at the last build */
    int status_bits;        /* raw device status word */
} mix_stats;

/* Create a context on the current CUDA device: one force-mixing simulation
 * (Sec. 4, Alg. 4) of a system with an expensive and a cheap potential
 * (Sec. 2.1: a linear atomic cluster expansion and a 2+3-body spline of the
 * UF3 family), each evaluated on its own set plus a one-cutoff buffer (Sec.
 * 4.5); the regions that weight them are set by mix_set_regions (Sec. 4.4) or
 * mix_set_seeds (Alg. 1-2).  The potentials' coefficients are copied (host
 * arrays may be freed after the call).  `cuda_stream` is a cudaStream_t
 * (NULL = legacy default stream).  Errors: MIX_EINVAL for unsupported sizes or
 * a box too small for the cutoff; MIX_ECUDA. */
int mix_init(const mix_system* sys, const mix_ace* expensive, const mix_spline* cheap,
             const mix_options* opt, void* cuda_stream, mix_ctx** out);

/* Device workspace the caller must provide to mix_bind (bytes, 256-aligned). */
int mix_workspace_bytes(const mix_ctx* ctx, size_t* bytes);

/* Borrow caller-owned device buffers: x, v, f are [N][4] float64; workspace has
 * at least mix_workspace_bytes bytes, 256-byte aligned.  Uploads the potential
 * tables into the workspace and marks the neighbour lists stale.  Does not read
 * x, v or f. */
int mix_bind(mix_ctx* ctx, double* x_dev, double* v_dev, double* f_dev, void* workspace_dev);

/* Set the core regions (at most MIX_MAX_REGIONS; n = 0 gives lambda = 0
 * everywhere, i.e. the pure cheap potential).  Takes effect at the next force
 * evaluation.  The paper rebuilds regions every step (Sec. 4.7); lambda is
 * recomputed at every force evaluation from the current positions. */
int mix_set_regions(mix_ctx* ctx, const mix_region* regions, int n);

/* Weights from seed atoms instead of regions (Alg. 1 and 2 of Sec. 4.4):
 * the seeds and every atom closer than r_core to a seed are core atoms
 * (lambda = 1); any other atom takes the largest 1 - r/r_blend over core atoms
 * closer than r_blend (lambda = 0 without one).  Distances are compared as
 * r^2 < r_core^2 and r^2 < r_blend^2 in float64, r = sqrt(r^2), with the
 * minimum image; the blend option (linear / cubic) applies to lambda as with
 * regions.  seeds: host array of n_seeds atom indices (duplicates allowed);
 * the mask is copied to the device before returning.  r_core and r_blend lie
 * in [0, largest cutoff] (both are found through the neighbour lists).
 * MIX_EINVAL for an index outside [0, N) or a radius out of range;
 * MIX_ESTATE before mix_bind.  mix_set_regions switches back to regions. */
int mix_set_seeds(mix_ctx* ctx, const int* seeds, int n_seeds, double r_core, double r_blend);

/* Seeds chosen on the device from the coordination number z_i (neighbours
 * closer than r_coord, strict), the defect criterion of the silicon vacancy
 * runs (Sec. 4.6): an atom is a seed when the mean of z_i lies in
 * [z_lo, z_hi].  The first force evaluation after this call seeds from its own
 * counts; after that z_i is summed over `period` evaluations and the seeds
 * are refreshed from the mean at the end of each period.  Core and blend
 * weights then follow mix_set_seeds.  r_coord, r_core, r_blend lie in
 * [0, largest cutoff]; period >= 1; z_lo <= z_hi.  MIX_EINVAL otherwise;
 * MIX_ESTATE before mix_bind. */
int mix_set_seed_rule(mix_ctx* ctx, double r_coord, double z_lo, double z_hi, int period, double r_core,
                      double r_blend);

/* Seed mask of the last evaluation ([N] 0/1, nullable) and the number of seeds
 * (nullable); synchronises. */
int mix_get_seeds(mix_ctx* ctx, uint8_t* seed /*[N]*/, int64_t* n_seeds);

/* f <- blended forces at the current positions (Alg. 4 with the buffer of
 * Sec. 4.5), rebuilding the neighbour lists first if needed. */
int mix_forces(mix_ctx* ctx);

/* nsteps velocity-Verlet steps of dt fs:
 *   v += dt/2 kappa F/m;  x += dt v;  F = mixed forces(x);  v += dt/2 kappa F/m,
 * kappa = 9.6485332e-3 A fs^-2 per (eV/A/amu).  Forces are evaluated first if
 * f does not hold the forces of the current positions. */
int mix_step(mix_ctx* ctx, double dt_fs, int nsteps);

/* End-to-end variant with host buffers: copies x and v ([N][4] float64, ideally
 * pinned) to the bound device buffers, runs nsteps steps, copies x, v and f
 * back, and synchronises.  x_host and v_host are updated in place; f_host
 * (nullable) receives the forces. */
int mix_step_host(mix_ctx* ctx, double* x_host, double* v_host, double* f_host, double dt_fs, int nsteps);

/* Wait for the context's stream and report device-side errors. */
int mix_sync(mix_ctx* ctx);

/* Counters of the last evaluation (synchronises). */
int mix_get_stats(mix_ctx* ctx, mix_stats* stats);

/* Debug / test exports: copy device state into caller host buffers
 * (synchronising).  Lists are the ones of the last build. */
int mix_get_cells(mix_ctx* ctx, int* ncell3, int* cell_of /*[N]*/);
int mix_get_neighbours(mix_ctx* ctx, int* cap_out, int* nnb /*[N] nullable*/, int* nbr /*[N][cap] nullable*/,
                       int* rev /*[N][cap] nullable*/);
int mix_get_lambda(mix_ctx* ctx, double* lam /*[N]*/, double* weight /*[N]*/);
/* flags bit0 lambda > 0, bit1 lambda < 1, bit2 expensive set or buffer,
 * bit3 cheap set or buffer; act lists ascending. */
int mix_get_sets(mix_ctx* ctx, uint8_t* flags /*[N]*/, int* act_exp /*[N] nullable*/, int64_t* n_exp,
                 int* act_cheap /*[N] nullable*/, int64_t* n_cheap);
int mix_get_site_energies(mix_ctx* ctx, double* e_exp /*[N]*/, double* e_cheap /*[N]*/);

/* Checkpoint: x, v, f, the list reference positions and the step counter.
 * mix_set_state marks the lists stale (they rebuild at the next evaluation). */
int mix_get_state(mix_ctx* ctx, double* x, double* v, double* f, int64_t* step);
int mix_set_state(mix_ctx* ctx, const double* x, const double* v, const double* f, int64_t step, int forces_valid);

int mix_destroy(mix_ctx* ctx);
const char* mix_strerror(int code);
const char* mix_last_error(const mix_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Measurement helpers.  The paper has no counterpart: they exist to time the  */
/* kernels and to state roofline fractions.                                   */

/* Kernel groups of one force evaluation, in launch order. */
#define MIX_PHASE_DISP 0     /* first half-kick, drift, skin test */
#define MIX_PHASE_LISTS 1    /* cell list and neighbour list (no-ops unless rebuilding) */
#define MIX_PHASE_SETS 2     /* weights, buffers, compaction */
#define MIX_PHASE_EXP 3      /* expensive potential (one kernel) */
#define MIX_PHASE_CHEAP 4    /* cheap potential (one kernel) */
#define MIX_PHASE_GATHER 5   /* gather, blend, second half-kick (one kernel) */
#define MIX_PHASES 6

typedef struct {
    int nbr_cap;            /* neighbour slots per atom */
    int n_tau;              /* l-triples of the nu = 3 basis */
    int64_t gaunt_nnz;      /* non-zero real Gaunt coefficients over all l-triples */
    int64_t tau_dim3_sum;   /* sum over l-triples of (2 l3 + 1) */
    int64_t basis_size;     /* number of product-basis functions */
    double nu3_flops_per_atom; /* nu = 3 readout and adjoint per evaluated atom, as
                                  the kernel contracts them (l1 >= l2 >= l3): sum over
                                  l-triples of U = W A3 and omega3 = W^T Z
                                  (2 (2l3+1) n^3 each), Z (2 nnz n^2), E (2 (2l3+1) n^2),
                                  omega1 (2 nnz n^2, unless all l equal) and omega2
                                  (2 nnz n^2, only for distinct l's) */
    size_t workspace_bytes;
    size_t exp_smem_bytes;  /* dynamic shared memory of the expensive kernel */
    int exp_grid;           /* its persistent grid (CTAs) */
    int exp_threads;
    size_t cheap_smem_bytes;
    int cheap_grid;
    int launches_per_evaluation;
    int64_t launches;       /* kernels enqueued since mix_bind */
    int gather_grid;        /* CTAs of the gather kernel */
    int build_grid;         /* CTAs of the neighbour-list kernel */
    int buffer_grid;        /* CTAs of the buffer-scan kernel */
    int exp_tensor_cores;   /* 1: the nu = 3 readout runs on the tensor cores (bf16 modes) */
    double tc_flops_per_atom;  /* algorithmic flops of that readout, V = Z W: sum over
                                  l-triples of 2 (2 l3 + 1) n^3 per evaluated atom */
    int cheap_lanes;        /* lanes per atom of the cheap kernel (8, 16 or 32); a periodic
                               bulk may narrow after its first evaluation, a 3-body
                               overflow widens to 32 */
    double nu3_flops_ref_per_atom; /* nu3_flops_per_atom with each l-triple's factors
                                  in ascending order (l3 the largest), the order the
                                  potential's coefficients are given in; the kernel
                                  contracts the factor of smallest l densely instead,
                                  which does less work (Sec. 2.1: the basis is
                                  symmetric in its three factors) */
    int potential_order;    /* MIX_ORDER_* in use */
} mix_info;

int mix_get_info(const mix_ctx* ctx, mix_info* info);

/* Enable (1) or disable (0) per-phase timing: CUDA events recorded on the
 * context stream between the kernel groups of every evaluation.  While
 * enabled, each evaluation synchronises on its last event so that the
 * durations can be accumulated.  Enabling resets the accumulators. */
int mix_profile(mix_ctx* ctx, int enable);

/* Accumulated and last-evaluation durations per phase (milliseconds). */
int mix_get_profile(mix_ctx* ctx, double* total_ms /*[MIX_PHASES] nullable*/, double* last_ms /*[MIX_PHASES]
                    nullable*/, int64_t* evaluations);

/* Measured fused multiply-add throughput of this device (flop/s, 2 per FMA)
 * for MIX_FP64 or MIX_FP32: independent FMA chains on every SM, timed with
 * CUDA events on `cuda_stream`.  Used as the arithmetic roofline.  Allocates
 * and frees a small device buffer (one value per block) for its result sink. */
int mix_fma_peak(int precision, void* cuda_stream, double* flops_per_s);

/* Check of the tensor-core building block of the bf16 readout (no counterpart
 * in the paper; used by the tests): D = A B^T with A [m][k] and B [n][k] bf16
 * (raw 16-bit patterns, row-major), m = 128 or 64, formed by one CTA with the
 * shared-memory operand layout, tcgen05.mma instructions and TMEM read-back of
 * the readout kernel.  d_dev [128][n] float32 receives TMEM lane l in row l
 * (for m = 128 row l of D; for m = 64, row r of D lies in lane
 * 32 (r / 16) + r % 16 and the other lanes hold no result).  All buffers are
 * caller-owned device memory.  16 <= n <= 256 and 16 <= k <= 160, both
 * multiples of 16 (else MIX_EINVAL).  *status_dev (device int, caller-cleared)
 * gets bit 0 set, and d is NaN, if the bounded wait for the MMAs gave up.
 * Asynchronous on cuda_stream. */
int mix_tc_selftest(const void* a_dev, const void* b_dev, int m, int n, int k, float* d_dev, int* status_dev,
                    void* cuda_stream);

/* ------------------------------------------------------------------------ */
/* Launch-shape autotuning and batches of trajectories.  The paper has no      */
/* counterpart (its runs are single LAMMPS jobs); these serve many independent */
/* defect cells on one GPU.                                                   */

/* Autotune one bound context: times force evaluations at the current
 * positions (which leave x, v and f unchanged) while varying, one at a time,
 * the order of the two potential kernels (MIX_ORDER_*), the lane groups of the
 * cheap kernel (a narrower group is tried only where the largest 3-body
 * neighbour count measured so far fills at most two thirds of its on-chip
 * slots; a later overflow reports MIX_EOVERFLOW and widens the groups again),
 * the persistent grid of each potential kernel and the grids of the gather and
 * buffer kernels, and keeps the fastest (reported by mix_get_info); the
 * forces do not depend on any of them.
 * reps: timed evaluations per candidate (median). */
int mix_tune(mix_ctx* ctx, int reps);

typedef struct mix_batch mix_batch;

/* Group n bound contexts that were all created on `cuda_stream`.  The batch
 * borrows them: keep them alive until mix_batch_destroy.  Each step of the
 * batch is one CUDA graph launch whose child graphs, one per member, have no
 * dependencies on one another, so the members' kernels overlap on the device.
 * Results equal those of stepping each member alone. */
int mix_batch_create(mix_ctx* const* members, int n, void* cuda_stream, mix_batch** out);

/* nsteps velocity-Verlet steps of every member (members whose forces are not
 * current, or whose lists are stale, are first evaluated individually). */
int mix_batch_step(mix_batch* b, double dt_fs, int nsteps);

/* Wait for the batch and report the first member error (mix_batch_last_error
 * names the member). */
int mix_batch_sync(mix_batch* b);

/* Autotune the batch: for grid divisors 1, 2, 4, 8, 16 applied to every
 * member's persistent and gather grids, times launches of a graph of all
 * members' force evaluations (state unchanged) and keeps the fastest divisor. */
int mix_batch_tune(mix_batch* b, int reps, int* chosen_divisor);

int mix_batch_destroy(mix_batch* b);
const char* mix_batch_last_error(const mix_batch* b);

/* Fused step (default on): when every member uses one precision and geometric
 * regions (mix_set_regions), a step is one launch per kernel for all members
 * together -- blocks are assigned to members by tables built when the batch
 * graph is (re)built, and the potentials walk flattened lists of every
 * member's evaluated atoms -- instead of one child graph per member.  Results
 * are identical either way.  The fused step allocates its own device arrays
 * (member descriptors, block tables, work lists: about 16 bytes per atom plus
 * 16 bytes per block) when its graph is built; mix_batch_destroy frees them.
 * Members with seed-atom weights fall back to child graphs.  Launch shapes of
 * the fused step do not use mix_batch_tune's divisor. */
int mix_batch_set_fused(mix_batch* b, int fused);

/* fused: 1 if the current step graph is the fused one; groups: kernel
 * instantiation groups of the expensive potential (members sharing lmax and
 * padded radial count); launches: kernels launched by fused steps so far.
 * Each pointer nullable. */
int mix_batch_info(const mix_batch* b, int* fused, int* groups, int64_t* launches);

/* ------------------------------------------------------------------------ */
/* Serving: many independent mixed-MD trajectories (requests) arriving over  */
/* time share one GPU.  The paper runs one trajectory at a time; this layer  */
/* packages the context and batch calls above for a stream of requests:      */
/* requests wait in a queue in arrival order, are admitted while their       */
/* device memory fits the server's budget (and the optional caps below), run */
/* together in one batched step graph (continuous batching: the batch is     */
/* rebuilt whenever a request joins or leaves), keep their state on the      */
/* device between steps, and leave when their step count is reached.  Each   */
/* request's results are those of the same context run alone (the batch     */
/* runs every member's own kernels on its own buffers).                      */
typedef struct mix_server mix_server;

typedef struct {
    double dt_fs;             /* time step of every request */
    size_t hbm_budget;        /* device bytes the requests may hold (0: free memory at creation minus hbm_reserve) */
    size_t hbm_reserve;       /* bytes kept free when hbm_budget = 0 (0: 2 GiB) */
    int64_t max_active_atoms; /* admission cap on atoms stepped together (0: none); a request larger than the
                                 cap is admitted only when nothing else runs */
    int max_active;           /* cap on concurrent requests (0: none) */
    int fifo;                 /* 1: strict arrival order; 0: a later request that fits may pass a blocked one */
} mix_server_options;

enum { MIX_REQ_QUEUED = 0, MIX_REQ_ACTIVE = 1, MIX_REQ_DONE = 2, MIX_REQ_FAILED = 3 };

typedef struct {
    int state;                /* MIX_REQ_* */
    int status;               /* MIX_OK, or the error that failed the request */
    int64_t n_atoms;
    int64_t steps_done, steps_total;
    size_t device_bytes;      /* x, v, f and workspace */
    double t_submit, t_admit, t_done;   /* seconds on the server's clock (-1: not yet) */
} mix_request_info;

typedef struct {
    int admitted, retired, failed;      /* by this tick */
    int active, queued;                 /* after this tick */
    int64_t active_atoms;               /* atoms stepped by this tick */
    int steps;                          /* steps run by this tick */
    size_t bytes_in_use;
    double step_ms;                     /* device time per step of the batched step graph */
    double admit_ms;                    /* host time of admission (allocation, upload, first forces) */
    double rebuild_ms;                  /* host time spent rebuilding the batch graph (after a join or leave) */
    double t;                           /* server clock at the end of the tick (s) */
} mix_tick_info;

/* All requests' work goes to cuda_stream.  MIX_ENOMEM when no budget is left. */
int mix_server_create(const mix_server_options* opt, void* cuda_stream, mix_server** out);

/* Queue a request: system, potentials, options (as for mix_init; the server's
 * stream is used), regions (as mix_set_regions), host x and v ([N][4] float64,
 * copied), nsteps >= 0.  The context is created here (host tables); device
 * memory is taken at admission.  MIX_ENOMEM if the request can never fit the
 * budget; other errors as mix_init.  *id receives the request's id (>= 1). */
int mix_server_submit(mix_server* s, const mix_system* sys, const mix_ace* expensive, const mix_spline* cheap,
                      const mix_options* opt, const mix_region* regions, int n_regions, const double* x_host,
                      const double* v_host, int64_t nsteps, int64_t* id);

/* Admit what fits, run min(max_steps, the fewest steps any active request has
 * left) batched steps (max_steps >= 1), retire finished requests (their final
 * x, v, f are copied to host memory and their device memory is released),
 * and fail requests whose own status reports an error (the others go on).
 * Synchronises.  info is nullable. */
int mix_server_tick(mix_server* s, int max_steps, mix_tick_info* info);

int mix_server_request(mix_server* s, int64_t id, mix_request_info* info);

/* Copy a finished request's final state ([N][4] float64 host arrays, each
 * nullable) and forget the request.  MIX_ESTATE if it is not DONE or FAILED
 * (a failed request returns its status and copies nothing). */
int mix_server_fetch(mix_server* s, int64_t id, double* x_host, double* v_host, double* f_host);

int mix_server_destroy(mix_server* s);
const char* mix_server_last_error(const mix_server* s);

/* The admission rule alone (host only, no GPU): queued requests in arrival
 * order with device bytes need[k] and atoms[k]; bytes_free left in the
 * budget; atoms_free left under max_active_atoms (< 0: no cap); active
 * requests now running; max_active (0: none); fifo as above.  admit[k] = 1
 * for each admitted request; returns how many. */
int mix_admission_plan(const size_t* need, const int64_t* atoms, int n_queued, size_t bytes_free, int64_t atoms_free,
                       int active, int max_active, int fifo, int* admit);

/* ------------------------------------------------------------------------ */
/* Neighbour lists for callers that cannot allocate device memory.  The paper  */
/* has no counterpart: this is a packaging of the library's own list build.   */
/*                                                                            */
/* Some callers may not call cudaMalloc: a plugin inside a host program that  */
/* owns every device allocation through its own pool, or a time-critical loop */
/* that cannot take the device-wide synchronisation an allocation implies.    */
/* This entry point builds the same full, sorted neighbour lists and reverse- */
/* slot map as a context does (cell list, r2 < r_list^2 with the minimum      */
/* image, rows ascending), but keeps all of its scratch -- a folded copy of   */
/* the positions, the cell list, status words -- in one fixed device array    */
/* inside the library (about 3.6 MB, reserved on every GPU that loads the     */
/* library until the process exits).  It calls no cudaMalloc, cudaFree or     */
/* allocating library routine.                                                */
/*                                                                            */
/* Inputs and outputs are the caller's device buffers: x_dev [N][4] float64   */
/* (16-byte aligned, read only), nnb_dev [N], nbr_dev [N][cap], rev_dev       */
/* [N][cap] int32.  The box follows mix_system's rules.  Limits: N <=         */
/* MIX_NOALLOC_MAX_ATOMS, cells <= MIX_NOALLOC_MAX_CELLS, 1 <= cap <= 256;     */
/* anything larger returns MIX_EINVAL before touching the GPU.  A row longer  */
/* than cap returns MIX_EOVERFLOW (rows are then truncated).  A non-finite    */
/* coordinate returns MIX_ENUMERIC, one outside a non-periodic dimension of   */
/* the box MIX_EBOX (the lists are then meaningless).                         */
/*                                                                            */
/* The call enqueues its work on cuda_stream and waits for it.  The first     */
/* call on a device looks up the array's device address (cudaGetSymbolAddress */
/* with that device current); make that first call before any stream capture. */
/* Every call shares the one array and clears what must start at zero; calls  */
/* whose work overlaps on the GPU (other streams, other host threads) race on */
/* it and must be serialised by the caller.                                   */
#define MIX_NOALLOC_MAX_ATOMS 32768
#define MIX_NOALLOC_MAX_CELLS 16384
int mix_neighbours_noalloc(int64_t n_atoms, const double* x_dev, const double* box_lo /*[3]*/,
                           const double* box_len /*[3]*/, const int* periodic /*[3]*/, double r_list, int cap,
                           int* nnb_dev, int* nbr_dev, int* rev_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MIX_H */
