// Internal definitions shared by the library's kernels and its host code.
// Not part of the public interface (include/mix.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mix.h"

namespace mixd {

// ---------------------------------------------------------------------------
// status words (int32, start of the workspace)
enum StatusBits : int {
    ST_NBR_OVERFLOW = 1,     // a neighbour list exceeded its capacity
    ST_REV_MISSING = 2,      // list asymmetry (should never happen)
    ST_NB3_OVERFLOW = 4,     // more than NB3MAX three-body neighbours
    ST_NONFINITE = 8,        // non-finite position or force
    ST_OUT_OF_BOX = 16,      // atom outside a non-periodic dimension
    ST_TC_TIMEOUT = 32,      // a bounded wait for tensor-core MMAs gave up
};
enum StatusWord : int {
    SW_STATUS = 0,
    SW_REBUILD = 1,     // 1: lists must be rebuilt in this evaluation
    SW_MAXNB = 2,       // largest list length at the last build
    SW_NEXP = 3,        // |A_exp|
    SW_NCHEAP = 4,      // |A_cheap|
    SW_REBUILDS = 5,    // number of builds
    SW_NCORE = 6,
    SW_NRAMP = 7,
    SW_NLE = 8,         // lambda > 0
    SW_NLC = 9,         // lambda < 1
    SW_NB3MAX = 10,     // largest 3-body neighbour count seen
    SW_EVALS = 11,      // evaluations since the seed rule was set (coordination averaging)
    SW_NSEED = 12,      // number of seed atoms
    SW_EPOCH = 13,      // force evaluations since binding (stamps the incoming gradient rows)
    SW_ACE_NEXT = 14,   // next group of expensive atoms to hand out (0 between launches)
    SW_ACE_DONE = 15,   // CTAs of the expensive kernel that have finished (0 between launches)
    SW_COUNT = 64,
};

constexpr int NB3MAX = 32;          // three-body neighbours per atom handled on chip
constexpr int MAX_CAP = 256;        // neighbour slots per atom
constexpr int SCAN_BLOCK = 1024;    // atoms per block in the set compaction

struct Box {
    double lo[3], L[3], invL[3];
    int per[3];
};

struct Cells {
    int nc[3];
    int ncell;
    double invh[3];
    double h[3];     // cell widths L / nc
    float hf[3];
};

// position relative to the origin of cell (cx, cy, cz), rounded once to float
__device__ __forceinline__ float4 cell_relative(const Box& b, const Cells& c, const double4& x, int c3) {
    const int cc[3] = {c3 & 1023, (c3 >> 10) & 1023, (c3 >> 20) & 1023};
    const double xs[3] = {x.x, x.y, x.z};
    float r[3];
    for (int k = 0; k < 3; ++k) r[k] = (float)(xs[k] - (b.lo[k] + (double)cc[k] * c.h[k]));
    return make_float4(r[0], r[1], r[2], 0.f);
}

struct Regions {
    int n;
    int blend;
    double r[MIX_MAX_REGIONS][9];   // kind, centre[3], axis[3] (unit), r_core, ramp
    // float screen of the weights (when screen != 0): an atom whose float
    // position of the last list build lies farther than sqrt(far2[k]) from region
    // k (from its axis for a cylinder) gets lambda 0 from it and leaves the
    // buffer hints alone; far2 = (r_core + ramp + r_buffer_exp + skin/2 + 0.01)^2
    // covers the drift since the build (< skin/2) and the float rounding (< 1e-3 A)
    int screen;
    float cf[MIX_MAX_REGIONS][6];   // centre[3], axis[3]
    float far2[MIX_MAX_REGIONS];
    float Lf[3], iLf[3];            // box lengths and inverses
};

// Weights from seed atoms instead of geometric regions (Alg. 1-2).
struct SeedRule {
    int mode;          // 0: geometric regions; 1: explicit seeds; 2: seeds from coordination
    int blend;         // MIX_BLEND_*
    double rcore2, rblend2, rblend;
    double rz2;        // coordination radius squared
    double zlo, zhi;   // seed when the averaged coordination lies in [zlo, zhi]
    int period;        // evaluations averaged per seed refresh
};

// Pointers into the workspace plus scalar parameters, passed by value.
constexpr double MIX_KAPPA = 9.6485332e-3;   // (eV / Angstrom / amu) in Angstrom / fs^2

// half-kick factor of velocity Verlet, h = dt/2 kappa / m (one expression for
// every caller, so single and batched steps round identically)
__host__ __device__ __forceinline__ double half_kick(double dt, double mass) {
    return 0.5 * dt * MIX_KAPPA / mass;
}

struct Dev {
    int64_t n;
    int cap;
    double mass;         // amu
    Box box;
    Cells cells;
    double rlist2;       // (rc_max + skin)^2
    double half_skin2;   // (skin / 2)^2
    double rce, rce2;    // expensive cutoff
    double rcc, rcc2;    // cheap 2-body cutoff
    double rc3;          // cheap 3-body cutoff
    double bufe2, bufc2; // buffer radii squared
    double bufe, bufc;   // buffer radii
    // float screen of the buffer test: a float squared distance below lo is
    // inside, above hi outside (1e-3 A^2 either side of the radius, against a
    // float error below 1e-4 A^2); in between the float64 test decides
    float bufe2_lo, bufe2_hi, bufc2_lo, bufc2_hi;
    int gat_lpa;         // lanes per atom of the gather (8, 16, 32), from the mean list length
    int exact_lists;     // 1: every neighbour candidate takes the float64 test
                         // (boxes beyond the float pre-filter's error bound)
    double4* x;
    double4* v;
    double4* f;
    double4* xb;
    float4* xf;          // float copy of the folded positions at the last build
    float4* xr;          // position minus the origin of its cell (cell of the last build), float
    int* cell3;          // cell coordinates of the last build, packed cx | cy << 10 | cz << 20
    int* status;
    int* cell_of;
    int* cell_count;
    int* cell_start;
    int* cell_fill;
    int* cell_atoms;
    int* nnb;
    int* nbr;
    int* rev;
    double* lam;
    double* wgt;
    uint8_t* flags;
    int* act_e;
    int* act_c;
    int* pos_e;
    int* pos_c;
    int* blk_e;
    int* blk_c;
    void* ge;            // [N][cap] real4: dE_i/dr_ij of the expensive potential, row of atom i
    void* gc;            // [N][cap] real4: same for the cheap potential
    void* ge_in;         // [N][cap] real4: row of atom j, slot rev: the partner's dE_i/dr_ij,
    void* gc_in;         //   w = the evaluation (epoch) that wrote it; same for the cheap potential
    double* esite_e;
    double* esite_c;
    // float path: the compensated (sum, correction) pairs of the site energies
    // of the two potentials ([N] each); the gather turns them into float64 site
    // energies 32 atoms at a time
    float2* epark_e;
    float2* epark_c;
    uint8_t* seed;       // [N] seed atoms (seed-atom weights)
    uint8_t* core;       // [N] core atoms
    int* zsum;           // [N] coordination summed over the current averaging period
    int nblk;            // blocks of the compaction kernels
    // launch shapes chosen by the autotuner (0: default)
    int grid_build;      // CTAs of the neighbour-list build (4 warps each)
    int grid_buffer;     // CTAs of the buffer scan (8 warps each)
    int grid_gather;     // CTAs of the gather (8 warps each)
};

// ---------------------------------------------------------------------------
// Multi-system launches (batches of independent systems).  A launch's blocks
// are assigned to systems by a table of int4 {system, local block index,
// local block count, 0}; every block works on one system and loads that
// system's Dev into shared memory, so kernel bodies written for one system
// (taking d, the local block index bx and the local grid size gx) run
// unchanged.  Kernels whose work list is built on the device (the potentials)
// instead walk a flattened list of {system, index in the system's list}.
struct BatchArgs {
    const Dev* devs;     // [nsys]
    const int4* tab;     // block table of this launch
};

// block-wide copy of a parameter struct into shared memory (callers sync)
template <typename S>
__device__ __forceinline__ void copy_shared(S* dst, const S* src) {
    static_assert(sizeof(S) % 8 == 0, "8-byte words");
    const unsigned long long* a = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* b = reinterpret_cast<unsigned long long*>(dst);
    for (int k = threadIdx.x; k < (int)(sizeof(S) / 8); k += blockDim.x) b[k] = a[k];
}

__device__ __forceinline__ void load_dev(Dev* dst, const Dev* src) { copy_shared(dst, src); }

// Opens a batched kernel: s_dev (the block's system), s_ent (its table entry).
#define MIX_BATCH_BLOCK(ba)                                  \
    __shared__ Dev s_dev;                                    \
    __shared__ int4 s_ent;                                   \
    if (threadIdx.x == 0) s_ent = (ba).tab[blockIdx.x];      \
    __syncthreads();                                         \
    load_dev(&s_dev, (ba).devs + s_ent.x);                   \
    __syncthreads();

// The same for kernels that only work on list rebuilds: the block returns
// before loading anything when its system keeps its lists.
#define MIX_BATCH_BLOCK_REBUILD(ba)                                       \
    __shared__ Dev s_dev;                                                 \
    __shared__ int4 s_ent;                                                \
    __shared__ int s_go;                                                  \
    if (threadIdx.x == 0) {                                               \
        s_ent = (ba).tab[blockIdx.x];                                     \
        s_go = (ba).devs[s_ent.x].status[SW_REBUILD];                     \
    }                                                                     \
    __syncthreads();                                                      \
    if (s_go == 0) return;                                                \
    load_dev(&s_dev, (ba).devs + s_ent.x);                                \
    __syncthreads();

template <typename T> struct Vec4;
template <> struct Vec4<double> { using type = double4; };
template <> struct Vec4<float> { using type = float4; };

// Expensive-potential tables in the workspace (element type T).
// Warps per CTA of the expensive kernel (both element types) = atoms per CTA
// group (a warp per atom), and the CTAs per SM each kernel is compiled for.
// Two atoms a CTA spread a small expensive set evenly over the SMs (1396
// atoms: at most 10 a SM against 12 with groups of 4); the float kernel's
// ~36 KB of shared memory a CTA (Fe, n = 10, lmax = 4, 128 neighbour slots)
// leaves room for 6 CTAs, the float64 kernel's ~71 KB for 3.
// A single context's CTA may also hold 4 warps (ACE_MAX_WARPS): the two
// tile buffers are then shared by twice the atoms, which lets more warps fit an
// SM when the evaluated set is many waves large (the 256,000-atom cylinder:
// 3 CTAs of 4 warps against 5 of 2).  The batched kernel keeps groups of 2.
constexpr int ACE_GROUP = 2;
constexpr int ACE_MAX_WARPS = 4;
template <typename T>
__host__ __device__ constexpr int ace_warps() {
    return ACE_GROUP;
}
template <typename T>
__host__ __device__ constexpr int ace_min_ctas() {
    return sizeof(T) == 4 ? 6 : 2;
}
// the same register budget for CTAs of ACE_MAX_WARPS warps
template <typename T>
__host__ __device__ constexpr int ace_min_ctas_max() {
    return ace_min_ctas<T>() * ACE_GROUP / ACE_MAX_WARPS;
}
// The tensor-core readout (float, bf16 operands) takes groups of 4 atoms, a
// warp each: 4 x 16 rows (atom, m3) fill the M = 64 rows of one MMA tile, and
// three such CTAs fit an SM (8 atoms and M = 128 would need a CTA of 8 warps,
// one an SM).
constexpr int TC_ACE_WARPS = 4;
constexpr int TC_M = 16 * TC_ACE_WARPS;
constexpr int TC_MIN_CTAS = 3;

// One Gaunt coefficient with the packed m indices of its two other factors
// (ma | mb << 8, 0-based; the ordering by m3 also flags run ends, see
// AceTileHdr), loaded as one 8- or 16-byte word.
constexpr int GE_RUN_END = 1 << 24;   // last entry of a run of equal m1 in an m3 row

template <typename T>
struct __align__(sizeof(T) == 4 ? 8 : 16) GEnt {
    int pk;
    T g;
};

// Header of one l-triple tile of the nu = 3 tables.  A tile is one contiguous,
// 16-byte aligned block (a multiple of 16 bytes) holding, at these byte offsets:
//   W[q1 q2][q3]  (n*n rows of np, zero padded) right after the header,
//   the Gaunt entries GEnt<T> ordered by m2 (m1 | m3 << 8) at o_ge,
//   their offset rows (2 l2 + 2 ints: the first entry of each m2, then the
//     end; entry indices relative to o_ge) at o_go.
// The ordering by m3 (m1 | m2 << 8, m1 ascending within a row, GE_RUN_END on
// the last entry of each run of equal m1) is the same for every potential and
// sits in constant memory, from row cg on; float64 tiles also hold it, at
// o_ge3 with its 2 l3 + 2 offset rows at o_go3 (the float64 kernel reads it
// there: its entries are twice the size, and where few warps run a shared-
// memory read is the quicker).
// mode: 0 l's distinct, 1 l1 == l2, 2 l2 == l3, 3 all equal (W symmetrised over
// the matching n indices).  Tiles of the tensor-core readout (bf16 modes) also
// hold, at o_wb (128-byte aligned; 0 otherwise), W as the MMA's B operand: 16
// rows (q3, zero beyond n) by kp columns (q1 n + q2, zero beyond n^2) of bf16
// in the K-major core-matrix layout (tc.cuh, K stride TC_LBO_B), followed for
// the hi/lo split by the same layout of the remainders W - bf16(W).
struct AceTileHdr {
    int l1, l2, l3, mode;
    int o_ge, o_go, bytes, o_wb;
    int cg;             // first row of the triple in the constant-memory Gaunt table
    int o_ge3, o_go3;   // float64 tiles: their own ordering by m3 and its offset rows (0 in float tiles)
    int pad;            // 16-byte multiple: W follows
};

// The constant-memory Gaunt table of the expensive kernels (every l-triple
// l1 >= l2 >= l3 up to MIX_MAX_LMAX, ordered by m3; built on the host): entry
// and row capacities, and the magnitude below which a quadrature value is zero.
constexpr int GAUNT_ENT_CAP = 2048;
constexpr int GAUNT_ROW_CAP = 192;
constexpr double GAUNT_ZERO = 1e-12;

template <typename T>
struct AceTab {
    int n, L, nu, nlm, ntau;
    int np;             // n rounded up to a multiple of 4 (row length of padded tables)
    int qb;             // q2 block per lane in the nu = 3 U/Z pass (divides np)
    int tile_max;       // bytes of the largest nu = 3 tile
    double rc;
    const T* c1;        // [n]
    const T* S2;        // [L+1][n][n]  symmetric: W2 + W2^T, W2 upper-triangular c2
    const unsigned char* tiles;  // the ntau l-triple tiles, back to back
    const int* tile_off;         // [ntau + 1] byte offset of each tile, then the end
    const T* ylmk;      // [nlm] normalisation of Y_lm times sqrt2 for m != 0
    const T* pair;      // [16] pair-term B-spline coefficients
    int has_pair;
};

constexpr int SPL_W2 = 13;   // pair-term intervals on [0, rc]
constexpr int SPL_W3 = 5;    // three-body intervals along each argument

template <typename T>
struct SplTab {
    double rc, rc3;
    // coefficient windows, one aligned 4-vector each (the four control points
    // one cubic B-spline interval reads): c2w[q] = c2[q..q+3] for q < SPL_W2,
    // c3w[(a * 8 + b) * SPL_W3 + z] = c3[a][b][z..z+3] for z < SPL_W3
    const T* c2w;   // [SPL_W2][4]
    const T* c3w;   // [64][SPL_W3][4]
    // derived constants in T, formed on the host in float64 and rounded once
    // (no float64 division per atom on the device)
    T rc2, rc32;            // rc^2 (2-body), rc3^2
    T invh2, invh3, invhc;  // 13/rc, 5/rc3, 5/(2 rc3)
};

// ---------------------------------------------------------------------------
// bit-reproducible geometry: explicit round-to-nearest ops, no FMA contraction

__device__ __forceinline__ double mi_comp(double t, double L, double invL, int per) {
    if (per) t = __dsub_rn(t, __dmul_rn(L, rint(__dmul_rn(t, invL))));
    return t;
}

// d = x_j - x_i with the minimum image in periodic dimensions
__device__ __forceinline__ void delta_rn(const Box& b, const double4& xi, const double4& xj, double d[3]) {
    d[0] = mi_comp(__dsub_rn(xj.x, xi.x), b.L[0], b.invL[0], b.per[0]);
    d[1] = mi_comp(__dsub_rn(xj.y, xi.y), b.L[1], b.invL[1], b.per[1]);
    d[2] = mi_comp(__dsub_rn(xj.z, xi.z), b.L[2], b.invL[2], b.per[2]);
}

__device__ __forceinline__ double norm2_rn(const double d[3]) {
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__device__ __forceinline__ int cell_coord(const Box& b, const Cells& c, double x, int d) {
    double s = __dmul_rn(__dsub_rn(x, b.lo[d]), c.invh[d]);
    int q = (int)floor(s);
    q = q < 0 ? 0 : q;
    q = q > c.nc[d] - 1 ? c.nc[d] - 1 : q;
    return q;
}

__device__ __forceinline__ void set_status(int* st, int bits) { atomicOr(st + SW_STATUS, bits); }

// Warp-wide sum delivered to lane 0 as float64, lanes combined in a fixed
// order.  float64 inputs are summed in float64; float inputs are summed in
// float with a compensation term (Knuth's TwoSum at every step), so the float
// path keeps double-like accuracy for the sum without float64 arithmetic per
// lane (float64 runs at 1/62 of float on GB300).
// The sum and its compensation stay in T through the shuffles; only lane 0's
// result is meaningful, and callers convert it with lane0_double() inside a
// lane-0 branch, so no warp-wide float64 instruction is issued (float64 is the
// scarcest pipe on this part).
struct WSum {
    float s, c;
};
struct WSumD {
    double s;
};
__device__ __forceinline__ WSumD warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return {v};
}
__device__ __forceinline__ WSum warp_sum(float v) {
    float s = v, c = 0.f;
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, s, o);
        const float c2 = __shfl_down_sync(0xffffffffu, c, o);
        const float t = __fadd_rn(s, s2);
        const float bb = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(s2, bb));
        s = t;
        c = __fadd_rn(__fadd_rn(c, c2), e);
    }
    return {s, c};
}
// Compensated sum over the LPA lanes of a group (fixed order; lane 0 of the
// group holds the result).  For LPA = 32 this is warp_sum.
template <int LPA>
__device__ __forceinline__ WSum group_sum(float v, unsigned mask) {
    float s = v, c = 0.f;
#pragma unroll
    for (int o = LPA / 2; o > 0; o >>= 1) {
        const float s2 = __shfl_down_sync(mask, s, o, LPA);
        const float c2 = __shfl_down_sync(mask, c, o, LPA);
        const float t = __fadd_rn(s, s2);
        const float bb = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(s2, bb));
        s = t;
        c = __fadd_rn(__fadd_rn(c, c2), e);
    }
    return {s, c};
}
template <int LPA>
__device__ __forceinline__ WSumD group_sum(double v, unsigned mask) {
#pragma unroll
    for (int o = LPA / 2; o > 0; o >>= 1) v += __shfl_down_sync(mask, v, o, LPA);
    return {v};
}

__device__ __forceinline__ double lane0_double(WSumD w) { return w.s; }
__device__ __forceinline__ double lane0_double(WSum w) { return (double)w.s + (double)w.c; }

// Evaluation stamp in the w component of an incoming gradient row (the bits of
// the integer epoch; a row counts only when its stamp is the current epoch).
__device__ __forceinline__ float stamp_as(float, int e) { return __int_as_float(e); }
__device__ __forceinline__ double stamp_as(double, int e) { return __longlong_as_double((long long)e); }
__device__ __forceinline__ bool stamp_is(float w, int e) { return __float_as_int(w) == e; }
__device__ __forceinline__ bool stamp_is(double w, int e) { return __double_as_longlong(w) == (long long)e; }

// Pair vector for the potentials: the difference and minimum image in float64
// (positions are absolute coordinates of up to hundreds of Angstrom), then
// rounded once to T; length and direction in T.
template <typename T>
__device__ __forceinline__ void pair_vec(const Box& b, const double4& xi, const double4& xj, T v[3], T& r2) {
    const double dd[3] = {xj.x - xi.x, xj.y - xi.y, xj.z - xi.z};
    for (int k = 0; k < 3; ++k) {
        double t = dd[k];
        if (b.per[k]) t = fma(-b.L[k], rint(t * b.invL[k]), t);
        v[k] = (T)t;
    }
    r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
}

// Pair vectors of atom i in the kernel's arithmetic.  float64: pair_vec above.
// float: from cell-relative float positions, x_j - x_i = xr_j - xr_i + dc h with
// dc the cell offset (in {-1, 0, 1} per dimension for list neighbours, wrapped
// in periodic dimensions), so no float64 operation is spent per pair.
template <typename T>
struct PairFrame;

// lanes per atom of the kernels that walk one list row with a lane group (the
// gather, the buffer scan): the system's d.gat_lpa, a quarter warp for mean
// list lengths up to 40, half a warp up to 80, else a warp; 32 when unset
__host__ __device__ inline int gather_lpa(const Dev& d) { return d.gat_lpa == 8 || d.gat_lpa == 16 ? d.gat_lpa : 32; }

// Pt: what vec() reads of the partner atom, loadable ahead of its use; Geo:
// what it reads of the system's box and cells, loadable once into registers
template <>
struct PairFrame<double> {
    struct Pt {
        double4 x;
    };
    struct Geo {
        const Box* b;
    };
    double4 xi;
    __device__ __forceinline__ PairFrame(const Dev& d, int i) : xi(d.x[i]) {}
    static __device__ __forceinline__ Pt load(const Dev& d, int j) { return Pt{d.x[j]}; }
    static __device__ __forceinline__ Geo geo(const Dev& d) { return Geo{&d.box}; }
    __device__ __forceinline__ void vec(const Geo& g, const Pt& p, double v[3], double& r2) const {
        pair_vec<double>(*g.b, xi, p.x, v, r2);
    }
    __device__ __forceinline__ void vec(const Dev& d, const Pt& p, double v[3], double& r2) const {
        pair_vec<double>(d.box, xi, p.x, v, r2);
    }
    __device__ __forceinline__ void vec(const Dev& d, int j, double v[3], double& r2) const {
        vec(d, load(d, j), v, r2);
    }
};

template <>
struct PairFrame<float> {
    struct Pt {
        float4 x;
        int c;
    };
    float4 xri;
    int ci;
    __device__ __forceinline__ PairFrame(const Dev& d, int i) : xri(d.xr[i]), ci(d.cell3[i]) {}
    __device__ __forceinline__ PairFrame(float4 x, int c) : xri(x), ci(c) {}
    struct Geo {
        int per[3], nc[3];
        float hf[3];
    };
    static __device__ __forceinline__ Pt load(const Dev& d, int j) { return Pt{d.xr[j], d.cell3[j]}; }
    static __device__ __forceinline__ Geo geo(const Dev& d) {
        Geo g;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            g.per[k] = d.box.per[k];
            g.nc[k] = d.cells.nc[k];
            g.hf[k] = d.cells.hf[k];
        }
        return g;
    }
    __device__ __forceinline__ void vec(const Dev& d, int j, float v[3], float& r2) const {
        vec(d, load(d, j), v, r2);
    }
    __device__ __forceinline__ void vec(const Dev& d, const Pt& p, float v[3], float& r2) const {
        vec(geo(d), p, v, r2);
    }
    __device__ __forceinline__ void vec(const Geo& g, const Pt& p, float v[3], float& r2) const {
        const float4 xrj = p.x;
        const int cj = p.c;
        const float a[3] = {xrj.x - xri.x, xrj.y - xri.y, xrj.z - xri.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int dc = ((cj >> (10 * k)) & 1023) - ((ci >> (10 * k)) & 1023);
            if (g.per[k]) {
                if (dc > 1) dc -= g.nc[k];
                else if (dc < -1) dc += g.nc[k];
            }
            v[k] = a[k] + (float)dc * g.hf[k];
        }
        r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    }
};

// squared length of the float pair vector to atom j from the frame (xri, ci)
__device__ __forceinline__ float pair_r2_float(const Dev& d, float4 xri, int ci, int j) {
    float v[3], r2;
    PairFrame<float>(xri, ci).vec(d, j, v, r2);
    return r2;
}

}  // namespace mixd
