// Cell list and full neighbour list with a reverse-slot map (the region and
// force steps reuse one neighbour list, as the paper's region fix reuses the
// pair style's lists, Sec. 4.4), plus the first half of velocity Verlet and
// the skin test that decides when the lists are rebuilt.
//
// Bit-reproducibility: positions are folded, binned and compared with explicit
// round-to-nearest operations (no FMA), in the same order as a plain CPU
// evaluation: d = x_j - x_i; d -= L rint(d / L); r2 = dx*dx + dy*dy + dz*dz;
// neighbour iff r2 < (rc + skin)^2.  Each row of the list is sorted ascending.
#include <climits>

#include <mutex>

#include "mix_launch.h"

namespace mixd {

// v += h F; x += dt v (when integrating); then flag a rebuild if any atom moved
// more than skin/2 since the last build.  Atom 0's thread resets the
// per-evaluation counters.  (Bodies take the system d, this block's index bx
// among the gx blocks working on d, and stride over d's atoms.)
__device__ __forceinline__ void disp_body(const Dev& d, int bx, int gx, int integrate, double dt, double h,
                                          int force_rebuild) {
    const int64_t stride = (int64_t)gx * blockDim.x;
    for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x;; i += stride) {
        if (i == 0) {
            d.status[SW_NCORE] = 0;
            d.status[SW_NRAMP] = 0;
            d.status[SW_NLE] = 0;
            d.status[SW_NLC] = 0;
            d.status[SW_EPOCH] += 1;
            if (force_rebuild) d.status[SW_REBUILD] = 1;
        }
        if (i >= d.n) return;
        // every load first, so that one memory latency covers them all (the
        // arrays never overlap, which the compiler cannot know)
        double4 x = d.x[i];
        double4 v = make_double4(0.0, 0.0, 0.0, 0.0), f = v, xb = v;
        int c3 = 0;
        if (integrate) {
            v = d.v[i];
            f = d.f[i];
        }
        if (!force_rebuild) {
            xb = d.xb[i];
            if (d.xr) c3 = d.cell3[i];
        }
        if (integrate) {
            v.x = __dadd_rn(v.x, __dmul_rn(h, f.x));
            v.y = __dadd_rn(v.y, __dmul_rn(h, f.y));
            v.z = __dadd_rn(v.z, __dmul_rn(h, f.z));
            x.x = __dadd_rn(x.x, __dmul_rn(dt, v.x));
            x.y = __dadd_rn(x.y, __dmul_rn(dt, v.y));
            x.z = __dadd_rn(x.z, __dmul_rn(dt, v.z));
            d.v[i] = v;
            d.x[i] = x;
        }
        const bool finite = isfinite(x.x) && isfinite(x.y) && isfinite(x.z);
        if (!finite) {
            set_status(d.status, ST_NONFINITE);
            continue;
        }
        const double xs[3] = {x.x, x.y, x.z};
        for (int k = 0; k < 3; ++k)
            if (!d.box.per[k] && (xs[k] < d.box.lo[k] || xs[k] >= d.box.lo[k] + d.box.L[k]))
                set_status(d.status, ST_OUT_OF_BOX);
        if (!force_rebuild) {
            const double dx = x.x - xb.x, dy = x.y - xb.y, dz = x.z - xb.z;
            if (dx * dx + dy * dy + dz * dz > d.half_skin2) d.status[SW_REBUILD] = 1;
            // relative to the cell of the last build (recomputed by k_cell_bin on rebuilds)
            if (d.xr) d.xr[i] = cell_relative(d.box, d.cells, x, c3);
        }
    }
}

__global__ void k_disp(Dev d, int integrate, double dt, double h, int force_rebuild) {
    disp_body(d, blockIdx.x, gridDim.x, integrate, dt, h, force_rebuild);
}

// Fold periodic coordinates into [0, L), bin into cells, count per cell.
__device__ __forceinline__ void cell_bin_atom(const Dev& d, int64_t i) {
    double4 x = d.x[i];
    double xs[3] = {x.x, x.y, x.z};
    for (int k = 0; k < 3; ++k)
        if (d.box.per[k]) xs[k] = __dsub_rn(xs[k], __dmul_rn(d.box.L[k], floor(__dmul_rn(xs[k], d.box.invL[k]))));
    x.x = xs[0];
    x.y = xs[1];
    x.z = xs[2];
    d.x[i] = x;
    d.xf[i] = make_float4((float)xs[0], (float)xs[1], (float)xs[2], 0.f);
    const int cx = cell_coord(d.box, d.cells, xs[0], 0);
    const int cy = cell_coord(d.box, d.cells, xs[1], 1);
    const int cz = cell_coord(d.box, d.cells, xs[2], 2);
    const int c = (cz * d.cells.nc[1] + cy) * d.cells.nc[0] + cx;
    d.cell_of[i] = c;
    const int c3 = cx | (cy << 10) | (cz << 20);
    d.cell3[i] = c3;
    d.xr[i] = cell_relative(d.box, d.cells, x, c3);
    atomicAdd(d.cell_count + c, 1);
}

__device__ __forceinline__ void cell_bin_body(const Dev& d, int bx, int gx) {
    if (d.status[SW_REBUILD] == 0) return;
    for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x; i < d.n; i += (int64_t)gx * blockDim.x)
        cell_bin_atom(d, i);
}
__global__ void k_cell_bin(Dev d) { cell_bin_body(d, blockIdx.x, gridDim.x); }

// Exclusive scan of the cell counts (one block), zeroing counts and fill slots.
__device__ __forceinline__ void cell_scan_body(const Dev& d) {
    if (d.status[SW_REBUILD] == 0) return;
    __shared__ int wsum[32];
    __shared__ int carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) {
        carry_s = 0;
        d.status[SW_MAXNB] = 0;
    }
    __syncthreads();
    const int nc = d.cells.ncell;
    for (int base = 0; base < nc; base += blockDim.x) {
        const int k = base + tid;
        const int v = k < nc ? d.cell_count[k] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nw ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            if (lane < nw) wsum[lane] = w;
        }
        __syncthreads();
        const int carry = carry_s;
        const int excl = carry + (warp > 0 ? wsum[warp - 1] : 0) + incl - v;
        if (k < nc) {
            d.cell_start[k] = excl;
            d.cell_fill[k] = 0;
            d.cell_count[k] = 0;
        }
        __syncthreads();
        if (tid == blockDim.x - 1) carry_s = excl + v;
        __syncthreads();
    }
    if (tid == 0) d.cell_start[nc] = carry_s;
}
__global__ void k_cell_scan(Dev d) { cell_scan_body(d); }

__device__ __forceinline__ void cell_fill_body(const Dev& d, int bx, int gx) {
    if (d.status[SW_REBUILD] == 0) return;
    for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x; i < d.n; i += (int64_t)gx * blockDim.x) {
        const int c = d.cell_of[i];
        const int slot = d.cell_start[c] + atomicAdd(d.cell_fill + c, 1);
        d.cell_atoms[slot] = (int)i;
    }
}
__global__ void k_cell_fill(Dev d) { cell_fill_body(d, blockIdx.x, gridDim.x); }

constexpr int NB_WARPS = 4;

// One warp per atom: the 27-cell stencil is up to 18 contiguous runs of cells
// (9 rows (dz, dy), one or two runs along x each); lane r < 18 finds run r, a
// warp prefix sum numbers all candidates of all runs, and the lanes take 32
// consecutive candidates at a time across run boundaries (in run order, so the
// compacted row is the same as a run-by-run scan) with the next 32 loaded
// ahead.  Candidates with r2 < rlist2 are compacted into shared memory with a
// ballot; each lane then ranks its entries among the row (atom indices are
// distinct) and writes them to their sorted places.
__device__ __forceinline__ int pow2_cap(int cap) {
    int c = 32;
    while (c < cap) c <<= 1;
    return c;
}

constexpr int NB_RUNS = 18;

// The candidate test of the list build: a float pre-filter (the float distance
// is within 2e-5 relative of the float64 one for boxes up to a few thousand
// Angstrom, so only candidates inside a +-2e-4 band around the threshold take
// the exact float64 test, r^2 formed as in the oracle).
struct NbTest {
    float lo2, hi2;
    float Lf[3], iLf[3];
    __device__ __forceinline__ explicit NbTest(const Dev& d) {
        lo2 = (float)(d.rlist2 * (1.0 - 2e-4));
        hi2 = (float)(d.rlist2 * (1.0 + 2e-4));
        for (int k = 0; k < 3; ++k) {
            Lf[k] = (float)d.box.L[k];
            iLf[k] = (float)d.box.invL[k];
        }
    }
    __device__ __forceinline__ bool accept(const Dev& d, const double4& xi, const float4& xif, const float4& xjf,
                                           int j) const {
        float df[3] = {xjf.x - xif.x, xjf.y - xif.y, xjf.z - xif.z};
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (d.box.per[k]) df[k] -= Lf[k] * rintf(df[k] * iLf[k]);
        const float r2f = df[0] * df[0] + df[1] * df[1] + df[2] * df[2];
        if (r2f < lo2 && !d.exact_lists) return true;
        if (r2f <= hi2 || d.exact_lists) {
            double dd[3];
            delta_rn(d.box, xi, d.x[j], dd);
            return norm2_rn(dd) < d.rlist2;
        }
        return false;
    }
};

// The runs of the 27-cell stencil of cell (cx, cy, cz): lane r < NB_RUNS gets
// run r's first cell_atoms index t0 and length len (0 for an absent run):
// rows (dz, dy) of three cells along x, one or two runs each.
__device__ __forceinline__ void nb_run(const Dev& d, int cx, int cy, int cz, int lane, int& t0, int& len) {
    const int ncx = d.cells.nc[0], ncy = d.cells.nc[1], ncz = d.cells.nc[2];
    t0 = 0;
    len = 0;
    if (lane >= NB_RUNS) return;
    const int rr = lane >> 1, run = lane & 1;
    int qz = cz + rr / 3 - 1, qy = cy + rr % 3 - 1;
    bool in = true;
    if (d.box.per[2]) qz = (qz + ncz) % ncz;
    else in = qz >= 0 && qz < ncz;
    if (d.box.per[1]) qy = (qy + ncy) % ncy;
    else in = in && qy >= 0 && qy < ncy;
    // runs of cells along x: [a0, b0] and optionally [a1, b1]
    int a0, b0, a1 = 1, b1 = 0;
    if (d.box.per[0]) {
        if (cx == 0) { a0 = 0; b0 = 1; a1 = ncx - 1; b1 = ncx - 1; }
        else if (cx == ncx - 1) { a0 = ncx - 2; b0 = ncx - 1; a1 = 0; b1 = 0; }
        else { a0 = cx - 1; b0 = cx + 1; }
    } else {
        a0 = cx > 0 ? cx - 1 : 0;
        b0 = cx < ncx - 1 ? cx + 1 : ncx - 1;
    }
    const int ra = run == 0 ? a0 : a1, rb = run == 0 ? b0 : b1;
    if (in && ra <= rb) {
        const int row = (qz * ncy + qy) * ncx;
        t0 = d.cell_start[row + ra];
        len = d.cell_start[row + rb + 1] - t0;
    }
}

// The row of atom i from its cnt accepted candidates in buf (this warp's
// capp2 ints): capacity check, then each lane ranks its entries among the row
// (atom indices are distinct) and stores them at their sorted places.
__device__ __forceinline__ void nb_write_row(const Dev& d, int64_t i, const double4& xi, int cnt, int* buf, int lane) {
    const int cap = d.cap;
    if (lane == 0) {
        atomicMax(d.status + SW_MAXNB, cnt);
        if (cnt > cap) set_status(d.status, ST_NBR_OVERFLOW);
    }
    const int mlen = cnt < cap ? cnt : cap;
    // pad to whole 4-vectors with INT_MAX (ranks unaffected): m4 <= capp2
    const int m4 = (mlen + 3) & ~3;
    if (mlen + lane < m4) buf[mlen + lane] = INT_MAX;
    __syncwarp();
    int* row = d.nbr + i * (int64_t)cap;
    const int4* b4 = reinterpret_cast<const int4*>(buf);
    for (int p = lane; p < mlen; p += 32) {
        const int v = buf[p];
        int rank = 0;
        for (int q = 0; q < (m4 >> 2); ++q) {
            const int4 w = b4[q];
            rank += (w.x < v) + (w.y < v) + (w.z < v) + (w.w < v);
        }
        row[rank] = v;
    }
    if (lane == 0) {
        d.nnb[i] = mlen;
        d.xb[i] = xi;
    }
    __syncwarp();
}

// AHEAD2: also load the float positions a pass ahead (the batched kernel; the
// single-context one, on longer candidate runs, measured faster without)
template <bool AHEAD2>
__device__ __forceinline__ void neigh_build_body(const Dev& d, int bx, int gx, int capp2, int* sbuf) {
    if (d.status[SW_REBUILD] == 0) return;
    __shared__ int s_runx[NB_WARPS][NB_RUNS];   // cell_atoms index of a run's first candidate, less its number
    __shared__ int s_runi[NB_WARPS][NB_RUNS];   // candidates in runs 0..r
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* buf = sbuf + warp * capp2;
    int* runx = s_runx[warp];
    int* runi = s_runi[warp];
    const unsigned lt = (1u << lane) - 1u;
    const int ncx = d.cells.nc[0], ncy = d.cells.nc[1];
    const NbTest test(d);
    for (int64_t i = (int64_t)bx * NB_WARPS + warp; i < d.n; i += (int64_t)gx * NB_WARPS) {
        const double4 xi = d.x[i];
        const float4 xif = d.xf[i];
        const int c = d.cell_of[i];
        const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
        int len, t0;
        nb_run(d, cx, cy, cz, lane, t0, len);
        int inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const int total = __shfl_sync(0xffffffffu, inc, 31);
        if (lane < NB_RUNS) {
            runi[lane] = inc;
            runx[lane] = t0 - (inc - len);
        }
        __syncwarp();
        // AHEAD2: the atom two passes ahead and the position one pass ahead are
        // loaded before this pass is tested; else the atom one pass ahead
        // (r: run of the furthest candidate loaded)
        int r = 0;
        int jn = -1, jnn = -1;
        float4 xn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < total) {
            while (lane >= runi[r]) ++r;
            jn = d.cell_atoms[runx[r] + lane];
            if (AHEAD2) xn = d.xf[jn];
        }
        if (AHEAD2 && lane + 32 < total) {
            while (lane + 32 >= runi[r]) ++r;
            jnn = d.cell_atoms[runx[r] + lane + 32];
        }
        int cnt = 0;
        for (int u = lane; u - lane < total; u += 32) {
            const int j = jn;
            float4 xjf;
            if (AHEAD2) {
                xjf = xn;
                jn = jnn;
                if (u + 32 < total) xn = d.xf[jnn];
                if (u + 64 < total) {
                    while (u + 64 >= runi[r]) ++r;
                    jnn = d.cell_atoms[runx[r] + u + 64];
                }
            } else if (u + 32 < total) {
                while (u + 32 >= runi[r]) ++r;
                jn = d.cell_atoms[runx[r] + u + 32];
            }
            bool ok = false;
            if (u < total && j != (int)i) {
                if (!AHEAD2) xjf = d.xf[j];
                ok = test.accept(d, xi, xif, xjf, j);
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const int p = cnt + __popc(m & lt);
                if (p < capp2) buf[p] = j;
            }
            cnt += __popc(m);
        }
        nb_write_row(d, i, xi, cnt, buf, lane);
    }
}

__global__ void __launch_bounds__(NB_WARPS * 32) k_neigh_build(Dev d, int capp2) {
    extern __shared__ __align__(16) int sbuf[];
    neigh_build_body<false>(d, blockIdx.x, gridDim.x, capp2, sbuf);
}

// The list build of a single context with neighbour-cell tiles staged in shared
// memory: a CTA takes a cell at a time, copies the candidates of its 27-cell
// stencil (atom index and float position, in run order) into shared memory
// once, and its warps take the cell's atoms, a warp per atom, testing 32
// staged candidates at a time; the candidates cross L2 once per cell instead
// of once per atom.  A stencil with more than NB_TILE candidates (a dense
// spot) is tested from global memory instead.  The same test and row writing
// as the batched build (neigh_build_body), so the rows are the same.
constexpr int NB_TILE = 1024;

inline size_t nb_tiled_smem(int capp2) {
    return (size_t)NB_TILE * (sizeof(float4) + sizeof(int)) + (size_t)NB_WARPS * capp2 * sizeof(int);
}

__global__ void __launch_bounds__(NB_WARPS * 32) k_neigh_build_tiled(Dev d, int capp2) {
    if (d.status[SW_REBUILD] == 0) return;
    extern __shared__ __align__(16) unsigned char nb_smem[];
    float4* tpos = reinterpret_cast<float4*>(nb_smem);
    int* tidx = reinterpret_cast<int*>(tpos + NB_TILE);
    int* sbuf = tidx + NB_TILE;
    __shared__ int s_runx[NB_RUNS], s_runi[NB_RUNS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* buf = sbuf + warp * capp2;
    const unsigned lt = (1u << lane) - 1u;
    const int ncx = d.cells.nc[0], ncy = d.cells.nc[1];
    const int ncell = d.cells.ncell;
    const NbTest test(d);
    for (int c = blockIdx.x; c < ncell; c += gridDim.x) {
        const int a0 = d.cell_start[c], a1 = d.cell_start[c + 1];
        if (a0 == a1) continue;   // the same for the whole CTA
        const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
        if (warp == 0) {
            int t0, len;
            nb_run(d, cx, cy, cz, lane, t0, len);
            int inc = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            if (lane < NB_RUNS) {
                s_runi[lane] = inc;
                s_runx[lane] = t0 - (inc - len);
            }
        }
        __syncthreads();
        const int total = s_runi[NB_RUNS - 1];
        const bool staged = total <= NB_TILE;
        if (staged) {
            for (int t = threadIdx.x; t < total; t += blockDim.x) {
                int r = 0;
                while (t >= s_runi[r]) ++r;
                const int j = d.cell_atoms[s_runx[r] + t];
                tidx[t] = j;
                tpos[t] = d.xf[j];
            }
        }
        __syncthreads();
        for (int a = a0 + warp; a < a1; a += NB_WARPS) {
            const int i = d.cell_atoms[a];
            const double4 xi = d.x[i];
            const float4 xif = d.xf[i];
            int cnt = 0;
            int r = 0;
            for (int u = lane; u - lane < total; u += 32) {
                bool ok = false;
                int j = -1;
                if (u < total) {
                    float4 xjf;
                    if (staged) {
                        j = tidx[u];
                        xjf = tpos[u];
                    } else {
                        while (u >= s_runi[r]) ++r;
                        j = d.cell_atoms[s_runx[r] + u];
                        xjf = d.xf[j];
                    }
                    if (j != i) ok = test.accept(d, xi, xif, xjf, j);
                }
                const unsigned m = __ballot_sync(0xffffffffu, ok);
                if (ok) {
                    const int p = cnt + __popc(m & lt);
                    if (p < capp2) buf[p] = j;
                }
                cnt += __popc(m);
            }
            nb_write_row(d, i, xi, cnt, buf, lane);
        }
        __syncthreads();   // the tile and the runs are rewritten for the next cell
    }
}

// rev[i][s] = position of i in the row of j = nbr[i][s] (binary search in the
// sorted row).  A warp per atom, lanes over its row's slots.
__device__ __forceinline__ void neigh_rev_body(const Dev& d, int bx, int gx) {
    if (d.status[SW_REBUILD] == 0) return;
    const int lane = threadIdx.x & 31, wpb = (int)(blockDim.x >> 5);
    const int cap = d.cap;
    for (int64_t i = (int64_t)bx * wpb + (threadIdx.x >> 5); i < d.n; i += (int64_t)gx * wpb) {
        const int m = d.nnb[i];
        const int* ri = d.nbr + i * cap;
        for (int s = lane; s < m; s += 32) {
            const int j = ri[s];
            const int* row = d.nbr + (int64_t)j * cap;
            int lo = 0, hi = d.nnb[j] - 1, pos = -1;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int v = row[mid];
                if (v == (int)i) {
                    pos = mid;
                    break;
                }
                if (v < (int)i) lo = mid + 1;
                else hi = mid - 1;
            }
            if (pos < 0) {
                set_status(d.status, ST_REV_MISSING);
                pos = 0;
            }
            d.rev[i * cap + s] = pos;
        }
    }
}

__global__ void k_neigh_rev(Dev d) { neigh_rev_body(d, blockIdx.x, gridDim.x); }

// ---------------------------------------------------------------------------
// multi-system versions (one launch for all systems of a batch)

__global__ void kb_disp(BatchArgs ba, int integrate, double dt, int force_rebuild) {
    MIX_BATCH_BLOCK(ba)
    disp_body(s_dev, s_ent.y, s_ent.z, integrate, dt, half_kick(dt, s_dev.mass), force_rebuild);
}
__global__ void kb_cell_bin(BatchArgs ba) {
    MIX_BATCH_BLOCK_REBUILD(ba)
    cell_bin_body(s_dev, s_ent.y, s_ent.z);
}
__global__ void kb_cell_scan(BatchArgs ba) {
    MIX_BATCH_BLOCK_REBUILD(ba)
    cell_scan_body(s_dev);
}
__global__ void kb_cell_fill(BatchArgs ba) {
    MIX_BATCH_BLOCK_REBUILD(ba)
    cell_fill_body(s_dev, s_ent.y, s_ent.z);
}
__global__ void __launch_bounds__(NB_WARPS * 32) kb_neigh_build(BatchArgs ba) {
    extern __shared__ __align__(16) int sbuf[];
    MIX_BATCH_BLOCK_REBUILD(ba)
    neigh_build_body<true>(s_dev, s_ent.y, s_ent.z, pow2_cap(s_dev.cap), sbuf);
}
__global__ void kb_neigh_rev(BatchArgs ba) {
    MIX_BATCH_BLOCK_REBUILD(ba)
    neigh_rev_body(s_dev, s_ent.y, s_ent.z);
}

static int g_sms = 0;

int sm_count() {
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

cudaError_t raise_smem_limit(const void* func, size_t bytes) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_disp(const Dev& d, cudaStream_t s, int integrate, double dt, double h, int force_rebuild) {
    const int nb = (int)((d.n + 255) / 256);
    k_disp<<<nb > 0 ? nb : 1, 256, 0, s>>>(d, integrate, dt, h, force_rebuild);
}

void launch_build(const Dev& d, cudaStream_t s) {
    const int nb = (int)((d.n + 255) / 256);
    k_cell_bin<<<nb > 0 ? nb : 1, 256, 0, s>>>(d);
    k_cell_scan<<<1, 1024, 0, s>>>(d);
    k_cell_fill<<<nb > 0 ? nb : 1, 256, 0, s>>>(d);
    int capp2 = 32;
    while (capp2 < d.cap) capp2 <<= 1;
    // Cells to spare (at least 8 an SM, e.g. 24,000 for the 256,000-atom
    // cylinder): a CTA a cell with the stencil's candidates staged in shared
    // memory (C3's full build 631 -> 477 us).  Few cells (324 for the 8,001-atom
    // dumbbell): a warp per atom over every SM instead (32 against 58 us there).
    if (d.cells.ncell >= 8 * sm_count()) {
        const int64_t want = d.cells.ncell;
        const int64_t lim = d.grid_build > 0 ? d.grid_build : (int64_t)sm_count() * 8;
        const int grid = (int)(want < lim ? want : lim);
        k_neigh_build_tiled<<<grid > 0 ? grid : 1, NB_WARPS * 32, nb_tiled_smem(capp2), s>>>(d, capp2);
    } else {
        const int64_t want = (d.n + NB_WARPS - 1) / NB_WARPS;
        const int64_t lim = d.grid_build > 0 ? d.grid_build : (int64_t)sm_count() * 16;
        const int grid = (int)(want < lim ? want : lim);
        k_neigh_build<<<grid > 0 ? grid : 1, NB_WARPS * 32, NB_WARPS * capp2 * sizeof(int), s>>>(d, capp2);
    }
    // a warp per atom, striding; the grid is bounded (two waves of 8 CTAs an
    // SM) so that the steps without a rebuild, where every CTA exits at once,
    // launch few of them
    const int64_t want_r = (d.n + 7) / 8, lim_r = (int64_t)sm_count() * 16;
    const int nr = (int)(want_r < lim_r ? want_r : lim_r);
    k_neigh_rev<<<nr > 0 ? nr : 1, 256, 0, s>>>(d);
}

void launch_disp_batch(const BatchPlan& p, cudaStream_t s, int integrate, double dt, int force_rebuild) {
    kb_disp<<<p.nblk[BT_ATOM], 256, 0, s>>>(p.ba[BT_ATOM], integrate, dt, force_rebuild);
}

void launch_build_batch(const BatchPlan& p, cudaStream_t s) {
    kb_cell_bin<<<p.nblk[BT_ATOM], 256, 0, s>>>(p.ba[BT_ATOM]);
    kb_cell_scan<<<p.nblk[BT_ONE], 1024, 0, s>>>(p.ba[BT_ONE]);
    kb_cell_fill<<<p.nblk[BT_ATOM], 256, 0, s>>>(p.ba[BT_ATOM]);
    kb_neigh_build<<<p.nblk[BT_NB], NB_WARPS * 32, NB_WARPS * p.capp2 * sizeof(int), s>>>(p.ba[BT_NB]);
    kb_neigh_rev<<<p.nblk[BT_REV], 256, 0, s>>>(p.ba[BT_REV]);
}

}  // namespace mixd
