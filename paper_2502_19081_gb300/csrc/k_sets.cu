// Blend weights, evaluated sets and their compaction into ascending index lists.
//
// lambda (Sec. 4.4, Alg. 2 in its geometric reading): distance d from each
// region (sphere: centre; cylinder: axis line; minimum image in periodic
// dimensions), lambda = 1 for d < r_core, 1 - (d - r_core)/ramp for
// d < r_core + ramp, else 0, maximum over regions.  Sets (Sec. 4.5, buffer-set
// equation; Alg. 3): Lambda_exp = {lambda > 0}, Lambda_cheap = {lambda < 1};
// each is evaluated together with its buffer, the atoms outside it that have a
// member closer than the buffer radius (strict).  All comparisons use explicit
// round-to-nearest arithmetic so that the sets are bit-reproducible.
#include "mix_launch.h"

namespace mixd {

__device__ __forceinline__ void lambda_atom(const Dev& d, const Regions& r, int64_t i);

__device__ __forceinline__ void lambda_body(const Dev& d, const Regions& r, int bx, int gx) {
    for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x;; i += (int64_t)gx * blockDim.x) {
        if (i == 0 && d.status[SW_REBUILD]) {
            d.status[SW_REBUILDS] += 1;
            d.status[SW_REBUILD] = 0;
        }
        if (i >= d.n) return;
        lambda_atom(d, r, i);
    }
}

__global__ void k_lambda(Dev d, Regions r) { lambda_body(d, r, blockIdx.x, gridDim.x); }

__device__ __forceinline__ void lambda_atom(const Dev& d, const Regions& r, int64_t i) {
    double4 x = make_double4(0.0, 0.0, 0.0, 0.0);   // read once some region is not screened out
    bool have_x = false;
    double best = 0.0;
    // buffer-scan hints from the exact distances (triangle inequality, 1e-9 A
    // margin): with every region farther than r_core + ramp + r_buffer_exp no
    // neighbour closer than r_buffer_exp has lambda > 0 (bit 4); deeper than
    // r_buffer_cheap inside some core no neighbour that close has lambda < 1 (bit 5)
    bool far_e = true, deep_c = false;
    float4 xs = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r.screen) xs = d.xf[i];
    for (int k = 0; k < r.n; ++k) {
        const double* R = r.r[k];
        if (r.screen) {
            // float screen: clearly beyond the ramp and the expensive buffer of
            // this region, which then contributes nothing (see Regions)
            float v[3] = {xs.x - r.cf[k][0], xs.y - r.cf[k][1], xs.z - r.cf[k][2]};
            for (int t = 0; t < 3; ++t)
                if (d.box.per[t]) v[t] -= r.Lf[t] * rintf(v[t] * r.iLf[t]);
            float d2f = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            if ((int)R[0] == MIX_REGION_CYLINDER) {
                const float tt = v[0] * r.cf[k][3] + v[1] * r.cf[k][4] + v[2] * r.cf[k][5];
                d2f -= tt * tt;
            }
            if (d2f > r.far2[k]) continue;
        }
        if (!have_x) {
            x = d.x[i];
            have_x = true;
        }
        const double4 c = make_double4(R[1], R[2], R[3], 0.0);
        double v[3];
        delta_rn(d.box, c, x, v);
        double d2 = norm2_rn(v);
        if ((int)R[0] == MIX_REGION_CYLINDER) {
            const double t = __dadd_rn(__dadd_rn(__dmul_rn(v[0], R[4]), __dmul_rn(v[1], R[5])), __dmul_rn(v[2], R[6]));
            d2 = __dsub_rn(d2, __dmul_rn(t, t));
            if (d2 < 0.0) d2 = 0.0;
        }
        const double dist = __dsqrt_rn(d2);
        const double rc = R[7], ramp = R[8];
        if (!(dist >= rc + ramp + d.bufe + 1e-9)) far_e = false;
        if (dist + d.bufc + 1e-9 <= rc) deep_c = true;
        double lr;
        if (dist < rc) lr = 1.0;
        else if (ramp > 0.0 && dist < __dadd_rn(rc, ramp)) lr = __dsub_rn(1.0, __ddiv_rn(__dsub_rn(dist, rc), ramp));
        else lr = 0.0;
        if (lr > best) best = lr;
    }
    d.lam[i] = best;
    double w = best;
    if (r.blend == MIX_BLEND_CUBIC) w = __dmul_rn(__dmul_rn(best, best), __dsub_rn(3.0, __dmul_rn(2.0, best)));
    d.wgt[i] = w;
    d.flags[i] = (uint8_t)((best > 0.0 ? 1 : 0) | (best < 1.0 ? 2 : 0) | (far_e ? 16 : 0) | (deep_c ? 32 : 0));
    d.esite_e[i] = 0.0;
    d.esite_c[i] = 0.0;
}

// --- weights from seed atoms (Alg. 1-2), in gather form: each atom looks at its
// own neighbours, which yields the same sets of candidates as the scatter loops
// of the algorithms, so the results (flags and maxima) are identical.

constexpr int SEED_WARPS = 8;

// Coordination: neighbours closer than r_coord.  The first evaluation after the
// rule is set seeds from its own counts; after that the counts are summed over
// `period` evaluations and the seeds refreshed from their mean at the end of
// each period (the sums then restart).
__global__ void __launch_bounds__(SEED_WARPS * 32) k_coord(Dev d, SeedRule sr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int evals = d.status[SW_EVALS];
    const bool refresh = evals % sr.period == 0;
    const double navg = evals == 0 ? 1.0 : (double)sr.period;
    for (int64_t i = (int64_t)blockIdx.x * SEED_WARPS + warp; i < d.n; i += (int64_t)gridDim.x * SEED_WARPS) {
        const double4 xi = d.x[i];
        const int m = d.nnb[i];
        const int* row = d.nbr + i * (int64_t)d.cap;
        int cnt = 0;
        for (int s = lane; s < m; s += 32) {
            double dd[3];
            delta_rn(d.box, xi, d.x[row[s]], dd);
            cnt += norm2_rn(dd) < sr.rz2 ? 1 : 0;
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        if (lane == 0) {
            const int z = d.zsum[i] + cnt;
            if (refresh) {
                const double avg = (double)z / navg;
                const bool s = avg >= sr.zlo && avg <= sr.zhi;
                d.seed[i] = s ? 1 : 0;
                d.zsum[i] = 0;
            } else {
                d.zsum[i] = z;
            }
        }
    }
}

// Alg. 1: core = seeds and atoms closer than r_core to a seed.
__global__ void __launch_bounds__(SEED_WARPS * 32) k_core(Dev d, SeedRule sr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d.status[SW_EVALS] += 1;
        d.status[SW_NSEED] = 0;
    }
    for (int64_t j = (int64_t)blockIdx.x * SEED_WARPS + warp; j < d.n; j += (int64_t)gridDim.x * SEED_WARPS) {
        bool c = d.seed[j] != 0;
        if (!c) {
            const double4 xj = d.x[j];
            const int m = d.nnb[j];
            const int* row = d.nbr + j * (int64_t)d.cap;
            for (int s = lane; s < m; s += 32) {
                const int i = row[s];
                if (d.seed[i]) {
                    double dd[3];
                    delta_rn(d.box, xj, d.x[i], dd);
                    c = c || norm2_rn(dd) < sr.rcore2;
                }
            }
            c = __any_sync(0xffffffffu, c);
        }
        if (lane == 0) d.core[j] = c ? 1 : 0;
    }
}

// Alg. 2: weight 1 on core atoms, else the largest 1 - r/r_blend over core
// neighbours closer than r_blend (0 without one).
__global__ void __launch_bounds__(SEED_WARPS * 32) k_blend(Dev d, SeedRule sr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0 && d.status[SW_REBUILD]) {
        d.status[SW_REBUILDS] += 1;
        d.status[SW_REBUILD] = 0;
    }
    for (int64_t j = (int64_t)blockIdx.x * SEED_WARPS + warp; j < d.n; j += (int64_t)gridDim.x * SEED_WARPS) {
        double best = 0.0;
        if (d.core[j]) {
            best = 1.0;
        } else {
            const double4 xj = d.x[j];
            const int m = d.nnb[j];
            const int* row = d.nbr + j * (int64_t)d.cap;
            for (int s = lane; s < m; s += 32) {
                const int i = row[s];
                if (d.core[i]) {
                    double dd[3];
                    delta_rn(d.box, xj, d.x[i], dd);
                    const double r2 = norm2_rn(dd);
                    if (r2 < sr.rblend2) {
                        const double v = __dsub_rn(1.0, __ddiv_rn(__dsqrt_rn(r2), sr.rblend));
                        best = v > best ? v : best;
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double t = __shfl_down_sync(0xffffffffu, best, o);
                best = t > best ? t : best;
            }
        }
        if (lane == 0) {
            d.lam[j] = best;
            double w = best;
            if (sr.blend == MIX_BLEND_CUBIC) w = __dmul_rn(__dmul_rn(best, best), __dsub_rn(3.0, __dmul_rn(2.0, best)));
            d.wgt[j] = w;
            d.flags[j] = (uint8_t)((best > 0.0 ? 1 : 0) | (best < 1.0 ? 2 : 0));
            d.esite_e[j] = 0.0;
            d.esite_c[j] = 0.0;
            if (d.seed[j]) atomicAdd(d.status + SW_NSEED, 1);
        }
    }
}

constexpr int BUF_WARPS = 8;

// Buffer membership through the neighbour list.  A warp takes apw <= 32
// consecutive atoms: each lane tests its atom's flags (and the hints k_lambda
// left), then groups of LPA lanes scan the lists of the atoms that need it,
// 32 / LPA atoms at a time (the flags are ORs over a row, so the result does
// not depend on LPA).  In a large system most atoms need no scan and then cost
// a lane rather than a warp (apw = 32); a small one keeps a warp per atom (apw
// = 1, LPA = 32) so that its few scans run side by side.
template <int LPA>
__device__ __forceinline__ void buffer_body(const Dev& d, int bx, int gx, int apw) {
    constexpr int G = 32 / LPA;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / LPA, sub = lane & (LPA - 1);
    const unsigned gmask = LPA == 32 ? 0xffffffffu : (((1u << LPA) - 1u) << (grp * LPA));
    // float screen from the cell-relative float positions the potentials use;
    // float64 only within 1e-3 A^2 of a buffer radius
    const bool screen = d.xr != nullptr && !d.exact_lists;
    for (int64_t base = ((int64_t)bx * BUF_WARPS + warp) * apw; base < d.n;
         base += (int64_t)gx * BUF_WARPS * apw) {
        const int64_t im = base + lane;
        const bool valid = lane < apw && im < d.n;
        const int fl = valid ? (int)d.flags[im] : 0;
        const int f = fl & 3;
        // scan unless k_lambda's hints (bits 4, 5; geometric regions only) rule it out
        const bool my_ne = valid && !(f & 1) && !(fl & 16), my_nc = valid && !(f & 2) && !(fl & 32);
        unsigned todo = __ballot_sync(0xffffffffu, my_ne || my_nc);
        bool my_he = false, my_hc = false;
        while (todo) {
            // group g takes the (g + 1)-th atom still to scan
            unsigned t = todo;
            for (int k = 0; k < grp; ++k) t &= t - 1;
            const int src = t ? __ffs(t) - 1 : -1;
#pragma unroll
            for (int k = 0; k < G; ++k) todo &= todo - 1;
            const int sl = src < 0 ? 0 : src;
            const bool need_e = __shfl_sync(0xffffffffu, my_ne, sl) && src >= 0;
            const bool need_c = __shfl_sync(0xffffffffu, my_nc, sl) && src >= 0;
            bool he = false, hc = false;
            if (src >= 0) {
                const int64_t i = base + src;
                const int m = d.nnb[i];
                const int* row = d.nbr + i * (int64_t)d.cap;
                float4 xri = make_float4(0.f, 0.f, 0.f, 0.f);
                int ci = 0;
                if (screen) {
                    xri = d.xr[i];
                    ci = d.cell3[i];
                }
                for (int s = sub; s < m; s += LPA) {
                    const int j = row[s];
                    const int fj = d.flags[j] & 3;
                    const bool cand_e = need_e && (fj & 1), cand_c = need_c && (fj & 2);
                    if (cand_e || cand_c) {
                        bool ie = false, ic = false, exact = !screen;
                        if (screen) {
                            const float r2f = pair_r2_float(d, xri, ci, j);
                            if (cand_e) {
                                if (r2f < d.bufe2_lo) ie = true;
                                else if (r2f <= d.bufe2_hi) exact = true;
                            }
                            if (cand_c) {
                                if (r2f < d.bufc2_lo) ic = true;
                                else if (r2f <= d.bufc2_hi) exact = true;
                            }
                        }
                        if (exact) {
                            double dd[3];
                            delta_rn(d.box, d.x[i], d.x[j], dd);
                            const double r2 = norm2_rn(dd);
                            ie = cand_e && r2 < d.bufe2;
                            ic = cand_c && r2 < d.bufc2;
                        }
                        he = he || ie;
                        hc = hc || ic;
                    }
                }
            }
            he = (__ballot_sync(0xffffffffu, he) & gmask) != 0;
            hc = (__ballot_sync(0xffffffffu, hc) & gmask) != 0;
            // hand each group's result to its atom's lane
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int sg = __shfl_sync(0xffffffffu, src, g * LPA);
                const bool eg = __shfl_sync(0xffffffffu, he, g * LPA);
                const bool cg = __shfl_sync(0xffffffffu, hc, g * LPA);
                if (lane == sg) {
                    my_he = eg;
                    my_hc = cg;
                }
            }
        }
        if (valid) {
            const int ae = (f & 1) || my_he ? 4 : 0;
            const int ac = (f & 2) || my_hc ? 8 : 0;
            d.flags[im] = (uint8_t)(f | ae | ac);
        }
    }
}

// one atom a warp (apw = 1) takes the whole warp; else the system's lane groups
__device__ __forceinline__ void buffer_dispatch(const Dev& d, int bx, int gx, int apw) {
    const int lpa = apw == 1 ? 32 : gather_lpa(d);
    if (lpa == 8) buffer_body<8>(d, bx, gx, apw);
    else if (lpa == 16) buffer_body<16>(d, bx, gx, apw);
    else buffer_body<32>(d, bx, gx, apw);
}

__global__ void __launch_bounds__(BUF_WARPS * 32) k_buffer(Dev d, int apw) {
    buffer_dispatch(d, blockIdx.x, gridDim.x, apw);
}

// Per-block counts of the two evaluated sets (and of the diagnostic sets).
__device__ __forceinline__ void count_body(const Dev& d, int bx) {
    const int64_t i = bx * (int64_t)SCAN_BLOCK + threadIdx.x;
    int f = 0;
    double lam = 0.0;
    if (i < d.n) {
        f = d.flags[i];
        lam = d.lam[i];
    }
    const bool in = i < d.n;
    const int ne = __syncthreads_count(in && (f & 4));
    const int ncheap = __syncthreads_count(in && (f & 8));
    const int ncore = __syncthreads_count(in && lam == 1.0);
    const int nramp = __syncthreads_count(in && lam > 0.0 && lam < 1.0);
    const int nle = __syncthreads_count(in && (f & 1));
    const int nlc = __syncthreads_count(in && (f & 2));
    if (threadIdx.x == 0) {
        d.blk_e[bx] = ne;
        d.blk_c[bx] = ncheap;
        atomicAdd(d.status + SW_NCORE, ncore);
        atomicAdd(d.status + SW_NRAMP, nramp);
        atomicAdd(d.status + SW_NLE, nle);
        atomicAdd(d.status + SW_NLC, nlc);
    }
}
__global__ void __launch_bounds__(SCAN_BLOCK) k_count(Dev d) { count_body(d, blockIdx.x); }

// Ordered compaction: act lists ascending, pos maps (-1 when not evaluated).
__device__ __forceinline__ void scatter_body(const Dev& d, int bx, int gx) {
    __shared__ int red_e[32], red_c[32];
    __shared__ int off_e_s, off_c_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = bx;
    // offset of this block: sum of the counts of the blocks before it
    int se = 0, sc = 0;
    for (int k = tid; k < b; k += SCAN_BLOCK) {
        se += d.blk_e[k];
        sc += d.blk_c[k];
    }
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xffffffffu, se, o);
        sc += __shfl_down_sync(0xffffffffu, sc, o);
    }
    if (lane == 0) {
        red_e[warp] = se;
        red_c[warp] = sc;
    }
    __syncthreads();
    if (warp == 0) {
        int a = red_e[lane], c = red_c[lane];
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            c += __shfl_down_sync(0xffffffffu, c, o);
        }
        if (lane == 0) {
            off_e_s = a;
            off_c_s = c;
        }
    }
    __syncthreads();
    const int64_t i = (int64_t)b * SCAN_BLOCK + tid;
    const int f = i < d.n ? d.flags[i] : 0;
    const bool ie = (f & 4) != 0, ic = (f & 8) != 0;
    const unsigned be = __ballot_sync(0xffffffffu, ie), bc = __ballot_sync(0xffffffffu, ic);
    const unsigned lt = (1u << lane) - 1u;
    __syncthreads();
    if (lane == 0) {
        red_e[warp] = __popc(be);
        red_c[warp] = __popc(bc);
    }
    __syncthreads();
    if (warp == 0) {
        int a = red_e[lane], c = red_c[lane];
        int ia = a, ic2 = c;
        for (int o = 1; o < 32; o <<= 1) {
            int ta = __shfl_up_sync(0xffffffffu, ia, o);
            int tc = __shfl_up_sync(0xffffffffu, ic2, o);
            if (lane >= o) {
                ia += ta;
                ic2 += tc;
            }
        }
        red_e[lane] = ia - a;   // exclusive per-warp offsets
        red_c[lane] = ic2 - c;
        if (lane == 31 && b == gx - 1) {
            d.status[SW_NEXP] = off_e_s + ia;
            d.status[SW_NCHEAP] = off_c_s + ic2;
        }
    }
    __syncthreads();
    if (i < d.n) {
        if (ie) {
            const int p = off_e_s + red_e[warp] + __popc(be & lt);
            d.act_e[p] = (int)i;
            d.pos_e[i] = p;
        } else {
            d.pos_e[i] = -1;
        }
        if (ic) {
            const int p = off_c_s + red_c[warp] + __popc(bc & lt);
            d.act_c[p] = (int)i;
            d.pos_c[i] = p;
        } else {
            d.pos_c[i] = -1;
        }
    }
}
__global__ void __launch_bounds__(SCAN_BLOCK) k_scatter(Dev d) { scatter_body(d, blockIdx.x, gridDim.x); }

// ---------------------------------------------------------------------------
// multi-system versions (geometric regions only)

__global__ void kb_lambda(BatchArgs ba, const Regions* __restrict__ regions) {
    MIX_BATCH_BLOCK(ba)
    __shared__ Regions s_reg;   // the system's regions, read per atom
    copy_shared(&s_reg, regions + s_ent.x);
    __syncthreads();
    lambda_body(s_dev, s_reg, s_ent.y, s_ent.z);
}
__global__ void __launch_bounds__(BUF_WARPS * 32) kb_buffer(BatchArgs ba) {
    MIX_BATCH_BLOCK(ba)
    buffer_dispatch(s_dev, s_ent.y, s_ent.z, 32);
}
__global__ void __launch_bounds__(SCAN_BLOCK) kb_count(BatchArgs ba) {
    MIX_BATCH_BLOCK(ba)
    count_body(s_dev, s_ent.y);
}
__global__ void __launch_bounds__(SCAN_BLOCK) kb_scatter(BatchArgs ba) {
    MIX_BATCH_BLOCK(ba)
    scatter_body(s_dev, s_ent.y, s_ent.z);
}

// Flattened lists of the evaluated atoms of every system: block s writes
// {s, i} for each atom i of its cheap list, and {s, ACE_GROUP k} for each group of
// ACE_GROUP consecutive atoms of its expensive list (a CTA of the expensive
// kernel takes one such group), at the sum of the counts of the systems before
// it (within its expensive group; all systems for cheap).  The last system of
// a group writes the group's total; the last system the cheap total.
__global__ void kb_flatten(FlatArgs f) {
    __shared__ int red[2][32];
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = f.egroup[s];
    int oe = 0, oc = 0;
    for (int t = tid; t < s; t += blockDim.x) {
        const int* st = f.devs[t].status;
        if (f.egroup[t] == g) oe += (st[SW_NEXP] + ACE_GROUP - 1) / ACE_GROUP;
        oc += st[SW_NCHEAP];
    }
    for (int o = 16; o > 0; o >>= 1) {
        oe += __shfl_down_sync(0xffffffffu, oe, o);
        oc += __shfl_down_sync(0xffffffffu, oc, o);
    }
    if (lane == 0) {
        red[0][warp] = oe;
        red[1][warp] = oc;
    }
    __syncthreads();
    oe = 0;
    oc = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        oe += red[0][w];
        oc += red[1][w];
    }
    const int* st = f.devs[s].status;
    const int ne = (st[SW_NEXP] + ACE_GROUP - 1) / ACE_GROUP, nc = st[SW_NCHEAP];
    int2* le = f.list_e + f.ebase[g] + oe;
    int2* lc = f.list_c + oc;
    for (int k = tid; k < ne; k += blockDim.x) le[k] = make_int2(s, k * ACE_GROUP);
    const int* act_c = f.devs[s].act_c;
    for (int k0 = tid; k0 < nc; k0 += 4 * blockDim.x) {   // four reads in flight a thread
        int v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (k0 + u * (int)blockDim.x < nc) v[u] = act_c[k0 + u * blockDim.x];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (k0 + u * (int)blockDim.x < nc) lc[k0 + u * blockDim.x] = make_int2(s, v[u]);
    }
    if (tid == 0) {
        if (f.elast[s]) f.counts[g] = oe + ne;
        if (s == f.nsys - 1) f.counts[f.ngrp] = oc + nc;
    }
}

int sets_launches(const SeedRule& sr) { return sr.mode == 0 ? 4 : (sr.mode == 1 ? 5 : 6); }

void launch_sets(const Dev& d, const Regions& r, const SeedRule& sr, cudaStream_t s) {
    const int nb = (int)((d.n + 255) / 256);
    if (sr.mode == 0) {
        k_lambda<<<nb > 0 ? nb : 1, 256, 0, s>>>(d, r);
    } else {
        int64_t want = (d.n + SEED_WARPS - 1) / SEED_WARPS;
        int64_t lim = (int64_t)sm_count() * 8;
        const int gs = (int)(want < lim ? want : lim);
        if (sr.mode == 2) k_coord<<<gs > 0 ? gs : 1, SEED_WARPS * 32, 0, s>>>(d, sr);
        k_core<<<gs > 0 ? gs : 1, SEED_WARPS * 32, 0, s>>>(d, sr);
        k_blend<<<gs > 0 ? gs : 1, SEED_WARPS * 32, 0, s>>>(d, sr);
    }
    // atoms per warp: one up to 512 atoms per SM (a 256,000-atom system gets 3,
    // which keeps its shell of scanning atoms spread over many warps), up to 32
    // beyond
    const int64_t warps_full = (int64_t)sm_count() * 512;
    int64_t apw = (d.n + warps_full - 1) / warps_full;
    apw = apw < 1 ? 1 : (apw > 32 ? 32 : apw);
    int64_t want = (d.n + BUF_WARPS * apw - 1) / (BUF_WARPS * apw);
    int64_t lim = d.grid_buffer > 0 ? d.grid_buffer : (int64_t)sm_count() * 8;
    const int gb = (int)(want < lim ? want : lim);
    k_buffer<<<gb > 0 ? gb : 1, BUF_WARPS * 32, 0, s>>>(d, (int)apw);
    k_count<<<d.nblk, SCAN_BLOCK, 0, s>>>(d);
    k_scatter<<<d.nblk, SCAN_BLOCK, 0, s>>>(d);
}

}  // namespace mixd

namespace mixd {

void launch_sets_batch(const BatchPlan& p, cudaStream_t s) {
    kb_lambda<<<p.nblk[BT_ATOM], 256, 0, s>>>(p.ba[BT_ATOM], p.regions);
    kb_buffer<<<p.nblk[BT_WARP8], BUF_WARPS * 32, 0, s>>>(p.ba[BT_WARP8]);
    kb_count<<<p.nblk[BT_SCAN], SCAN_BLOCK, 0, s>>>(p.ba[BT_SCAN]);
    kb_scatter<<<p.nblk[BT_SCAN], SCAN_BLOCK, 0, s>>>(p.ba[BT_SCAN]);
    kb_flatten<<<p.flat.nsys, 1024, 0, s>>>(p.flat);
}

}  // namespace mixd
