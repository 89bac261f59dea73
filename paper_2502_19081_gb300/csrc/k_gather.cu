// Force assembly and blend (Alg. 4) without atomics, fused with the second
// half of velocity Verlet.
//
// With g^p_ij = dE^p_i / dr_ij stored per list slot by the potential kernels
// (in atom i's own row, and in atom j's incoming row at the slot of i), the
// force of potential p on atom k restricted to its evaluated set A_p is
//   Phi^p_k = [k in A_p] sum_j g^p_kj - sum_{i in N(k), i in A_p} g^p_{i, rev(k in i)},
// two coalesced rows per potential and atom.
// the site-energy derivative sum of Sec. 4.5.  Then
//   F_k = w_k Phi^exp_k + (1 - w_k) Phi^cheap_k,
// each term evaluated only where its weight is non-zero.  One warp per atom,
// lanes over the list slots, a fixed-order shuffle reduction in float64.
#include "mix_launch.h"

namespace mixd {

constexpr int G_WARPS = 8;

constexpr int G_ATOMS = 32;   // most atoms a warp gathers before finishing them lane-parallel

template <typename T>
using GSum = decltype(warp_sum(T(0)));

// A warp gathers ga <= G_ATOMS atoms one after another (lanes over list slots, float
// or float64 sums per potential and component, compensated for float) and parks
// the six lane-0 sums per atom in shared memory; then thread t of the block
// finishes atom t of the block's chunk of G_WARPS * ga atoms in float64 (blend,
// non-finite check, second half-kick).  The float64 pipe of this part runs at
// 1/64 of the float rate and a warp-wide float64 instruction costs the same
// with one active lane as with 32, so one float64 instruction should serve many
// atoms: finishing per block rather than per warp keeps that true when ga is
// small (ga trades gather latency against the warps a small system keeps busy).
// LPA lanes gather one atom (a warp, or half or a quarter of a warp where lists
// are short: two or four atoms of the warp's share at a time).
template <typename T, int LPA>
__device__ __forceinline__ void gather_body(const Dev& d, int bx, int gx, int integrate, double h, int ga,
                                            GSum<T>* park) {
    using V = typename Vec4<T>::type;
    constexpr int G = 32 / LPA;
    constexpr int GU = LPA == 8 ? 4 : 2;   // slots a lane loads before summing them
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane & (LPA - 1), grp = lane / LPA;
    const unsigned mask = LPA == 32 ? 0xffffffffu : (((1u << LPA) - 1u) << (lane & ~(LPA - 1)));
    const V* GE = reinterpret_cast<const V*>(d.ge);
    const V* GC = reinterpret_cast<const V*>(d.gc);
    const V* GEI = reinterpret_cast<const V*>(d.ge_in);
    const V* GCI = reinterpret_cast<const V*>(d.gc_in);
    const int cap = d.cap;
    const int stamp = d.status[SW_EPOCH];
    // the block takes chunks of G_WARPS * ga consecutive atoms, warp w atoms w*ga ..
    const int64_t per_block = (int64_t)G_WARPS * ga;
    for (int64_t b0 = (int64_t)bx * per_block; b0 < d.n; b0 += (int64_t)gx * per_block) {
        const int nb = (int)(d.n - b0 < per_block ? d.n - b0 : per_block);
        const int a0 = warp * ga;
        const int na = nb - a0 >= ga ? ga : (nb - a0 > 0 ? nb - a0 : 0);
        // the next atom's list length and flags are loaded ahead
        int mn = 0, fn = 0;
        if (grp < na) {
            mn = d.nnb[b0 + a0 + grp];
            fn = d.flags[b0 + a0 + grp];
        }
        for (int a = grp; a < na; a += G) {
            const int64_t k = b0 + a0 + a;
            const int m = mn, fk = fn;
            if (a + G < na) {
                mn = d.nnb[k + G];
                fn = d.flags[k + G];
            }
            const bool own_e = (fk & 4) != 0, own_c = (fk & 8) != 0;
            // w > 0 iff lambda > 0 and w < 1 iff lambda < 1 (flags bits 0, 1)
            const bool use_e = (fk & 1) != 0, use_c = (fk & 2) != 0;
            const int64_t base = k * cap;
            // own row: dE_k/dr_kj; incoming row: dE_j/dr_jk, present when j was
            // evaluated in this evaluation (its stamp is current).  A lane loads
            // GU of its slots before it sums them (in slot order).
            T tex = T(0), tey = T(0), tez = T(0), tcx = T(0), tcy = T(0), tcz = T(0);
            for (int s0 = sub; s0 < m; s0 += GU * LPA) {
                if (use_e) {   // few atoms: slot by slot
#pragma unroll 1
                    for (int s = s0; s < m && s < s0 + GU * LPA; s += LPA) {
                        if (own_e) {
                            const V g = GE[base + s];
                            tex += g.x;
                            tey += g.y;
                            tez += g.z;
                        }
                        const V g = GEI[base + s];
                        if (stamp_is(g.w, stamp)) {
                            tex -= g.x;
                            tey -= g.y;
                            tez -= g.z;
                        }
                    }
                }
                if (use_c) {
                    V go[GU], gi[GU];
#pragma unroll
                    for (int u = 0; u < GU; ++u) {
                        const int s = s0 + u * LPA;
                        if (s < m) {
                            if (own_c) go[u] = GC[base + s];
                            gi[u] = GCI[base + s];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < GU; ++u) {
                        if (s0 + u * LPA < m) {
                            if (own_c) {
                                tcx += go[u].x;
                                tcy += go[u].y;
                                tcz += go[u].z;
                            }
                            if (stamp_is(gi[u].w, stamp)) {
                                tcx -= gi[u].x;
                                tcy -= gi[u].y;
                                tcz -= gi[u].z;
                            }
                        }
                    }
                }
            }
            // lanes combined in a fixed order (only for the potentials the atom uses:
            // the flags are uniform over the group)
            GSum<T> r0{}, r1{}, r2{}, r3{}, r4{}, r5{};
            if (use_e) {
                r0 = group_sum<LPA>(tex, mask);
                r1 = group_sum<LPA>(tey, mask);
                r2 = group_sum<LPA>(tez, mask);
            }
            if (use_c) {
                r3 = group_sum<LPA>(tcx, mask);
                r4 = group_sum<LPA>(tcy, mask);
                r5 = group_sum<LPA>(tcz, mask);
            }
            if (sub == 0) {
                GSum<T>* q = park + (a0 + a) * 6;
                q[0] = r0;
                q[1] = r1;
                q[2] = r2;
                q[3] = r3;
                q[4] = r4;
                q[5] = r5;
            }
        }
        // thread t finishes atom t of the chunk: one float64 instruction serves
        // up to 32 atoms however the chunk was split over the warps (with a
        // full warp's worth of atoms per warp, each warp finishes its own)
        const bool own = ga == G_ATOMS;
        if (own) __syncwarp();
        else __syncthreads();
        const int t = own ? a0 + lane : (int)threadIdx.x;
        if (own ? lane < na : t < nb) {
            const int64_t k = b0 + t;
            const GSum<T>* q = park + t * 6;
            const double ex = lane0_double(q[0]), ey = lane0_double(q[1]), ez = lane0_double(q[2]);
            const double cx = lane0_double(q[3]), cy = lane0_double(q[4]), cz = lane0_double(q[5]);
            const double w = d.wgt[k];
            const double wc = 1.0 - w;
            double4 F;
            F.x = (w > 0.0 ? w * ex : 0.0) + (wc > 0.0 ? wc * cx : 0.0);
            F.y = (w > 0.0 ? w * ey : 0.0) + (wc > 0.0 ? wc * cy : 0.0);
            F.z = (w > 0.0 ? w * ez : 0.0) + (wc > 0.0 ? wc * cz : 0.0);
            F.w = 0.0;
            if (!(isfinite(F.x) && isfinite(F.y) && isfinite(F.z))) set_status(d.status, ST_NONFINITE);
            d.f[k] = F;
            if constexpr (sizeof(T) == 4) {
                // site energies of the float path (warp sums parked by the potentials)
                const int fl = d.flags[k];
                double ee = 0.0, ec = 0.0;
                if (fl & 4) {
                    const float2 pe = d.epark_e[k];
                    ee = (double)pe.x + (double)pe.y;
                }
                if (fl & 8) {
                    const float2 pc = d.epark_c[k];
                    ec = (double)pc.x + (double)pc.y;
                }
                d.esite_e[k] = ee;
                d.esite_c[k] = ec;
            }
            if (integrate) {
                double4 v = d.v[k];
                v.x = __dadd_rn(v.x, __dmul_rn(h, F.x));
                v.y = __dadd_rn(v.y, __dmul_rn(h, F.y));
                v.z = __dadd_rn(v.z, __dmul_rn(h, F.z));
                d.v[k] = v;
            }
        }
        if (own) __syncwarp();
        else __syncthreads();   // the park is reused by the next chunk
    }
}

template <typename T, int LPA>
__global__ void __launch_bounds__(G_WARPS * 32, sizeof(T) == 4 ? 4 : 2) k_gather(Dev d, int integrate, double h, int ga) {
    __shared__ GSum<T> park[G_WARPS * G_ATOMS * 6];
    gather_body<T, LPA>(d, blockIdx.x, gridDim.x, integrate, h, ga, park);
}


// Each block belongs to one system and gathers with that system's own lane
// groups, so a system's forces are bit for bit those it gets alone.
template <typename T>
__global__ void __launch_bounds__(G_WARPS * 32) kb_gather(BatchArgs ba, int integrate, double dt) {
    __shared__ GSum<T> park[G_WARPS * G_ATOMS * 6];
    MIX_BATCH_BLOCK(ba)
    const double h = half_kick(dt, s_dev.mass);
    const int lpa = gather_lpa(s_dev);
    if (lpa == 8) gather_body<T, 8>(s_dev, s_ent.y, s_ent.z, integrate, h, G_ATOMS, park);
    else if (lpa == 16) gather_body<T, 16>(s_dev, s_ent.y, s_ent.z, integrate, h, G_ATOMS, park);
    else gather_body<T, 32>(s_dev, s_ent.y, s_ent.z, integrate, h, G_ATOMS, park);
}

void launch_gather_batch(const BatchPlan& p, int precision, int integrate, double dt, cudaStream_t s) {
    if (precision == MIX_FP64)
        kb_gather<double><<<p.nblk[BT_GATHER], G_WARPS * 32, 0, s>>>(p.ba[BT_GATHER], integrate, dt);
    else
        kb_gather<float><<<p.nblk[BT_GATHER], G_WARPS * 32, 0, s>>>(p.ba[BT_GATHER], integrate, dt);
}

void launch_gather(const Dev& d, int precision, int integrate, double h, cudaStream_t s) {
    const int lpa = gather_lpa(d);
    // atoms per warp: enough warps for about half occupancy, at most G_ATOMS, and
    // with quarter-warp groups at least one atom per group; in large systems
    // small enough that every resident CTA takes about four chunks, so the last
    // wave of chunks is not a partly empty one (256,000 atoms in chunks of
    // 8 x 32 are 1.6 waves of the 608 resident CTAs)
    const int64_t warps_wanted = (int64_t)sm_count() * 32;
    int ga = (int)((d.n + warps_wanted - 1) / warps_wanted);
    const int64_t resident = (int64_t)sm_count() * (precision == MIX_FP64 ? 2 : 4);   // the launch bounds
    const int64_t ga_waves = (d.n + G_WARPS * resident * 4 - 1) / (G_WARPS * resident * 4);
    if (ga > ga_waves) ga = (int)ga_waves;
    ga = ga < 32 / lpa ? 32 / lpa : (ga > G_ATOMS ? G_ATOMS : ga);
    const int64_t per_block = (int64_t)G_WARPS * ga;
    int64_t want = (d.n + per_block - 1) / per_block;
    int64_t lim = d.grid_gather > 0 ? d.grid_gather : (int64_t)sm_count() * 8;
    const int grid = (int)(want < lim ? want : lim);
    const int gr = grid > 0 ? grid : 1;
    if (precision == MIX_FP64) {
        if (lpa == 8) k_gather<double, 8><<<gr, G_WARPS * 32, 0, s>>>(d, integrate, h, ga);
        else if (lpa == 16) k_gather<double, 16><<<gr, G_WARPS * 32, 0, s>>>(d, integrate, h, ga);
        else k_gather<double, 32><<<gr, G_WARPS * 32, 0, s>>>(d, integrate, h, ga);
    } else {
        if (lpa == 8) k_gather<float, 8><<<gr, G_WARPS * 32, 0, s>>>(d, integrate, h, ga);
        else if (lpa == 16) k_gather<float, 16><<<gr, G_WARPS * 32, 0, s>>>(d, integrate, h, ga);
        else k_gather<float, 32><<<gr, G_WARPS * 32, 0, s>>>(d, integrate, h, ga);
    }
}

}  // namespace mixd
