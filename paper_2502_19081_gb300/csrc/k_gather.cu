// Force assembly and blend (Alg. 4) without atomics, fused with the second
// half of velocity Verlet.
//
// With g^p_ij = dE^p_i / dr_ij stored per list slot by the potential kernels,
// the force of potential p on atom k restricted to its evaluated set A_p is
//   Phi^p_k = [k in A_p] sum_j g^p_kj - sum_{i in N(k), i in A_p} g^p_{i, rev(k in i)},
// the site-energy derivative sum of Sec. 4.5.  Then
//   F_k = w_k Phi^exp_k + (1 - w_k) Phi^cheap_k,
// each term evaluated only where its weight is non-zero.  One warp per atom,
// lanes over the list slots, a fixed-order shuffle reduction in float64.
#include "mix_launch.h"

namespace mixd {

constexpr int G_WARPS = 8;

template <typename T>
__global__ void __launch_bounds__(G_WARPS * 32) k_gather(Dev d, int integrate, double h) {
    using V = typename Vec4<T>::type;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const V* GE = reinterpret_cast<const V*>(d.ge);
    const V* GC = reinterpret_cast<const V*>(d.gc);
    const int cap = d.cap;
    for (int64_t k = (int64_t)blockIdx.x * G_WARPS + warp; k < d.n; k += (int64_t)gridDim.x * G_WARPS) {
        const double w = d.wgt[k];
        const int m = d.nnb[k];
        const int pe = d.pos_e[k], pc = d.pos_c[k];
        const int* row = d.nbr + k * cap;
        const int* rv = d.rev + k * cap;
        // each lane sums its few slots in T; lanes are combined in float64 below
        T tex = T(0), tey = T(0), tez = T(0), tcx = T(0), tcy = T(0), tcz = T(0);
        for (int s = lane; s < m; s += 32) {
            const int j = row[s];
            const int r = rv[s];
            if (w > 0.0) {
                if (pe >= 0) {
                    const V g = GE[(int64_t)pe * cap + s];
                    tex += g.x;
                    tey += g.y;
                    tez += g.z;
                }
                const int pj = d.pos_e[j];
                if (pj >= 0) {
                    const V g = GE[(int64_t)pj * cap + r];
                    tex -= g.x;
                    tey -= g.y;
                    tez -= g.z;
                }
            }
            if (w < 1.0) {
                if (pc >= 0) {
                    const V g = GC[(int64_t)pc * cap + s];
                    tcx += g.x;
                    tcy += g.y;
                    tcz += g.z;
                }
                const int pj = d.pos_c[j];
                if (pj >= 0) {
                    const V g = GC[(int64_t)pj * cap + r];
                    tcx -= g.x;
                    tcy -= g.y;
                    tcz -= g.z;
                }
            }
        }
        // lanes combined in a fixed order; float partials with a compensated sum
        const double ex = warp_sum_to_double(tex), ey = warp_sum_to_double(tey), ez = warp_sum_to_double(tez);
        const double cx = warp_sum_to_double(tcx), cy = warp_sum_to_double(tcy), cz = warp_sum_to_double(tcz);
        if (lane == 0) {
            const double wc = 1.0 - w;
            double4 F;
            F.x = (w > 0.0 ? w * ex : 0.0) + (wc > 0.0 ? wc * cx : 0.0);
            F.y = (w > 0.0 ? w * ey : 0.0) + (wc > 0.0 ? wc * cy : 0.0);
            F.z = (w > 0.0 ? w * ez : 0.0) + (wc > 0.0 ? wc * cz : 0.0);
            F.w = 0.0;
            if (!(isfinite(F.x) && isfinite(F.y) && isfinite(F.z))) set_status(d.status, ST_NONFINITE);
            d.f[k] = F;
            if (integrate) {
                double4 v = d.v[k];
                v.x = __dadd_rn(v.x, __dmul_rn(h, F.x));
                v.y = __dadd_rn(v.y, __dmul_rn(h, F.y));
                v.z = __dadd_rn(v.z, __dmul_rn(h, F.z));
                d.v[k] = v;
            }
        }
    }
}

void launch_gather(const Dev& d, int precision, int integrate, double h, cudaStream_t s) {
    int64_t want = (d.n + G_WARPS - 1) / G_WARPS;
    int64_t lim = d.grid_gather > 0 ? d.grid_gather : (int64_t)sm_count() * 8;
    const int grid = (int)(want < lim ? want : lim);
    if (precision == MIX_FP64)
        k_gather<double><<<grid > 0 ? grid : 1, G_WARPS * 32, 0, s>>>(d, integrate, h);
    else
        k_gather<float><<<grid > 0 ? grid : 1, G_WARPS * 32, 0, s>>>(d, integrate, h);
}

}  // namespace mixd
