// Cheap potential: a 2+3-body cubic B-spline site energy evaluated on the
// compacted list of atoms in Lambda_cheap plus its buffer (Sec. 4.5, Alg. 4):
//   E_i = 1/2 sum_j V2(r_ij) + sum_{j<k; r_ij, r_ik < rc3} V3(r_ij, r_ik, r_jk).
// A group of LPA lanes per evaluated atom (a whole warp, or half or a quarter
// of a warp where atoms have few neighbours: two or four atoms a warp).  Lanes own list slots for the
// 2-body part and the final write; the 3-body pairs (p, q), p < q, numbered
// t = q (q - 1) / 2 + p (so the pairs of the first n3 neighbours are t <
// n3 (n3 - 1) / 2 whatever n3 is), are spread over the lanes, their partial
// derivatives go to per-group tables, and each lane then sums the pairs of its
// own 3-body neighbour in a fixed order (no atomics, so results are
// bit-reproducible).
//   dV3 -> g_p += a_p u_p + c_pq (r_p - r_q),  a_p = dV3/d r_p,
//          c_pq = (dV3/dr_pq) / r_pq  (c3 symmetric in its first two indices).
// Coefficients are read as windows: the four control points of one interval
// are one aligned vector (one shared-memory load).
#include "mix_launch.h"

namespace mixd {

constexpr int SPL_WARPS = 4;

// three-body neighbours an atom may have on chip: NB3MAX with a warp per atom,
// fewer with half or a quarter of a warp (the per-group tables grow as the square)
template <int LPA>
__host__ __device__ constexpr int spl_nb() {
    return LPA == 32 ? NB3MAX : (LPA == 16 ? 24 : 16);
}

__device__ __forceinline__ double trsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float trsqrt(float x) { return rsqrtf(x); }

template <typename T>
__device__ __forceinline__ void bspline4(T x, int qmax, int& q, T b[4], T db[4]) {
    q = (int)floor(x);
    q = q < 0 ? 0 : (q > qmax ? qmax : q);
    const T u = x - T(q), w = T(1) - u;
    const T u2 = u * u, u3 = u2 * u;
    b[0] = w * w * w * T(1.0 / 6.0);
    b[1] = (T(3) * u3 - T(6) * u2 + T(4)) * T(1.0 / 6.0);
    b[2] = (T(-3) * u3 + T(3) * u2 + T(3) * u + T(1)) * T(1.0 / 6.0);
    b[3] = u3 * T(1.0 / 6.0);
    db[0] = T(-0.5) * w * w;
    db[1] = T(1.5) * u2 - T(2) * u;
    db[2] = T(-1.5) * u2 + u + T(0.5);
    db[3] = T(0.5) * u2;
}

// An atom's list length and the first list slot and reverse slot of a lane,
// loaded while the previous atom is evaluated, so that an atom's first partner
// positions wait on one load rather than three in a chain.
struct AtomHead {
    int m, j0, r0;
};

template <typename T, int NB>
struct SplWarp {   // per-group shared scratch
    static constexpr int NP = NB * (NB - 1) / 2;
    typename Vec4<T>::type v[NB];   // r_ij (x, y, z) and |r_ij| of the 3-body neighbours
    T hp[NB];           // (dV2/dr) / (2 r): the slot's 2-body gradient is hp r_ij
    T ir[NB];           // 1 / |r_ij|
    int slot[NB];
    T a1[NP];           // pair t = (p, q): dV3/dr_p
    T a2[NP];           //                  dV3/dr_q
    T cc[NP];           //                  (dV3/dr_pq) / r_pq
};

// shared bytes of the pair-number table tq[t] = q of pair t (the block's groups share it)
template <int NB>
__host__ __device__ constexpr int spl_tq_bytes() {
    return (NB * (NB - 1) / 2 + 15) / 16 * 16;
}

template <int NB>
__device__ __forceinline__ void spl_fill_tq(unsigned char* tq) {
    for (int t = threadIdx.x; t < NB * (NB - 1) / 2; t += blockDim.x) {
        int q = 1;
        while (q * (q + 1) / 2 <= t) ++q;
        tq[t] = (unsigned char)q;
    }
}

// One evaluated atom i (an entry of the system's cheap list), by the group of
// LPA lanes that owns W; the coefficient windows c2w, c3w may sit in shared or
// global memory.  Returns the atom's 3-body neighbour count (before any clamp
// to the on-chip slots).
template <typename T, int LPA>
__device__ __forceinline__ int spline_atom(const Dev& d, const SplTab<T>& tab, int i,
                                            const typename Vec4<T>::type* c2w, const typename Vec4<T>::type* c3w,
                                            const unsigned char* tq, SplWarp<T, spl_nb<LPA>()>& W,
                                            const AtomHead* head = nullptr) {
    constexpr int NB = spl_nb<LPA>();
    using V = typename Vec4<T>::type;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (LPA - 1);
    const unsigned mask = LPA == 32 ? 0xffffffffu : (((1u << LPA) - 1u) << (lane & ~(LPA - 1)));
    V* GC = reinterpret_cast<V*>(d.gc);
    V* GIN = reinterpret_cast<V*>(d.gc_in);
    const int stamp = d.status[SW_EPOCH];
    const T rc2 = tab.rc2, rc32 = tab.rc32;
    const T invh2 = tab.invh2, invh3 = tab.invh3, invhc = tab.invhc;
    const unsigned lt = (1u << lane) - 1u;   // the ballots carry this group's lanes only
    const int cap = d.cap;
    int n3_all = 0;
    {
        using Pt = typename PairFrame<T>::Pt;
        const PairFrame<T> pf(d, i);
        const typename PairFrame<T>::Geo geo = PairFrame<T>::geo(d);   // once per atom, in registers
        const int m = head ? head->m : d.nnb[i];
        const int* row = d.nbr + (int64_t)i * cap;
        const int* rvr = d.rev + (int64_t)i * cap;
        V* grow = GC + (int64_t)i * cap;
        T ep = T(0);
        int n3 = 0;
        // 2-body part; a slot without 3-body terms is final here (own row and the
        // partner's incoming row); a 3-body slot waits in the group's table.
        // The next chunk's partner, reverse slot and position are loaded before
        // this chunk is evaluated, so their latency overlaps its arithmetic.
        int jn = 0, rn = 0;
        Pt ptn{};
        if (sub < m) {
            jn = head ? head->j0 : row[sub];
            rn = head ? head->r0 : rvr[sub];
            ptn = PairFrame<T>::load(d, jn);
        }
        for (int c = 0; c * LPA < m; ++c) {
            const int s = c * LPA + sub;
            const int j = jn, rj = rn;
            const Pt pt = ptn;
            if (s + LPA < m) {
                jn = row[s + LPA];
                rn = rvr[s + LPA];
                ptn = PairFrame<T>::load(d, jn);
            }
            bool is3 = false;
            T dv3[3] = {T(0), T(0), T(0)}, r = T(0), hp = T(0), ri = T(0);
            if (s < m) {
                T r2;
                pf.vec(geo, pt, dv3, r2);
                if (r2 < rc2) {
                    ri = trsqrt(r2);
                    r = r2 * ri;
                    int q;
                    T b[4], db[4];
                    bspline4<T>(r * invh2, SPL_W2 - 1, q, b, db);
                    const V w = c2w[q];
                    const T v = w.x * b[0] + w.y * b[1] + w.z * b[2] + w.w * b[3];
                    const T dv = (w.x * db[0] + w.y * db[1] + w.z * db[2] + w.w * db[3]) * invh2;
                    ep += T(0.5) * v;
                    hp = T(0.5) * dv * ri;
                    is3 = r2 < rc32;
                }
            }
            const unsigned bal = __ballot_sync(mask, is3);
            const int p = is3 ? n3 + __popc(bal & lt) : -1;
            if (is3 && p < NB) {
                V u;
                u.x = dv3[0];
                u.y = dv3[1];
                u.z = dv3[2];
                u.w = r;
                W.v[p] = u;
                W.hp[p] = hp;
                W.ir[p] = ri;
                W.slot[p] = s;
            } else if (s < m) {
                V gv;
                gv.x = hp * dv3[0];
                gv.y = hp * dv3[1];
                gv.z = hp * dv3[2];
                gv.w = T(0);
                grow[s] = gv;
                gv.w = stamp_as(T(0), stamp);
                GIN[(int64_t)j * cap + rj] = gv;   // the partner's incoming row
            }
            n3 += __popc(bal);
        }
        n3_all = n3;
        if (n3 > NB) {
            if (sub == 0) {
                set_status(d.status, ST_NB3_OVERFLOW);
                atomicMax(d.status + SW_NB3MAX, n3);
            }
            n3 = NB;
        }
        __syncwarp(mask);
        // 3-body pairs t = q (q - 1) / 2 + p, p < q < n3, over the lanes
        const int npair = n3 * (n3 - 1) / 2;
        for (int t = sub; t < npair; t += LPA) {
            const int q = tq[t], p = t - q * (q - 1) / 2;
            const V vp = W.v[p], vq = W.v[q];
            const T wx = vq.x - vp.x, wy = vq.y - vp.y, wz = vq.z - vp.z;
            const T w2 = wx * wx + wy * wy + wz * wz;
            const T ri3 = w2 > T(0) ? trsqrt(w2) : T(0);
            const T r3 = w2 * ri3;
            int qa, qb, qc;
            T ba[4], dba[4], bb[4], dbb[4], bc[4], dbc[4];
            bspline4<T>(vp.w * invh3, SPL_W3 - 1, qa, ba, dba);
            bspline4<T>(vq.w * invh3, SPL_W3 - 1, qb, bb, dbb);
            bspline4<T>(r3 * invhc, SPL_W3 - 1, qc, bc, dbc);
            // contract the third argument, then the second, then the first
            T val = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const V* cr = c3w + ((qa + x) * 8 + qb) * SPL_W3 + qc;
                T s0 = T(0), s1 = T(0), s3 = T(0);
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const V w = cr[y * SPL_W3];
                    const T t0 = w.x * bc[0] + w.y * bc[1] + w.z * bc[2] + w.w * bc[3];
                    const T t1 = w.x * dbc[0] + w.y * dbc[1] + w.z * dbc[2] + w.w * dbc[3];
                    s0 += t0 * bb[y];
                    s1 += t0 * dbb[y];
                    s3 += t1 * bb[y];
                }
                val += s0 * ba[x];
                d1 += s0 * dba[x];
                d2 += s1 * ba[x];
                d3 += s3 * ba[x];
            }
            ep += val;
            W.a1[t] = d1 * invh3;
            W.a2[t] = d2 * invh3;
            W.cc[t] = d3 * invhc * ri3;
        }
        __syncwarp(mask);
        // 3-body slots: 2-body part plus the sum over the other 3-body neighbours
        // (q ascending: first the pairs (q, p), then the pairs (p, q))
        for (int p = sub; p < n3; p += LPA) {
            T sa = T(0), cx = T(0), cy = T(0), cz = T(0), cs = T(0);
            const int tp = p * (p - 1) / 2;
            for (int q = 0; q < p; ++q) {
                const T c = W.cc[tp + q];
                const V vq = W.v[q];
                sa += W.a2[tp + q];
                cs += c;
                cx += c * vq.x;
                cy += c * vq.y;
                cz += c * vq.z;
            }
            for (int q = p + 1; q < n3; ++q) {
                const int t = q * (q - 1) / 2 + p;
                const T c = W.cc[t];
                const V vq = W.v[q];
                sa += W.a1[t];
                cs += c;
                cx += c * vq.x;
                cy += c * vq.y;
                cz += c * vq.z;
            }
            const V vp = W.v[p];
            const T k = W.hp[p] + sa * W.ir[p] + cs;
            V gv;
            gv.x = k * vp.x - cx;
            gv.y = k * vp.y - cy;
            gv.z = k * vp.z - cz;
            gv.w = T(0);
            const int s = W.slot[p];
            grow[s] = gv;
            gv.w = stamp_as(T(0), stamp);
            GIN[(int64_t)row[s] * cap + rvr[s]] = gv;
        }
        __syncwarp(mask);
        const auto epart = group_sum<LPA>(ep, mask);   // fixed order; compensated for float
        if constexpr (sizeof(T) == 4) {
            if (sub == 0) d.epark_c[i] = make_float2(epart.s, epart.c);   // converted in the gather
        } else {
            if (sub == 0) d.esite_c[i] = lane0_double(epart);
        }
        __syncwarp(mask);
    }
    return n3_all;
}

// window counts of the two coefficient tables (4-vectors)
constexpr int SPL_NW = 64 * SPL_W3 + SPL_W2;

template <typename T>
__device__ __forceinline__ void spl_stage(typename Vec4<T>::type* dst, const T* c3w, const T* c2w) {
    using V = typename Vec4<T>::type;
    const V* s3 = reinterpret_cast<const V*>(c3w);
    const V* s2 = reinterpret_cast<const V*>(c2w);
    for (int k = threadIdx.x; k < SPL_NW; k += blockDim.x) dst[k] = k < 64 * SPL_W3 ? s3[k] : s2[k - 64 * SPL_W3];
}

template <typename T, int LPA>
__global__ void __launch_bounds__(SPL_WARPS * 32, sizeof(T) == 4 ? 6 : 1) k_spline(Dev d, SplTab<T> tab) {
    constexpr int G = 32 / LPA;   // atoms a warp works on at a time
    constexpr int NB = spl_nb<LPA>();
    using V = typename Vec4<T>::type;
    using SW = SplWarp<T, NB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* c3s = reinterpret_cast<V*>(smem_raw);   // [64 * SPL_W3] then [SPL_W2]
    V* c2s = c3s + 64 * SPL_W3;
    SW* ws = reinterpret_cast<SW*>(c3s + SPL_NW);
    unsigned char* tq = reinterpret_cast<unsigned char*>(ws + SPL_WARPS * G);
    const int warp = threadIdx.x >> 5, grp = (threadIdx.x & 31) / LPA;
    spl_stage<T>(c3s, tab.c3w, tab.c2w);
    spl_fill_tq<NB>(tq);
    __syncthreads();
    const int count = d.status[SW_NCHEAP];
    const int stride = gridDim.x * SPL_WARPS * G;
    int a = (blockIdx.x * SPL_WARPS + warp) * G + grp;
    const int sub = threadIdx.x & (LPA - 1), cap = d.cap;
    // an atom's head (list length, this lane's first slot and reverse slot)
    // is loaded an atom ahead, and the atom index two atoms ahead; the slot
    // loads do not wait for the length (slot sub < cap lies in the atom's row)
    auto load_head = [&](int at) {
        AtomHead hd{0, 0, 0};
        hd.m = d.nnb[at];
        if (sub < cap) {
            hd.j0 = d.nbr[(int64_t)at * cap + sub];
            hd.r0 = d.rev[(int64_t)at * cap + sub];
        }
        return hd;
    };
    int i = a < count ? d.act_c[a] : 0;
    AtomHead hd{0, 0, 0};
    if (a < count) hd = load_head(i);
    int in = a + stride < count ? d.act_c[a + stride] : 0;
    int nb3 = 0;   // the largest 3-body count this lane's group met
    while (a < count) {
        const int an = a + stride;
        const int inn = an + stride < count ? d.act_c[an + stride] : 0;
        AtomHead hn{0, 0, 0};
        if (an < count) hn = load_head(in);
        nb3 = max(nb3, spline_atom<T, LPA>(d, tab, i, c2s, c3s, tq, ws[warp * G + grp], &hd));
        a = an;
        i = in;
        in = inn;
        hd = hn;
    }
    // one atomic a warp: the context's lane groups are narrowed from it
    nb3 = __reduce_max_sync(0xffffffffu, nb3);
    if ((threadIdx.x & 31) == 0 && nb3 > 0) atomicMax(d.status + SW_NB3MAX, nb3);
}

// Many systems: a lane group per entry {system, atom} of the flattened cheap
// list; the system's parameters are read through L1.  When every system has
// the same coefficient tables (uniform != 0) the block stages them once in
// shared memory, as the single-system kernel does; otherwise they are read
// through L1.
template <typename T, int LPA>
__global__ void __launch_bounds__(SPL_WARPS * 32, sizeof(T) == 4 ? 6 : 1) kb_spline(const Dev* __restrict__ devs,
                                                           const SplTab<T>* __restrict__ tabs,
                                                           const int2* __restrict__ list, const int* count_p,
                                                           int uniform) {
    constexpr int G = 32 / LPA;
    constexpr int NB = spl_nb<LPA>();
    using V = typename Vec4<T>::type;
    using SW = SplWarp<T, NB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* c3s = reinterpret_cast<V*>(smem_raw);   // uniform tables only
    V* c2s = c3s + 64 * SPL_W3;
    SW* ws = reinterpret_cast<SW*>(c3s + SPL_NW);
    unsigned char* tq = reinterpret_cast<unsigned char*>(ws + SPL_WARPS * G);
    const int warp = threadIdx.x >> 5, grp = (threadIdx.x & 31) / LPA;
    if (uniform) spl_stage<T>(c3s, tabs[0].c3w, tabs[0].c2w);
    spl_fill_tq<NB>(tq);
    __syncthreads();
    const int count = *count_p;
    const int stride = gridDim.x * SPL_WARPS * G;
    int g = (blockIdx.x * SPL_WARPS + warp) * G + grp;
    int2 e = g < count ? list[g] : make_int2(0, 0);
    while (g < count) {   // the next entry is loaded ahead
        const int gn = g + stride;
        const int2 en = gn < count ? list[gn] : make_int2(0, 0);
        const SplTab<T>& tab = tabs[e.x];
        spline_atom<T, LPA>(devs[e.x], tab, e.y, uniform ? c2s : reinterpret_cast<const V*>(tab.c2w),
                            uniform ? c3s : reinterpret_cast<const V*>(tab.c3w), tq, ws[warp * G + grp]);
        g = gn;
        e = en;
    }
}

template <typename T, int LPA>
static size_t spl_bytes() {
    constexpr int NB = spl_nb<LPA>();
    return SPL_NW * sizeof(typename Vec4<T>::type) + SPL_WARPS * (32 / LPA) * sizeof(SplWarp<T, NB>) +
           spl_tq_bytes<NB>();
}

template <typename T, int LPA>
static cudaError_t spl_shape(const void* kern, size_t* smem, int* grid) {
    const size_t bytes = spl_bytes<T, LPA>();
    cudaError_t e = raise_smem_limit(kern, bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SPL_WARPS * 32, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *smem = bytes;
    *grid = per_sm * sm_count();
    return cudaSuccess;
}

int spline_nb3(int lpa) { return lpa == 8 ? spl_nb<8>() : (lpa == 16 ? spl_nb<16>() : spl_nb<32>()); }

template <typename T>
static cudaError_t spl_batch_cfg(int lpa, size_t* smem, int* grid) {
    if (lpa == 8) return spl_shape<T, 8>((const void*)kb_spline<T, 8>, smem, grid);
    if (lpa == 16) return spl_shape<T, 16>((const void*)kb_spline<T, 16>, smem, grid);
    return spl_shape<T, 32>((const void*)kb_spline<T, 32>, smem, grid);
}

cudaError_t spline_batch_configure(int precision, int lpa, size_t* smem, int* grid) {
    return precision == MIX_FP64 ? spl_batch_cfg<double>(lpa, smem, grid) : spl_batch_cfg<float>(lpa, smem, grid);
}

template <typename T>
static void spl_batch_launch(int lpa, const Dev* devs, const SplTab<T>* t, const int2* list, const int* count,
                             int uniform, size_t smem, int grid, cudaStream_t s) {
    if (lpa == 8) kb_spline<T, 8><<<grid, SPL_WARPS * 32, smem, s>>>(devs, t, list, count, uniform);
    else if (lpa == 16) kb_spline<T, 16><<<grid, SPL_WARPS * 32, smem, s>>>(devs, t, list, count, uniform);
    else kb_spline<T, 32><<<grid, SPL_WARPS * 32, smem, s>>>(devs, t, list, count, uniform);
}

void launch_spline_batch(int precision, int lpa, const Dev* devs, const void* tabs, const int2* list,
                         const int* count, int uniform, size_t smem, int grid, cudaStream_t s) {
    if (precision == MIX_FP64)
        spl_batch_launch<double>(lpa, devs, static_cast<const SplTab<double>*>(tabs), list, count, uniform, smem,
                                 grid, s);
    else
        spl_batch_launch<float>(lpa, devs, static_cast<const SplTab<float>*>(tabs), list, count, uniform, smem,
                                grid, s);
}

template <typename T>
static cudaError_t spl_cfg(int lpa, size_t* smem, int* grid) {
    if (lpa == 8) return spl_shape<T, 8>((const void*)k_spline<T, 8>, smem, grid);
    if (lpa == 16) return spl_shape<T, 16>((const void*)k_spline<T, 16>, smem, grid);
    return spl_shape<T, 32>((const void*)k_spline<T, 32>, smem, grid);
}

cudaError_t spline_configure(int precision, int lpa, size_t* smem, int* grid) {
    return precision == MIX_FP64 ? spl_cfg<double>(lpa, smem, grid) : spl_cfg<float>(lpa, smem, grid);
}

template <typename T>
static void spl_launch(const Dev& d, const SplTab<T>& t, int lpa, size_t smem, int grid, cudaStream_t s) {
    if (lpa == 8) k_spline<T, 8><<<grid, SPL_WARPS * 32, smem, s>>>(d, t);
    else if (lpa == 16) k_spline<T, 16><<<grid, SPL_WARPS * 32, smem, s>>>(d, t);
    else k_spline<T, 32><<<grid, SPL_WARPS * 32, smem, s>>>(d, t);
}

void launch_spline(const Dev& d, const void* tab, int precision, int lpa, size_t smem, int grid, cudaStream_t s) {
    if (precision == MIX_FP64) spl_launch<double>(d, *static_cast<const SplTab<double>*>(tab), lpa, smem, grid, s);
    else spl_launch<float>(d, *static_cast<const SplTab<float>*>(tab), lpa, smem, grid, s);
}

}  // namespace mixd
