// Cheap potential: a 2+3-body cubic B-spline site energy evaluated on the
// compacted list of atoms in Lambda_cheap plus its buffer (Sec. 4.5, Alg. 4):
//   E_i = 1/2 sum_j V2(r_ij) + sum_{j<k; r_ij, r_ik < rc3} V3(r_ij, r_ik, r_jk).
// A group of LPA lanes per evaluated atom (a whole warp, or half or a quarter
// of a warp where atoms have few neighbours: two or four atoms a warp).  Lanes own list slots for the
// 2-body part and the final write; the 3-body pairs (j, k) are spread over the
// lanes, their partial derivatives go to a per-group table, and each lane then
// sums the rows of its own 3-body neighbour in a fixed order (no atomics, so
// results are bit-reproducible).
//   dV3 -> g_j += a_jk u_j + c_jk (r_j - r_k),  a_jk = dV3/d(first argument),
//          c_jk = (dV3/dr_jk) / r_jk  (c3 symmetric in its first two indices).
#include "mix_launch.h"

namespace mixd {

constexpr int SPL_WARPS = 4;

// three-body neighbours an atom may have on chip: NB3MAX with a warp per atom,
// fewer with half or a quarter of a warp (the per-group tables grow as the square)
template <int LPA>
__host__ __device__ constexpr int spl_nb() {
    return LPA == 32 ? NB3MAX : (LPA == 16 ? 24 : 16);
}

__device__ __forceinline__ double tsqrt3(double x) { return sqrt(x); }
__device__ __forceinline__ float tsqrt3(float x) { return sqrtf(x); }

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

// index of the pair p < q in a packed upper triangle of an NB x NB table
template <int NB>
__device__ __forceinline__ int tri3(int p, int q) { return p * NB - p * (p + 1) / 2 + (q - p - 1); }

template <typename T, int NB>
struct SplWarp {   // per-group shared scratch
    static constexpr int S = NB + 1;   // padded row stride of the pair table
    int slot[NB];
    T v[NB][4];         // r_ij vector (x, y, z) and |r_ij|
    T g2[NB][4];        // 2-body part of dE_i/dr_ij of the 3-body neighbours
    T al[NB * S];       // a_jk
    T cc[NB * (NB - 1) / 2];   // c_jk (symmetric: pairs p < q only)
};

// One evaluated atom (index a of the system's cheap list), by the group of
// LPA lanes that owns W; the coefficient tables c2s, c3s may sit in shared or
// global memory.
template <typename T, int LPA>
__device__ __forceinline__ void spline_atom(const Dev& d, const SplTab<T>& tab, int a, const T* c2s, const T* c3s,
                                            SplWarp<T, spl_nb<LPA>()>& W) {
    constexpr int NB = spl_nb<LPA>();
    constexpr int S = SplWarp<T, NB>::S;
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
    {
        const int i = d.act_c[a];
        const PairFrame<T> pf(d, i);
        const int m = d.nnb[i];
        const int* row = d.nbr + (int64_t)i * cap;
        const int* rvr = d.rev + (int64_t)i * cap;
        V* grow = GC + (int64_t)i * cap;
        T ep = T(0);
        int n3 = 0;
        // 2-body part; a slot without 3-body terms is final here (own row and the
        // partner's incoming row); a 3-body slot waits in the group's table
        for (int c = 0; c * LPA < m; ++c) {
            const int s = c * LPA + sub;
            bool is3 = false;
            T dv3[3] = {T(0), T(0), T(0)}, r = T(0), g2[3] = {T(0), T(0), T(0)};
            if (s < m) {
                T r2;
                pf.vec(d, row[s], dv3, r2);
                if (r2 < rc2) {
                    r = sqrt(r2);
                    T v, dv;
                    int q;
                    T b[4], db[4];
                    bspline4<T>(r * invh2, 12, q, b, db);
                    v = c2s[q] * b[0] + c2s[q + 1] * b[1] + c2s[q + 2] * b[2] + c2s[q + 3] * b[3];
                    dv = (c2s[q] * db[0] + c2s[q + 1] * db[1] + c2s[q + 2] * db[2] + c2s[q + 3] * db[3]) * invh2;
                    ep += T(0.5) * v;
                    const T hp = T(0.5) * dv / r;
                    g2[0] = hp * dv3[0];
                    g2[1] = hp * dv3[1];
                    g2[2] = hp * dv3[2];
                    is3 = r2 < rc32;
                }
            }
            const unsigned bal = __ballot_sync(mask, is3);
            const int p = is3 ? n3 + __popc(bal & lt) : -1;
            if (is3 && p < NB) {
                W.slot[p] = s;
                W.v[p][0] = dv3[0];
                W.v[p][1] = dv3[1];
                W.v[p][2] = dv3[2];
                W.v[p][3] = r;
                W.g2[p][0] = g2[0];
                W.g2[p][1] = g2[1];
                W.g2[p][2] = g2[2];
            } else if (s < m) {
                V gv;
                gv.x = g2[0];
                gv.y = g2[1];
                gv.z = g2[2];
                gv.w = T(0);
                grow[s] = gv;
                gv.w = stamp_as(T(0), stamp);
                GIN[(int64_t)row[s] * cap + rvr[s]] = gv;   // the partner's incoming row
            }
            n3 += __popc(bal);
        }
        if (n3 > NB) {
            if (sub == 0) {
                set_status(d.status, ST_NB3_OVERFLOW);
                atomicMax(d.status + SW_NB3MAX, n3);
            }
            n3 = NB;
        }
        __syncwarp(mask);
        // 3-body pairs p < q, flattened over the lanes
        const int npair = n3 * (n3 - 1) / 2;
        for (int t = sub; t < npair; t += LPA) {
            int p = 0, tt = t;
            while (tt >= n3 - 1 - p) {
                tt -= n3 - 1 - p;
                ++p;
            }
            const int q = p + 1 + tt;
            const T wx = W.v[q][0] - W.v[p][0], wy = W.v[q][1] - W.v[p][1], wz = W.v[q][2] - W.v[p][2];
            const T r3 = tsqrt3(wx * wx + wy * wy + wz * wz);
            int qa, qb, qc;
            T ba[4], dba[4], bb[4], dbb[4], bc[4], dbc[4];
            bspline4<T>(W.v[p][3] * invh3, 4, qa, ba, dba);
            bspline4<T>(W.v[q][3] * invh3, 4, qb, bb, dbb);
            bspline4<T>(r3 * invhc, 4, qc, bc, dbc);
            T val = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
#pragma unroll
            for (int x = 0; x < 4; ++x) {
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const T* cr = c3s + ((qa + x) * 8 + (qb + y)) * 8 + qc;
                    const T t0 = cr[0] * bc[0] + cr[1] * bc[1] + cr[2] * bc[2] + cr[3] * bc[3];
                    const T t1 = cr[0] * dbc[0] + cr[1] * dbc[1] + cr[2] * dbc[2] + cr[3] * dbc[3];
                    val += t0 * ba[x] * bb[y];
                    d1 += t0 * dba[x] * bb[y];
                    d2 += t0 * ba[x] * dbb[y];
                    d3 += t1 * ba[x] * bb[y];
                }
            }
            ep += val;
            const T c = r3 > T(0) ? d3 * invhc / r3 : T(0);
            W.al[p * S + q] = d1 * invh3;
            W.al[q * S + p] = d2 * invh3;
            W.cc[tri3<NB>(p, q)] = c;
        }
        __syncwarp(mask);
        // 3-body slots: 2-body part plus the sum over the other 3-body neighbours
        for (int p = sub; p < n3; p += LPA) {
            T sa = T(0), cx = T(0), cy = T(0), cz = T(0), cs = T(0);
            for (int q = 0; q < n3; ++q) {
                if (q == p) continue;
                const T c = W.cc[p < q ? tri3<NB>(p, q) : tri3<NB>(q, p)];
                sa += W.al[p * S + q];
                cs += c;
                cx += c * W.v[q][0];
                cy += c * W.v[q][1];
                cz += c * W.v[q][2];
            }
            const T ir = T(1) / W.v[p][3];
            V gv;
            gv.x = W.g2[p][0] + (sa * W.v[p][0] * ir + cs * W.v[p][0] - cx);
            gv.y = W.g2[p][1] + (sa * W.v[p][1] * ir + cs * W.v[p][1] - cy);
            gv.z = W.g2[p][2] + (sa * W.v[p][2] * ir + cs * W.v[p][2] - cz);
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
}

template <typename T, int LPA>
__global__ void __launch_bounds__(SPL_WARPS * 32) k_spline(Dev d, SplTab<T> tab) {
    constexpr int G = 32 / LPA;   // atoms a warp works on at a time
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* c3s = reinterpret_cast<T*>(smem_raw);                 // [512]
    T* c2s = c3s + 512;                                       // [16]
    SplWarp<T, spl_nb<LPA>()>* ws = reinterpret_cast<SplWarp<T, spl_nb<LPA>()>*>(c2s + 16);
    const int warp = threadIdx.x >> 5, grp = (threadIdx.x & 31) / LPA;
    for (int k = threadIdx.x; k < 512; k += blockDim.x) c3s[k] = tab.c3[k];
    if (threadIdx.x < 16) c2s[threadIdx.x] = tab.c2[threadIdx.x];
    __syncthreads();
    const int count = d.status[SW_NCHEAP];
    for (int a = (blockIdx.x * SPL_WARPS + warp) * G + grp; a < count; a += gridDim.x * SPL_WARPS * G)
        spline_atom<T, LPA>(d, tab, a, c2s, c3s, ws[warp * G + grp]);
}

// Many systems: a lane group per entry {system, index} of the flattened cheap
// list; the system's parameters are read through L1.  When every system has
// the same coefficient tables (uniform != 0) the block stages them once in
// shared memory, as the single-system kernel does; otherwise they are read
// through L1.
template <typename T, int LPA>
__global__ void __launch_bounds__(SPL_WARPS * 32) kb_spline(const Dev* __restrict__ devs,
                                                           const SplTab<T>* __restrict__ tabs,
                                                           const int2* __restrict__ list, const int* count_p,
                                                           int uniform) {
    constexpr int G = 32 / LPA;
    using SW = SplWarp<T, spl_nb<LPA>()>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SW* ws = reinterpret_cast<SW*>(smem_raw);
    T* c3s = reinterpret_cast<T*>(ws + SPL_WARPS * G);   // [512] (uniform tables only)
    T* c2s = c3s + 512;                                  // [16]
    const int warp = threadIdx.x >> 5, grp = (threadIdx.x & 31) / LPA;
    if (uniform) {
        const T* c3 = tabs[0].c3;
        const T* c2 = tabs[0].c2;
        for (int k = threadIdx.x; k < 512; k += blockDim.x) c3s[k] = c3[k];
        if (threadIdx.x < 16) c2s[threadIdx.x] = c2[threadIdx.x];
        __syncthreads();
    }
    const int count = *count_p;
    for (int g = (blockIdx.x * SPL_WARPS + warp) * G + grp; g < count; g += gridDim.x * SPL_WARPS * G) {
        const int2 e = list[g];
        const SplTab<T>& tab = tabs[e.x];
        spline_atom<T, LPA>(devs[e.x], tab, e.y, uniform ? c2s : tab.c2, uniform ? c3s : tab.c3, ws[warp * G + grp]);
    }
}

template <typename T, int LPA>
static size_t spl_bytes() {
    return SPL_WARPS * (32 / LPA) * sizeof(SplWarp<T, spl_nb<LPA>()>) + (512 + 16) * sizeof(T);
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
