// Expensive potential (templates): a linear atomic cluster expansion evaluated on the
// compacted list of atoms in Lambda_exp plus its buffer (Sec. 4.5, Alg. 4).
//
// A CTA of ACE_GROUP warps takes groups of ACE_GROUP consecutive atoms of the
// expensive list, and warp w owns atom w of its group through every step:
//   1. neighbours inside the cutoff, compacted in slot order (FP64 pair
//      vectors, rounded once to T);
//   2. density A[lm][q] = sum_k R_q(r_k) Y_lm(u_k): the lanes evaluate R
//      (Chebyshev recurrence x (1 - (r/rc)^2)^3) and Y (associated-Legendre
//      recurrence in z times Re/Im (x + iy)^m) for 32 neighbours at a time into
//      shared memory, then each lane accumulates fixed (lm, 4 q) outputs;
//   3. nu <= 2 readout; omega = dE/dA initialised;
//   4. nu = 3, one l-triple (l1, l2, l3) after the other.  The triple's tables
//      (W[q1 q2][q3], the Gaunt entries in three orderings and their offsets)
//      form one tile; the CTA streams the tiles from global memory into two
//      shared-memory buffers with cp.async, fetching tile t+1 while the warps
//      work on tile t, so a tile crosses L2 once per group of atoms rather
//      than once per atom.  Per warp, one pass over lane units (q1, block of qb
//      consecutive q2; the W rows of the block sit in registers) does all of
//        U[m3][q1][q2] = sum_q3 W[q1 q2][q3] A3[m3][q3]
//        Z[m3][q1 q2]  = sum_(m1 m2) G A1[m1][q1] A2[m2][q2]     (Gaunt-sparse)
//        E += sum Z U;  omega3 += W^T Z;  omega1 += G A2 U
//      with U and Z in registers (see nu3_units); omega2 += G A1 U, needed
//      for distinct l's only, reads U from shared memory afterwards.  Where two
//      l's coincide W is symmetrised on the host, the adjoints through the
//      coinciding factors are equal, and one of them is computed and scaled.
//      Each warp adds into its own atom's omega: no reduction across warps
//      and no balancing of triples over warps;
//   5. pair gradients dE_i/dr_ij = u sum_lm sigma_lm Y_lm
//        + (grad_u p - u (u . grad_u p)) / r,  rho = omega R, sigma = omega R',
//      a lane per neighbour with R, R', Y recomputed in registers; written per
//      list slot, to the atom's own row and to the partner's incoming row (slot
//      rev, stamped with the evaluation count).
// Per-atom arrays are stored transposed ([lm][q], q padded to NP = 4k with
// zeros) so that the inner products run over 4-wide vector loads with no index
// division.  The site energy is summed per lane in T and reduced once per atom
// in a fixed order (compensated for float).
#pragma once

#include "mix_launch.h"
#include "tc.cuh"

namespace mixd {

// The Gaunt coefficients ordered by m3 for every l-triple, shared by all
// potentials (AceTileHdr): a copy in the constant memory of each module that
// holds the float expensive kernels, so that the warp-uniform entry reads of
// the nu = 3 pass are constant-bank loads.
static __constant__ GEnt<float> c_gent_f[GAUNT_ENT_CAP];
static __constant__ int c_grow[GAUNT_ROW_CAP];

// this module's copy of the table (host side)
static inline cudaError_t gaunt_upload_module(const void* ent_f, int n_ent, const int* rows, int n_rows) {
    if (n_ent > GAUNT_ENT_CAP || n_rows > GAUNT_ROW_CAP) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbol(c_gent_f, ent_f, (size_t)n_ent * sizeof(GEnt<float>));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_grow, rows, (size_t)n_rows * sizeof(int));
    return e;
}

// entry i of the constant-memory table
__device__ __forceinline__ void gent_c(int i, int& pk, float& g) {
    const GEnt<float> x = c_gent_f[i];
    pk = x.pk;
    g = x.g;
}

template <typename T> struct V4;
template <> struct V4<float> {
    float x, y, z, w;
};
template <> struct V4<double> {
    double x, y, z, w;
};

template <typename T>
__device__ __forceinline__ V4<T> ld4(const T* p);
template <>
__device__ __forceinline__ V4<float> ld4<float>(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
}
template <>
__device__ __forceinline__ V4<double> ld4<double>(const double* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    return {a.x, a.y, b.x, b.y};
}
// one Gaunt entry of a tile in shared memory (one 8- or 16-byte load)
__device__ __forceinline__ void ld_gent(const GEnt<float>* p, int& pk, float& g) {
    const int2 v = *reinterpret_cast<const int2*>(p);
    pk = v.x;
    g = __int_as_float(v.y);
}
__device__ __forceinline__ void ld_gent(const GEnt<double>* p, int& pk, double& g) {
    const int4 v = *reinterpret_cast<const int4*>(p);
    pk = v.x;
    g = __hiloint2double(v.w, v.z);
}

// QB consecutive values from shared memory (QB in {1, 2, 4}, aligned to QB;
// QB = 6, float only, aligned to 2)
template <typename T, int QB>
__device__ __forceinline__ void ld_blk(const T* p, T* out) {
    if constexpr (QB == 6) {
        static_assert(sizeof(T) == 4, "6-wide blocks are float only");
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float2 v = reinterpret_cast<const float2*>(p)[k];
            out[2 * k] = v.x;
            out[2 * k + 1] = v.y;
        }
    } else if constexpr (QB == 4) {
        const V4<T> v = ld4<T>(p);
        out[0] = v.x;
        out[1] = v.y;
        out[2] = v.z;
        out[3] = v.w;
    } else if constexpr (QB == 2) {
        if constexpr (sizeof(T) == 4) {
            const float2 v = *reinterpret_cast<const float2*>(p);
            out[0] = v.x;
            out[1] = v.y;
        } else {
            const double2 v = *reinterpret_cast<const double2*>(p);
            out[0] = v.x;
            out[1] = v.y;
        }
    } else {
        out[0] = p[0];
    }
}

// s += a . b as one chain of four fused multiply-adds
template <typename T>
__device__ __forceinline__ void dot4_acc(T& s, const V4<T>& a, const V4<T>& b) {
    s += a.x * b.x;
    s += a.y * b.y;
    s += a.z * b.z;
    s += a.w * b.w;
}

// Pi[l][m] = d^m P_l / dz^m for 0 <= m <= l <= L (flattened l(l+1)/2 + m),
// C[m] + i S[m] = (x + i y)^m.
template <typename T, int L>
__device__ __forceinline__ void legendre_tables(T x, T y, T z, T* Pi, T* C, T* S) {
    Pi[0] = T(1);
#pragma unroll
    for (int m = 1; m <= L; ++m) Pi[m * (m + 1) / 2 + m] = T(2 * m - 1) * Pi[(m - 1) * m / 2 + m - 1];
#pragma unroll
    for (int m = 0; m < L; ++m) Pi[(m + 1) * (m + 2) / 2 + m] = T(2 * m + 1) * z * Pi[m * (m + 1) / 2 + m];
#pragma unroll
    for (int m = 0; m <= L; ++m)
#pragma unroll
        for (int l = m + 2; l <= L; ++l)
            Pi[l * (l + 1) / 2 + m] = (T(2 * l - 1) * z * Pi[(l - 1) * l / 2 + m] -
                                       T(l + m - 1) * Pi[(l - 2) * (l - 1) / 2 + m]) *
                                      (T(1) / T(l - m));
    C[0] = T(1);
    S[0] = T(0);
#pragma unroll
    for (int m = 1; m <= L; ++m) {
        C[m] = x * C[m - 1] - y * S[m - 1];
        S[m] = x * S[m - 1] + y * C[m - 1];
    }
}

template <typename T, int L>
__device__ __forceinline__ void ylm_eval(T x, T y, T z, const T* __restrict__ K, T* __restrict__ Y) {
    T Pi[(L + 1) * (L + 2) / 2], C[L + 1], S[L + 1];
    legendre_tables<T, L>(x, y, z, Pi, C, S);
#pragma unroll
    for (int l = 0; l <= L; ++l) {
        const int o = l * l + l;
        Y[o] = K[o] * Pi[l * (l + 1) / 2];
#pragma unroll
        for (int m = 1; m <= l; ++m) {
            const T p = Pi[l * (l + 1) / 2 + m];
            Y[o + m] = K[o + m] * p * C[m];
            Y[o - m] = K[o - m] * p * S[m];
        }
    }
}

// R_q(r) = T_q(2r/rc - 1) (1 - (r/rc)^2)^3 and dR_q/dr for q < n; zero for n <= q < NP
template <typename T, int NP>
__device__ __forceinline__ void radial(T r, T invrc, int n, T* R, T* dR) {
    const T sc = T(2) * r * invrc - T(1);
    const T q = r * invrc;
    const T om1 = T(1) - q * q;
    const T fc = om1 * om1 * om1;
    const T dfc = T(-6) * r * invrc * invrc * om1 * om1;
    const T ds = T(2) * invrc;
    T t0 = T(1), t1 = sc, dt0 = T(0), dt1 = T(1);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        T tv, dtv;
        if (p == 0) {
            tv = T(1);
            dtv = T(0);
        } else if (p == 1) {
            tv = sc;
            dtv = T(1);
        } else {
            tv = T(2) * sc * t1 - t0;
            dtv = T(2) * t1 + T(2) * sc * dt1 - dt0;
            t0 = t1;
            t1 = tv;
            dt0 = dt1;
            dt1 = dtv;
        }
        const bool in = p < n;
        R[p] = in ? tv * fc : T(0);
        dR[p] = in ? dtv * ds * fc + tv * dfc : T(0);
    }
}

// uniform cubic B-spline with 16 coefficients on knots (a - 3) h
template <typename T>
__device__ __forceinline__ void spline16(const T* __restrict__ c, T invh, T r, T& v, T& dv) {
    T x = r * invh;
    int q = (int)floor(x);
    q = q < 0 ? 0 : (q > 12 ? 12 : q);
    const T u = x - T(q), w = T(1) - u;
    const T u2 = u * u, u3 = u2 * u;
    const T b0 = w * w * w * T(1.0 / 6.0);
    const T b1 = (T(3) * u3 - T(6) * u2 + T(4)) * T(1.0 / 6.0);
    const T b2 = (T(-3) * u3 + T(3) * u2 + T(3) * u + T(1)) * T(1.0 / 6.0);
    const T b3 = u3 * T(1.0 / 6.0);
    const T d0 = T(-0.5) * w * w;
    const T d1 = T(1.5) * u2 - T(2) * u;
    const T d2 = T(-1.5) * u2 + u + T(0.5);
    const T d3 = T(0.5) * u2;
    v = c[q] * b0 + c[q + 1] * b1 + c[q + 2] * b2 + c[q + 3] * b3;
    dv = (c[q] * d0 + c[q + 1] * d1 + c[q + 2] * d2 + c[q + 3] * d3) * invh;
}

__host__ __device__ constexpr int ace_a16(int b) { return (b + 15) & ~15; }

// Shared memory (byte offsets, used by the host sizing and the kernels): the
// tile buffers, then one region per warp: the atom's density A and adjoint
// omega, and a scratch area holding in turn the density chunk (R and Y of 32
// neighbours), the nu = 3 scratch of a triple (U, kept for omega2, and the
// omega1 partials of the lane units) and, for the pair gradients, the
// compacted unit vectors, distances and list slots.  U is kept only for
// triples of three distinct l's, whose smallest l (the densely contracted
// third factor) is at most L - 2: 2 L - 3 rows m3 at most.
struct AceLay {
    int tile;                  // bytes of one tile buffer (nbuf buffers)
    int o_w, wb;               // first warp region, bytes per warp region
    int o_at, o_om, o_scr;     // offsets inside a warp region
    int o_p1;                  // omega1 partials, inside the scratch area
    int o_slot;                // list slots of the pair-gradient step, inside the scratch area
    int total;
    __host__ __device__ AceLay(int tile_max, int cap, int n, int qb, int L, int NP, int ts, int warps,
                               int nbuf = 2) {
        const int nlm = (L + 1) * (L + 1), D = 2 * L + 1;
        const int du = 2 * L - 3 > 1 ? 2 * L - 3 : 1;
        tile = ace_a16(tile_max);
        o_w = nbuf * tile;
        o_at = 0;                                 // A[lm][q]
        o_om = o_at + ace_a16(nlm * NP * ts);     // omega[lm][q]
        o_scr = o_om + ace_a16(nlm * NP * ts);
        o_p1 = ace_a16(du * n * NP * ts);         // after U[m3][q1][q2]; P1[m1][unit]
        const int nu3 = o_p1 + D * n * (NP / qb) * ts;
        const int chunk = (32 * NP + 32 * nlm) * ts;   // R[32][NP], Y[32][nlm]
        o_slot = ace_a16(4 * cap * ts);           // after [cap][4]: unit vector, r
        const int pairs = o_slot + 4 * cap;
        int scr = nu3 > chunk ? nu3 : chunk;
        scr = scr > pairs ? scr : pairs;
        wb = o_scr + ace_a16(scr);
        total = o_w + warps * wb;
    }
};

// asynchronous global -> shared copies (16 bytes per instruction; completion is
// awaited per thread, then published to the CTA by a barrier)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// the CTA copies tile t (a multiple of 16 bytes, 16-byte aligned) into buf
__device__ __forceinline__ void tile_fetch(const unsigned char* tiles, const int* off, int t, unsigned char* buf) {
    const int b0 = __ldg(off + t), nb = __ldg(off + t + 1) - b0;
    for (int o = (int)threadIdx.x * 16; o < nb; o += (int)blockDim.x * 16) cp_async16(buf + o, tiles + b0 + o);
    cp_async_commit();
}

// Reduce-scatter of C <= 16 per-lane values over the warp.  At lane bit MASK
// (16, 8, 4, 2, 1 in turn) the lanes with the bit set keep the upper half of
// their block (padded with a zero when the count is odd) and send the lower
// half to their partner, the others the reverse, and each adds what it
// receives, so the count halves at every bit; once one value is left the
// remaining bits sum it (both partners add the same two numbers).  The
// additions are in a fixed order.  rs_entry gives the entry a lane ends with.
template <typename T, int C, int MASK>
__device__ __forceinline__ T warp_rs(T* v, int lane) {
    if constexpr (MASK == 0) {
        return v[0];
    } else if constexpr (C == 1) {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], MASK);
        return warp_rs<T, 1, MASK / 2>(v, lane);
    } else {
        constexpr int H = (C + 1) / 2;
        const bool up = (lane & MASK) != 0;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const T hi = i + H < C ? v[i + H] : T(0);
            const T send = up ? v[i] : hi;
            const T keep = up ? hi : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, MASK);
        }
        return warp_rs<T, H, MASK / 2>(v, lane);
    }
}

// The entry of warp_rs<T, C, 16> a lane holds (idx), and whether the lane is
// the one of its group that writes it (a real entry, the lowest lane of the
// lanes that hold the same sum).
template <int C, int MASK>
__device__ __forceinline__ void rs_entry(int lane, int& idx, int& real, bool& writer) {
    if constexpr (MASK == 0) {
        writer = real >= 1;
    } else if constexpr (C == 1) {
        writer = real >= 1 && (lane & (2 * MASK - 1)) == 0;
    } else {
        constexpr int H = (C + 1) / 2;
        if (lane & MASK) {
            idx += H;
            real = real > H ? real - H : 0;
        } else {
            real = real < H ? real : H;
        }
        rs_entry<H, MASK / 2>(lane, idx, real, writer);
    }
}

// nu = 3 of one l-triple for this warp's atom, in one pass over lane units
// (q1, block of QB consecutive q2).  A unit keeps the W rows of its block in
// registers; for each m3 (uniform over the warp, so entry and A3 loads are
// broadcasts) it forms
//   U[m3][q1][q2] = sum_q3 W[q1 q2][q3] A3[m3][q3]           (registers)
//   Z[m3][q1][q2] = sum_(m1 m2) G A1[m1][q1] A2[m2][q2]       (registers, Gaunt-sparse)
// and from them, without storing Z:
//   E      += sum U Z                                          (lane-local)
//   omega3 += W^T Z: the unit's share sum_q2 W[q1 q2][q3] Z[m3][q1 q2] for all q3,
//             summed over the warp by a reduce-scatter;
//   omega1 += G A2 U: per Gaunt entry g sum_q2 A2[m2][q2] U[m3][q1][q2] from the
//             A2 values already loaded for Z, summed over the entries of a run of
//             equal m1 (the entries of one m3 are m1-major) in a register and
//             added to the unit's partial P1[m1][unit] in shared memory; the
//             partials of the units of one q1 are summed after the last m3;
// and, for distinct l's only (omega2 needs it after the pass), stores U.
// All three l's equal: U is not formed (no adjoint needs it) and the energy is
// taken as sum A3 (W^T Z), the same sum reordered.  This is the float64 pass;
// float runs nu3_units_f, the same arithmetic on packed pairs.
template <typename T, int NP, int QB>
__device__ __forceinline__ void nu3_units(const AceTileHdr& h, const T* W, const GEnt<T>* ge3, const int* g3o,
                                          const T* A1, const T* A2, const T* A3, int n, int lane, T* U1, T* P1,
                                          T* o3, T mult3, T& ep) {
    constexpr int nqb = NP / QB;
    const int units = n * nqb;
    const int d3 = 2 * h.l3 + 1;
    const bool withu = h.mode != 3;
    const bool keepu = h.mode == 0;
    int q3o = 0, q3real = NP;           // the omega3 entry this lane receives
    bool q3w = false;
    rs_entry<NP, 16>(lane, q3o, q3real, q3w);
    for (int u0 = 0; u0 < units; u0 += 32) {
        const int u = u0 + lane;
        const bool uv = u < units;
        const int uu = uv ? u : 0;
        const int q1 = uu / nqb;
        const int q2 = (uu - q1 * nqb) * QB;
        const T* A1q = A1 + q1;
        const T* A2q = A2 + q2;
        T w[QB][NP];
#pragma unroll
        for (int r = 0; r < QB; ++r) {
            const bool ok = uv && q2 + r < n;
            const T* wr = W + (q1 * n + (ok ? q2 + r : 0)) * NP;
#pragma unroll
            for (int p = 0; p < NP; p += 4) {
                V4<T> v = ld4<T>(wr + p);
                if (!ok) v = V4<T>{T(0), T(0), T(0), T(0)};
                w[r][p] = v.x;
                w[r][p + 1] = v.y;
                w[r][p + 2] = v.z;
                w[r][p + 3] = v.w;
            }
        }
        for (int m3 = 0; m3 < d3; ++m3) {
            T uo[QB], z[QB];
#pragma unroll
            for (int r = 0; r < QB; ++r) {
                uo[r] = T(0);
                z[r] = T(0);
            }
            if (withu) {
                T a[NP];
#pragma unroll
                for (int p = 0; p < NP; p += 4) {
                    const V4<T> v = ld4<T>(A3 + m3 * NP + p);
                    a[p] = v.x;
                    a[p + 1] = v.y;
                    a[p + 2] = v.z;
                    a[p + 3] = v.w;
                }
#pragma unroll
                for (int r = 0; r < QB; ++r) {
                    T s = T(0);
#pragma unroll
                    for (int p = 0; p < NP; ++p) s += w[r][p] * a[p];
                    uo[r] = s;
                }
            }
            const int e1 = g3o[m3 + 1];
            T c1 = T(0);
            for (int e = g3o[m3]; e < e1; ++e) {
                int pk;
                T g;
                ld_gent(ge3 + e, pk, g);
                const T ga = g * A1q[(pk & 255) * NP];
                T a2[QB];
                ld_blk<T, QB>(A2q + ((pk >> 8) & 255) * NP, a2);
#pragma unroll
                for (int r = 0; r < QB; ++r) z[r] += ga * a2[r];
                if (withu) {
                    T dd = T(0);
#pragma unroll
                    for (int r = 0; r < QB; ++r) dd += a2[r] * uo[r];
                    c1 += g * dd;
                    if (pk & GE_RUN_END) {   // uniform over the warp
                        if (uv) P1[(pk & 255) * units + u] += c1;
                        c1 = T(0);
                    }
                }
            }
            if (withu) {
#pragma unroll
                for (int r = 0; r < QB; ++r) ep += uo[r] * z[r];
                if (keepu && uv) {
#pragma unroll
                    for (int r = 0; r < QB; ++r) U1[(m3 * n + q1) * NP + q2 + r] = uo[r];
                }
            }
            // omega3 row m3
            T pv[16];
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                T s = T(0);
#pragma unroll
                for (int r = 0; r < QB; ++r) s += w[r][q] * z[r];
                pv[q] = s;
            }
            const T s3 = warp_rs<T, NP, 16>(pv, lane);
            if (q3w && q3o < n) {
                o3[m3 * NP + q3o] += mult3 * s3;
                if (!withu) ep += A3[m3 * NP + q3o] * s3;
            }
        }
    }
}

// QB / 2 pairs of consecutive floats from shared memory (QB in {2, 4, 6},
// 8-byte aligned; QB = 4 16-byte aligned)
template <int QB>
__device__ __forceinline__ void ld_pairs(const float* p, float2* out) {
    if constexpr (QB == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        out[0] = make_float2(v.x, v.y);
        out[1] = make_float2(v.z, v.w);
    } else {
#pragma unroll
        for (int k = 0; k < QB / 2; ++k) out[k] = reinterpret_cast<const float2*>(p)[k];
    }
}

// The float unit pass: the arithmetic of nu3_units on packed pairs
// (__ffma2_rn: two float fused multiply-adds an instruction), which halves the
// instructions of its dense products.  W rows are held as pairs of
// consecutive q3: U = W A3 runs as two interleaved sums (even and odd q3)
// added at the end, and the omega3 partials pair consecutive q3 against a
// broadcast Z (the same order of additions as the float64 pass).  Z, the
// omega1 dot product and the energy pair consecutive q2.
//
// TCM != 0 (the tensor-core readout): omega3 and the energy are not formed
// here.  Z goes, rounded to bf16 (TCM == 2: also its remainder, the lo part),
// into this atom's rows of the MMA operand tile (row m3, column q1 n + q2 of
// the K-major layout of tc.cuh), from which the tensor cores form V = Z W
// (omega3 = mult3 V, E = sum A3 V) after the pass.
template <int NP, int QB, int TCM>
__device__ __forceinline__ void nu3_units_f(const AceTileHdr& h, const float* W, const float* A1, const float* A2,
                                            const float* A3, int n, int lane, float* U1, float* P1, float* o3,
                                            float mult3, float& ep, unsigned char* zhi, unsigned char* zlo,
                                            int zsbo) {
    static_assert(QB % 2 == 0 && NP % 4 == 0, "the float pass works on pairs");
    constexpr int nqb = NP / QB, NH = NP / 2, QH = QB / 2;
    const int units = n * nqb;
    const int d3 = 2 * h.l3 + 1, rb = h.cg;
    const bool withu = h.mode != 3;
    const bool keepu = h.mode == 0;
    int q3o = 0, q3real = NP;
    bool q3w = false;
    rs_entry<NP, 16>(lane, q3o, q3real, q3w);
    float2 e2 = make_float2(0.f, 0.f);
    for (int u0 = 0; u0 < units; u0 += 32) {
        const int u = u0 + lane;
        const bool uv = u < units;
        const int uu = uv ? u : 0;
        const int q1 = uu / nqb;
        const int q2 = (uu - q1 * nqb) * QB;
        const float* A1q = A1 + q1;
        const float* A2q = A2 + q2;
        int zcol[TCM != 0 ? QH : 1];   // column part of the operand offset of each pair
#pragma unroll
        for (int k = 0; k < (TCM != 0 ? QH : 1); ++k) zcol[k] = tc_off(0, q1 * n + q2 + 2 * k, TC_LBO_A, 0);
        int e = c_grow[rb], pkn;   // the entries of all m3 rows follow each other
        float gn;
        gent_c(e, pkn, gn);
        float2 w[QB][NH];
#pragma unroll
        for (int r = 0; r < QB; ++r) {
            const bool ok = uv && q2 + r < n;
            const float* wr = W + (q1 * n + (ok ? q2 + r : 0)) * NP;
#pragma unroll
            for (int p = 0; p < NP; p += 4) {
                float4 v = *reinterpret_cast<const float4*>(wr + p);
                if (!ok) v = make_float4(0.f, 0.f, 0.f, 0.f);
                w[r][p / 2] = make_float2(v.x, v.y);
                w[r][p / 2 + 1] = make_float2(v.z, v.w);
            }
        }
        for (int m3 = 0; m3 < d3; ++m3) {
            float2 uo[QH], z[QH];
#pragma unroll
            for (int k = 0; k < QH; ++k) {
                uo[k] = make_float2(0.f, 0.f);
                z[k] = make_float2(0.f, 0.f);
            }
            if (withu) {
                float2 a[NH];
#pragma unroll
                for (int p = 0; p < NP; p += 4) {
                    const float4 v = *reinterpret_cast<const float4*>(A3 + m3 * NP + p);
                    a[p / 2] = make_float2(v.x, v.y);
                    a[p / 2 + 1] = make_float2(v.z, v.w);
                }
#pragma unroll
                for (int r = 0; r < QB; ++r) {
                    float2 s = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < NH; ++j) s = __ffma2_rn(w[r][j], a[j], s);
                    if (r & 1) uo[r / 2].y = s.x + s.y;
                    else uo[r / 2].x = s.x + s.y;
                }
            }
            const int e1 = c_grow[rb + m3 + 1];
            float2 c1 = make_float2(0.f, 0.f);
            for (; e < e1; ++e) {
                const int pk = pkn;
                const float g = gn;
                // the next entry (of this row, the next row or triple, or the
                // zero entry after the last) is in flight while this one works
                gent_c(e + 1, pkn, gn);
                const float ga = g * A1q[(pk & 255) * NP];
                const float2 ga2 = make_float2(ga, ga);
                float2 a2[QH];
                ld_pairs<QB>(A2q + ((pk >> 8) & 255) * NP, a2);
#pragma unroll
                for (int k = 0; k < QH; ++k) z[k] = __ffma2_rn(ga2, a2[k], z[k]);
                if (withu) {
                    float2 dd = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < QH; ++k) dd = __ffma2_rn(a2[k], uo[k], dd);
                    c1 = __ffma2_rn(make_float2(g, g), dd, c1);
                    if (pk & GE_RUN_END) {   // uniform over the warp
                        if (uv) P1[(pk & 255) * units + u] += c1.x + c1.y;
                        c1 = make_float2(0.f, 0.f);
                    }
                }
            }
            if (withu) {
                if constexpr (TCM == 0) {
#pragma unroll
                    for (int k = 0; k < QH; ++k) e2 = __ffma2_rn(uo[k], z[k], e2);
                }
                if (keepu && uv) {
#pragma unroll
                    for (int k = 0; k < QH; ++k)
                        *reinterpret_cast<float2*>(U1 + (m3 * n + q1) * NP + q2 + 2 * k) = uo[k];
                }
            }
            if constexpr (TCM != 0) {
                if (uv && (n & 1) == 0) {
                    // even n: columns q1 n + q2 + r, r even, are even, so each
                    // pair lies in one 4-byte word of a core-matrix row; the
                    // row part of the offset is the m3 one, the column part the unit's
                    const int orow = tc_off(m3, 0, TC_LBO_A, zsbo);
#pragma unroll
                    for (int k = 0; k < QH; ++k) {
                        if (q2 + 2 * k < n) {
                            const int o = orow + zcol[k];
                            const __nv_bfloat162 hi = __float22bfloat162_rn(z[k]);
                            *reinterpret_cast<__nv_bfloat162*>(zhi + o) = hi;
                            if constexpr (TCM == 2) {
                                const float2 hf = __bfloat1622float2(hi);
                                *reinterpret_cast<__nv_bfloat162*>(zlo + o) =
                                    __float22bfloat162_rn(make_float2(z[k].x - hf.x, z[k].y - hf.y));
                            }
                        }
                    }
                } else if (uv) {
#pragma unroll
                    for (int r = 0; r < QB; ++r) {
                        if (q2 + r < n) {
                            const float zr = (r & 1) ? z[r / 2].y : z[r / 2].x;
                            const int o = tc_off(m3, q1 * n + q2 + r, TC_LBO_A, zsbo);
                            const __nv_bfloat16 hi = __float2bfloat16_rn(zr);
                            *reinterpret_cast<__nv_bfloat16*>(zhi + o) = hi;
                            if constexpr (TCM == 2)
                                *reinterpret_cast<__nv_bfloat16*>(zlo + o) =
                                    __float2bfloat16_rn(zr - __bfloat162float(hi));
                        }
                    }
                }
            } else {
                // omega3 row m3
                float pv[16];
#pragma unroll
                for (int j = 0; j < NH; ++j) {
                    float2 s = make_float2(0.f, 0.f);
#pragma unroll
                    for (int r = 0; r < QB; ++r) {
                        const float zr = (r & 1) ? z[r / 2].y : z[r / 2].x;
                        s = __ffma2_rn(w[r][j], make_float2(zr, zr), s);
                    }
                    pv[2 * j] = s.x;
                    pv[2 * j + 1] = s.y;
                }
                const float s3 = warp_rs<float, NP, 16>(pv, lane);
                if (q3w && q3o < n) {
                    o3[m3 * NP + q3o] += mult3 * s3;
                    if (!withu) ep += A3[m3 * NP + q3o] * s3;
                }
            }
        }
    }
    ep += e2.x + e2.y;
}

// One l-triple for this warp's atom, from the tile in shared memory.
// PART 1: the unit pass; PART 2: omega1 from the unit partials and omega2;
// PART 3: both.
template <typename T, int NP, int TCM = 0, int PART = 3>
__device__ __forceinline__ void nu3_tile(const unsigned char* tile, const AceTab<T>& tab, const T* At, T* om,
                                         T* U1, T* P1, int lane, T& ep, unsigned char* zhi = nullptr,
                                         unsigned char* zlo = nullptr, int zsbo = 0) {
    constexpr int QM = 4;     // largest power-of-two q2 block of a lane unit
    const AceTileHdr h = *reinterpret_cast<const AceTileHdr*>(tile);
    const T* W = reinterpret_cast<const T*>(tile + sizeof(AceTileHdr));
    const GEnt<T>* ge = reinterpret_cast<const GEnt<T>*>(tile + h.o_ge);   // ordered by m2
    const int* g2o = reinterpret_cast<const int*>(tile + h.o_go);
    const int n = tab.n;
    const int d1 = 2 * h.l1 + 1, d2 = 2 * h.l2 + 1, d3 = 2 * h.l3 + 1;
    // coinciding l's (W symmetrised on the host): scale instead of recompute
    const T mult1 = h.mode == 1 ? T(2) : T(1);
    const T mult3 = h.mode == 3 ? T(3) : (h.mode == 2 ? T(2) : T(1));
    const T* A1 = At + h.l1 * h.l1 * NP;
    const T* A2 = At + h.l2 * h.l2 * NP;
    const T* A3 = At + h.l3 * h.l3 * NP;
    T* o3 = om + h.l3 * h.l3 * NP;
    const int qb = tab.qb;
    if constexpr ((PART & 1) != 0) {
        if constexpr (sizeof(T) == 4) {
            if constexpr (NP == 12) {
                // n = 11 or 12: 6-wide blocks keep the units within one warp pass
                if (qb == 6)
                    nu3_units_f<NP, 6, TCM>(h, W, A1, A2, A3, n, lane, U1, P1, o3, mult3, ep, zhi, zlo,
                                            zsbo);
            }
            if (qb == QM)
                nu3_units_f<NP, QM, TCM>(h, W, A1, A2, A3, n, lane, U1, P1, o3, mult3, ep, zhi, zlo, zsbo);
            else if (qb == QM / 2)
                nu3_units_f<NP, QM / 2, TCM>(h, W, A1, A2, A3, n, lane, U1, P1, o3, mult3, ep, zhi, zlo,
                                             zsbo);
        } else {
            static_assert(sizeof(T) == 4 || TCM == 0, "the tensor-core readout is float only");
            // float64 reads the ordering by m3 from its tile
            const GEnt<T>* ge3 = reinterpret_cast<const GEnt<T>*>(tile + h.o_ge3);
            const int* g3o = reinterpret_cast<const int*>(tile + h.o_go3);
            if (qb == QM)
                nu3_units<T, NP, QM>(h, W, ge3, g3o, A1, A2, A3, n, lane, U1, P1, o3, mult3, ep);
            else
                nu3_units<T, NP, QM / 2>(h, W, ge3, g3o, A1, A2, A3, n, lane, U1, P1, o3, mult3, ep);
        }
        __syncwarp();
    }
    if constexpr ((PART & 2) == 0) return;
    // omega1 (equal to omega3 when all three l's coincide): sum the unit
    // partials of each (m1, q1) and clear them for the next triple
    if (h.mode != 3) {
        const int nqb = NP / qb, units = n * nqb;
        T* o1 = om + h.l1 * h.l1 * NP;
        for (int o = lane; o < n * d1; o += 32) {
            const int m1 = o / n, q1 = o - m1 * n;
            T* pr = P1 + m1 * units + q1 * nqb;
            T s = T(0);
            for (int b = 0; b < nqb; ++b) {
                s += pr[b];
                pr[b] = T(0);
            }
            o1[m1 * NP + q1] += mult1 * s;
        }
    }
    // omega2 += G A1 U, needed only when the three l's are distinct (otherwise
    // it equals omega1 or omega3, already scaled in); a lane per (m2, 4 q2)
    if (h.mode == 0) {
        constexpr int NB4 = NP / 4;
        T* o2 = om + h.l2 * h.l2 * NP;
        for (int u = lane; u < d2 * NB4; u += 32) {
            const int m2 = u / NB4, q2 = (u - m2 * NB4) * 4;
            T c0 = T(0), c1 = T(0), c2 = T(0), c3 = T(0);
            for (int e = g2o[m2]; e < g2o[m2 + 1]; ++e) {
                int pk;
                T gv;
                ld_gent(ge + e, pk, gv);
                const T* ar = A1 + (pk & 255) * NP;
                const T* ur = U1 + (pk >> 8) * n * NP + q2;
                if constexpr (sizeof(T) == 4) {
                    // the same fused multiply-adds, two an instruction
                    float2 s01 = make_float2(0.f, 0.f), s23 = make_float2(0.f, 0.f);
                    for (int q1 = 0; q1 < n; ++q1) {
                        const float av = ar[q1];
                        const float2 a2 = make_float2(av, av);
                        const V4<T> u4 = ld4<T>(ur + q1 * NP);
                        s01 = __ffma2_rn(a2, make_float2(u4.x, u4.y), s01);
                        s23 = __ffma2_rn(a2, make_float2(u4.z, u4.w), s23);
                    }
                    const float2 g2 = make_float2(gv, gv);
                    const float2 c01 = __ffma2_rn(g2, s01, make_float2(c0, c1));
                    const float2 c23 = __ffma2_rn(g2, s23, make_float2(c2, c3));
                    c0 = c01.x;
                    c1 = c01.y;
                    c2 = c23.x;
                    c3 = c23.y;
                } else {
                    T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
                    for (int q1 = 0; q1 < n; ++q1) {
                        const T av = ar[q1];
                        const V4<T> u4 = ld4<T>(ur + q1 * NP);
                        s0 += av * u4.x;
                        s1 += av * u4.y;
                        s2 += av * u4.z;
                        s3 += av * u4.w;
                    }
                    c0 += gv * s0;
                    c1 += gv * s1;
                    c2 += gv * s2;
                    c3 += gv * s3;
                }
            }
            T* orow = o2 + m2 * NP + q2;
            orow[0] += c0;
            if (q2 + 1 < n) orow[1] += c1;
            if (q2 + 2 < n) orow[2] += c2;
            if (q2 + 3 < n) orow[3] += c3;
        }
    }
    __syncwarp();
}

// State of the tensor-core readout of one thread (TCM != 0).
struct TcState {
    unsigned char* zhi;   // A operand: Z rows of the CTA's atoms (bf16)
    unsigned char* zlo;   // their remainders (hi/lo split) or null
    uint32_t tmem;        // accumulator V (128 lanes x 16 columns f32)
    uint32_t bar;         // mbarrier the MMAs of a triple arrive on
    uint32_t phase;       // parity of its next completion
    int kp, sbo;          // K (n^2 padded to 16), A row-group stride in bytes
    int nbuf;             // tile buffers: 2 (the next tile streams in during this one) or 1
    int abort;            // a completion wait ran out: no further waits
};

// polls of an mbarrier before a readout MMA is declared lost (status bit
// ST_TC_TIMEOUT, reported as MIX_ETIMEOUT)
constexpr int TC_WAIT_POLLS = 1 << 20;

// One group of atoms a0 .. a0 + WN - 1 of the system's expensive list (those
// below nexp), warp w on atom a0 + w; every thread of the CTA calls it.
// TCM != 0 (float only): the nu = 3 readout V = Z W runs on the tensor cores
// for the CTA's TC_ACE_WARPS atoms at once (16 rows (atom, m3) per atom).
template <typename T, int L, int NP, int TCM = 0>
__device__ __forceinline__ void ace_group(const Dev& d, const AceTab<T>& tab, int a0, int nexp, unsigned char* smem,
                                          TcState* tc = nullptr, int wn = ACE_GROUP) {
    const int WN = TCM != 0 ? TC_ACE_WARPS : wn;   // warps (atoms) of the CTA
    constexpr int NLM = (L + 1) * (L + 1);
    constexpr int D = 2 * L + 1;
    constexpr int NQ4 = NP / 4;
    constexpr int NU = NLM * NQ4;               // density units (lm, 4 q)
    constexpr int NUL = (NU + 31) / 32;
    using V = typename Vec4<T>::type;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = tab.n, cap = d.cap, ntau = tab.ntau;
    const AceLay lay(tab.tile_max, cap, n, tab.qb, L, NP, (int)sizeof(T), WN, TCM != 0 ? tc->nbuf : 2);
    // the first tile lands while the warps run steps 1-3
    if (ntau > 0) tile_fetch(tab.tiles, tab.tile_off, 0, smem);

    unsigned char* wreg = smem + lay.o_w + warp * lay.wb;
    T* At = reinterpret_cast<T*>(wreg + lay.o_at);
    T* om = reinterpret_cast<T*>(wreg + lay.o_om);
    T* scr = reinterpret_cast<T*>(wreg + lay.o_scr);
    T* cR = scr;                 // density chunk
    T* cY = scr + 32 * NP;
    T* U1 = scr;                 // nu = 3
    T* P1 = reinterpret_cast<T*>(wreg + lay.o_scr + lay.o_p1);
    T* su = scr;                 // pair gradients
    int* slot = reinterpret_cast<int*>(wreg + lay.o_scr + lay.o_slot);

    const int a = a0 + warp;
    const bool has = a < nexp;
    const int i = has ? d.act_e[a] : 0;
    V* GE = reinterpret_cast<V*>(d.ge);
    V* GIN = reinterpret_cast<V*>(d.ge_in);
    const int stamp = d.status[SW_EPOCH];
    const T rc = (T)tab.rc;
    const T invrc = T(1) / rc;
    const T invh = T(13) / rc;
    const int* row = d.nbr + (int64_t)i * cap;
    const int* rvr = d.rev + (int64_t)i * cap;
    V* grow = GE + (int64_t)i * cap;
    T ep = T(0);
    const T rc2 = (T)d.rce2;
    const unsigned lt = (1u << lane) - 1u;
    const int m = has ? d.nnb[i] : 0;

    if (has) {
        // 1-2. density, 32 list slots at a time: the slots inside the cutoff
        // are compacted in slot order (ballot) into the chunk, where each lane
        // then accumulates its (lm, 4 q) outputs over them
        const PairFrame<T> pf(d, i);
        T acc[NUL][4];
#pragma unroll
        for (int j = 0; j < NUL; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = T(0);
        for (int b0 = 0; b0 < m; b0 += 32) {
            const int s = b0 + lane;
            bool ok = false;
            T dv[3] = {T(0), T(0), T(0)}, r2 = T(0);
            if (s < m) {
                pf.vec(d, row[s], dv, r2);
                ok = r2 < rc2;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            const int kc = __popc(bal);
            if (ok) {
                const int k = __popc(bal & lt);
                const T r = sqrt(r2), ir = T(1) / r;
                T R[NP], dR[NP];
                radial<T, NP>(r, invrc, n, R, dR);
#pragma unroll
                for (int p = 0; p < NP; ++p) cR[k * NP + p] = R[p];
                ylm_eval<T, L>(dv[0] * ir, dv[1] * ir, dv[2] * ir, tab.ylmk, cY + k * NLM);
                if (tab.has_pair) {
                    T v, dvv;
                    spline16<T>(tab.pair, invh, r, v, dvv);
                    ep += T(0.5) * v;
                }
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < NUL; ++j) {
                const int u = lane + 32 * j;
                if (u < NU) {
                    const int lm = u / NQ4, q4 = (u - lm * NQ4) * 4;
                    for (int kl = 0; kl < kc; ++kl) {
                        const T y = cY[kl * NLM + lm];
                        const V4<T> r4 = ld4<T>(cR + kl * NP + q4);
                        if constexpr (sizeof(T) == 4) {
                            const float2 yy = make_float2(y, y);
                            const float2 lo = __ffma2_rn(yy, make_float2(r4.x, r4.y), make_float2(acc[j][0], acc[j][1]));
                            const float2 hi = __ffma2_rn(yy, make_float2(r4.z, r4.w), make_float2(acc[j][2], acc[j][3]));
                            acc[j][0] = lo.x;
                            acc[j][1] = lo.y;
                            acc[j][2] = hi.x;
                            acc[j][3] = hi.y;
                        } else {
                            acc[j][0] += y * r4.x;
                            acc[j][1] += y * r4.y;
                            acc[j][2] += y * r4.z;
                            acc[j][3] += y * r4.w;
                        }
                    }
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int j = 0; j < NUL; ++j) {
            const int u = lane + 32 * j;
            if (u < NU) {
                const int lm = u / NQ4, q4 = (u - lm * NQ4) * 4;
#pragma unroll
                for (int c = 0; c < 4; ++c) At[lm * NP + q4 + c] = acc[j][c];
            }
        }
        __syncwarp();

        // 3. nu = 1 and nu = 2; initialises omega
        for (int o = lane; o < NLM * NP; o += 32) {
            const int lm = o / NP, q = o - lm * NP;
            T val = T(0);
            if (q < n) {
                int l = 0;
                while ((l + 1) * (l + 1) <= lm) ++l;
                if (tab.nu >= 2) {
                    // even and odd q2 in two chains; unrolled over the padded
                    // count so that the row's coefficient loads are all in flight
                    const T* S2 = tab.S2 + ((int64_t)l * n + q) * n;
                    const T* Ar = At + lm * NP;
                    T v2 = T(0);
#pragma unroll
                    for (int q2 = 0; q2 < NP; ++q2) {
                        if (q2 < n) {
                            if (q2 & 1) v2 += __ldg(S2 + q2) * Ar[q2];
                            else val += __ldg(S2 + q2) * Ar[q2];
                        }
                    }
                    val += v2;
                }
                const T av = At[o];
                ep += T(0.5) * av * val;
                if (lm == 0) {
                    const T c = __ldg(tab.c1 + q);
                    ep += c * av;
                    val += c;
                }
            }
            om[o] = val;
        }
        // the omega1 partials start at zero (each triple clears what it used)
        if (ntau > 0)
            for (int o = lane; o < D * n * (NP / tab.qb); o += 32) P1[o] = T(0);
        __syncwarp();
    }

    // 4. nu = 3, tile by tile (every thread takes part in the copies and barriers)
    if constexpr (TCM == 0) {
        for (int t = 0; t < ntau; ++t) {
            cp_async_wait_all();
            __syncthreads();   // tile t visible; every warp is done with the other buffer
            if (t + 1 < ntau) tile_fetch(tab.tiles, tab.tile_off, t + 1, smem + ((t + 1) & 1) * lay.tile);
            if (has) nu3_tile<T, NP>(smem + (t & 1) * lay.tile, tab, At, om, U1, P1, lane, ep);
        }
    } else {
        // Per triple: the warps write Z rows (and form U, omega1, omega2 as in
        // the CUDA-core pass); one thread issues V = Z W over K = kp (one MMA
        // per 16 columns, three with the hi/lo split: Zhi Whi + Zlo Whi +
        // Zhi Wlo); the warps take omega1 and omega2 meanwhile, then wait for
        // the MMAs and read their own rows of V: omega3 += mult3 V,
        // E += sum A3 V (lane-local, summed with the atom's other terms).
        // this warp's 16 rows of the MMA tile, placed so that their
        // accumulator rows lie in the TMEM lanes 32 (w % 4) .. + 31 the warp may
        // read: M = 128 puts row i in lane i, M = 64 rows 16 w .. 16 w + 15 in
        // lanes 32 w .. 32 w + 15
        const int slot_w = TC_M == 128 ? 2 * (warp & 3) + (warp >> 2) : warp;
        unsigned char* zh = tc->zhi + 2 * slot_w * tc->sbo;
        unsigned char* zl = TCM == 2 ? tc->zlo + 2 * slot_w * tc->sbo : nullptr;
        const bool own = TC_M == 128 ? (lane >> 4) == (warp >> 2) : lane < 16;   // TMEM lane 32 (w % 4) + lane
        const int m3r = lane & 15;
        const uint32_t idesc = tc_idesc_bf16(TC_M, 16);
        const int kp = tc->kp, sbo_b = (kp / 8) * TC_LBO_B;
        for (int t = 0; t < ntau; ++t) {
            unsigned char* tile = smem + (tc->nbuf == 2 ? (t & 1) : 0) * lay.tile;
            if (tc->nbuf == 1 && t > 0) {
                __syncthreads();   // every warp is done with tile t - 1
                tile_fetch(tab.tiles, tab.tile_off, t, tile);
            }
            cp_async_wait_all();
            fence_async_smem();    // the coefficient operand this thread copied, visible to the tensor cores
            __syncthreads();       // tile t visible; every warp is done with the other buffer and with V of t - 1
            if (tc->nbuf == 2 && t + 1 < ntau)
                tile_fetch(tab.tiles, tab.tile_off, t + 1, smem + ((t + 1) & 1) * lay.tile);
            const AceTileHdr h = *reinterpret_cast<const AceTileHdr*>(tile);
            if (has) nu3_tile<T, NP, TCM, 1>(tile, tab, At, om, U1, P1, lane, ep, zh, zl, tc->sbo);
            fence_async_smem();    // this thread's Z rows, visible to the tensor cores
            __syncthreads();
            if (tid == 0 && !tc->abort) {
                tc_fence_after();
                const unsigned char* wb = tile + h.o_wb;
                for (int s = 0; s < kp / 16; ++s) {
                    const uint64_t ah = tc_desc(smem_u32(tc->zhi + s * 2 * TC_LBO_A), TC_LBO_A, tc->sbo);
                    const uint64_t bh = tc_desc(smem_u32(wb + s * 2 * TC_LBO_B), TC_LBO_B, sbo_b);
                    tc_mma_bf16(tc->tmem, ah, bh, idesc, s > 0 ? 1u : 0u);
                    if constexpr (TCM == 2) {
                        const uint64_t al = tc_desc(smem_u32(tc->zlo + s * 2 * TC_LBO_A), TC_LBO_A, tc->sbo);
                        const uint64_t bl = tc_desc(smem_u32(wb + 2 * sbo_b + s * 2 * TC_LBO_B), TC_LBO_B, sbo_b);
                        tc_mma_bf16(tc->tmem, al, bh, idesc, 1u);
                        tc_mma_bf16(tc->tmem, ah, bl, idesc, 1u);
                    }
                }
                tc_commit(tc->bar);
            }
            if (has) nu3_tile<T, NP, TCM, 2>(tile, tab, At, om, U1, P1, lane, ep, zh, zl, tc->sbo);
            if (!tc->abort && !mbar_wait(tc->bar, tc->phase, TC_WAIT_POLLS)) {
                tc->abort = 1;
                set_status(d.status, ST_TC_TIMEOUT);
            }
            tc->phase ^= 1u;
            tc_fence_after();
            float v[16];
            tmem_ld16(tc->tmem + ((uint32_t)(32 * (warp & 3)) << 16), v);
            if (has && own && m3r < 2 * h.l3 + 1 && !tc->abort) {
                const T mult3 = h.mode == 3 ? T(3) : (h.mode == 2 ? T(2) : T(1));
                T* o3 = om + (h.l3 * h.l3 + m3r) * NP;
                const T* a3 = At + (h.l3 * h.l3 + m3r) * NP;
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    if (q < n) {
                        o3[q] += mult3 * (T)v[q];
                        ep += a3[q] * (T)v[q];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
        }
    }
    if (ntau > 0) __syncthreads();   // both buffers free for the next group's first tile

    if (has) {
        // 5. pair gradients: the neighbours inside the cutoff compacted again
        // in slot order (unit vector, r and list slot into the scratch area;
        // the slots outside get zero rows), then a lane per neighbour
        int nb = 0;
        {
            const PairFrame<T> pf(d, i);
            for (int b0 = 0; b0 < m; b0 += 32) {
                const int s = b0 + lane;
                bool ok = false;
                T dv[3] = {T(0), T(0), T(0)}, r2 = T(0);
                if (s < m) {
                    pf.vec(d, row[s], dv, r2);
                    ok = r2 < rc2;
                    if (!ok) {
                        V z;
                        z.x = z.y = z.z = z.w = T(0);
                        grow[s] = z;
                        z.w = stamp_as(T(0), stamp);
                        GIN[(int64_t)row[s] * cap + rvr[s]] = z;   // the partner's incoming row
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                if (ok) {
                    const int k = nb + __popc(bal & lt);
                    const T r = sqrt(r2), ir = T(1) / r;
                    slot[k] = s;
                    su[4 * k + 0] = dv[0] * ir;
                    su[4 * k + 1] = dv[1] * ir;
                    su[4 * k + 2] = dv[2] * ir;
                    su[4 * k + 3] = r;
                }
                nb += __popc(bal);
            }
            __syncwarp();
        }
        const T* K = tab.ylmk;
        for (int k = lane; k < nb; k += 32) {
            const T x = su[4 * k], y = su[4 * k + 1], z = su[4 * k + 2], r = su[4 * k + 3];
            T R[NP], dR[NP];
            radial<T, NP>(r, invrc, n, R, dR);
            T Pi[(L + 1) * (L + 2) / 2], C[L + 1], S[L + 1];
            legendre_tables<T, L>(x, y, z, Pi, C, S);
            T sy = T(0), Gx = T(0), Gy = T(0), Gz = T(0);
#pragma unroll
            for (int l = 0; l <= L; ++l) {
                const int pl = l * (l + 1) / 2;
#pragma unroll
                for (int mm = -l; mm <= l; ++mm) {
                    const int lm = l * l + l + mm;
                    const T* orow = om + lm * NP;
                    T rho = T(0), sig = T(0);
                    if constexpr (sizeof(T) == 4) {
                        // even and odd q in packed pairs, added at the end
                        float2 rr = make_float2(0.f, 0.f), ss = make_float2(0.f, 0.f);
#pragma unroll
                        for (int p = 0; p < NP; p += 4) {
                            const V4<T> o4 = ld4<T>(orow + p);
                            const float2 olo = make_float2(o4.x, o4.y), ohi = make_float2(o4.z, o4.w);
                            rr = __ffma2_rn(olo, make_float2(R[p], R[p + 1]), rr);
                            rr = __ffma2_rn(ohi, make_float2(R[p + 2], R[p + 3]), rr);
                            ss = __ffma2_rn(olo, make_float2(dR[p], dR[p + 1]), ss);
                            ss = __ffma2_rn(ohi, make_float2(dR[p + 2], dR[p + 3]), ss);
                        }
                        rho = rr.x + rr.y;
                        sig = ss.x + ss.y;
                    } else {
#pragma unroll
                        for (int p = 0; p < NP; p += 4) {
                            const V4<T> o4 = ld4<T>(orow + p);
                            rho += o4.x * R[p] + o4.y * R[p + 1] + o4.z * R[p + 2] + o4.w * R[p + 3];
                            sig += o4.x * dR[p] + o4.y * dR[p + 1] + o4.z * dR[p + 2] + o4.w * dR[p + 3];
                        }
                    }
                    const int mu = mm < 0 ? -mm : mm;
                    const T kk = __ldg(K + lm);
                    const T p = Pi[pl + mu];
                    const T pz = (mu < l) ? Pi[pl + mu + 1] : T(0);
                    T yv, gx, gy, gz;
                    if (mm == 0) {
                        yv = kk * p;
                        gx = T(0);
                        gy = T(0);
                        gz = kk * pz;
                    } else if (mm > 0) {
                        // p_{l,m} = K Pi C_m
                        yv = kk * p * C[mu];
                        gx = kk * p * T(mu) * C[mu - 1];
                        gy = -kk * p * T(mu) * S[mu - 1];
                        gz = kk * pz * C[mu];
                    } else {
                        // p_{l,-m} = K Pi S_m
                        yv = kk * p * S[mu];
                        gx = kk * p * T(mu) * S[mu - 1];
                        gy = kk * p * T(mu) * C[mu - 1];
                        gz = kk * pz * S[mu];
                    }
                    sy += sig * yv;
                    Gx += rho * gx;
                    Gy += rho * gy;
                    Gz += rho * gz;
                }
            }
            const T ug = x * Gx + y * Gy + z * Gz;
            const T ir = T(1) / r;
            T g[3] = {sy * x + (Gx - x * ug) * ir, sy * y + (Gy - y * ug) * ir, sy * z + (Gz - z * ug) * ir};
            if (tab.has_pair) {
                T v, dv;
                spline16<T>(tab.pair, invh, r, v, dv);
                const T hp = T(0.5) * dv;
                g[0] += hp * x;
                g[1] += hp * y;
                g[2] += hp * z;
            }
            V gv;
            gv.x = g[0];
            gv.y = g[1];
            gv.z = g[2];
            gv.w = T(0);
            const int sl = slot[k];
            grow[sl] = gv;
            gv.w = stamp_as(T(0), stamp);
            GIN[(int64_t)row[sl] * cap + rvr[sl]] = gv;
        }

        // site energy: fixed reduction order, compensated for float
        const auto e = warp_sum(ep);
        if (lane == 0) {
            if constexpr (sizeof(T) == 4) d.epark_e[i] = make_float2(e.s, e.c);   // float64 in the gather
            else d.esite_e[i] = lane0_double(e);
        }
    }
}

// Groups of atoms are handed out one at a time from a counter in the status
// words, so that CTAs that start late (the cheap kernel shares the SMs on its
// own stream) take fewer; every group's results are its own, whichever CTA
// computes them.  The last CTA to finish sets the counter back to zero.
__device__ __forceinline__ int ace_next_group(const Dev& d, int* s_g) {
    __syncthreads();   // every thread has read the previous group
    if (threadIdx.x == 0) *s_g = atomicAdd(d.status + SW_ACE_NEXT, 1);
    __syncthreads();
    return *s_g;
}
__device__ __forceinline__ void ace_groups_done(const Dev& d) {
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(d.status + SW_ACE_DONE, 1) == (int)gridDim.x - 1) {
            d.status[SW_ACE_NEXT] = 0;   // every CTA has taken its last group
            d.status[SW_ACE_DONE] = 0;
        }
    }
}

template <typename T, int L, int NP>
__global__ void __launch_bounds__(ACE_MAX_WARPS * 32, ace_min_ctas_max<T>()) k_ace(Dev d, AceTab<T> tab) {
    const int WN = (int)(blockDim.x >> 5);   // ACE_GROUP or ACE_MAX_WARPS atoms a CTA
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_g;
    const int count = d.status[SW_NEXP];
    const int ng = (count + WN - 1) / WN;
    for (int g = ace_next_group(d, &s_g); g < ng; g = ace_next_group(d, &s_g))
        ace_group<T, L, NP>(d, tab, g * WN, count, smem_raw, nullptr, WN);
    ace_groups_done(d);
}

// Many systems: walks the flattened list {system, first atom of a group} of
// one group of systems sharing (T, L, NP); the CTA reloads the system's Dev and
// tables into shared memory when the system changes.
template <typename T>
struct AceBatch {
    const Dev* devs;
    const AceTab<T>* tabs;
    const int2* list;
    const int* count;
};

template <typename T, int L, int NP>
__global__ void __launch_bounds__(ace_warps<T>() * 32, ace_min_ctas<T>()) kb_ace(AceBatch<T> b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Dev s_dev;
    __shared__ AceTab<T> s_tab;
    const int count = *b.count;
    int cur = -1;
    for (int g = blockIdx.x; g < count; g += gridDim.x) {
        const int2 e = b.list[g];
        if (e.x != cur) {
            __syncthreads();
            load_dev(&s_dev, b.devs + e.x);
            copy_shared(&s_tab, b.tabs + e.x);
            __syncthreads();
            cur = e.x;
        }
        ace_group<T, L, NP>(s_dev, s_tab, e.y, s_dev.status[SW_NEXP], smem_raw);
    }
}

// launch shape: the shared memory of the layout, and as many resident CTAs as fit
template <typename T, int L, int NP>
inline cudaError_t ace_shape(const void* kern, int n, int cap, int tile_max, int qb, size_t* smem, int* grid,
                             int wn = ACE_GROUP) {
    const AceLay lay(tile_max, cap, n, qb, L, NP, (int)sizeof(T), wn);
    const size_t bytes = (size_t)lay.total;
    cudaError_t e = raise_smem_limit(kern, bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wn * 32, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *smem = bytes;
    *grid = per_sm * sm_count();
    return cudaSuccess;
}

template <typename T, int L, int NP>
inline cudaError_t ace_cfg(bool batch, int n, int cap, int tile_max, int qb, size_t* smem, int* grid, int wn) {
    const void* kern = batch ? (const void*)kb_ace<T, L, NP> : (const void*)k_ace<T, L, NP>;
    return ace_shape<T, L, NP>(kern, n, cap, tile_max, qb, smem, grid, batch ? ACE_GROUP : wn);
}

template <typename T, int NP>
inline cudaError_t ace_cfg_l(bool batch, int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid,
                             int wn) {
    switch (L) {
        case 0: return ace_cfg<T, 0, NP>(batch, n, cap, tile_max, qb, smem, grid, wn);
        case 1: return ace_cfg<T, 1, NP>(batch, n, cap, tile_max, qb, smem, grid, wn);
        case 2: return ace_cfg<T, 2, NP>(batch, n, cap, tile_max, qb, smem, grid, wn);
        case 3: return ace_cfg<T, 3, NP>(batch, n, cap, tile_max, qb, smem, grid, wn);
        case 4: return ace_cfg<T, 4, NP>(batch, n, cap, tile_max, qb, smem, grid, wn);
        case 5: return ace_cfg<T, 5, NP>(batch, n, cap, tile_max, qb, smem, grid, wn);
        case 6: return ace_cfg<T, 6, NP>(batch, n, cap, tile_max, qb, smem, grid, wn);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
inline cudaError_t ace_cfg_t(bool batch, int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid,
                             int wn = ACE_GROUP) {
    if (n <= 4) return ace_cfg_l<T, 4>(batch, L, n, cap, tile_max, qb, smem, grid, wn);
    if (n <= 8) return ace_cfg_l<T, 8>(batch, L, n, cap, tile_max, qb, smem, grid, wn);
    if (n <= 12) return ace_cfg_l<T, 12>(batch, L, n, cap, tile_max, qb, smem, grid, wn);
    return ace_cfg_l<T, 16>(batch, L, n, cap, tile_max, qb, smem, grid, wn);
}

template <typename T, int NP>
inline void ace_launch_l(const Dev& d, const AceTab<T>& tab, int L, size_t smem, int grid, int wn, cudaStream_t s) {
    const int th = wn * 32;
    switch (L) {
        case 0: k_ace<T, 0, NP><<<grid, th, smem, s>>>(d, tab); break;
        case 1: k_ace<T, 1, NP><<<grid, th, smem, s>>>(d, tab); break;
        case 2: k_ace<T, 2, NP><<<grid, th, smem, s>>>(d, tab); break;
        case 3: k_ace<T, 3, NP><<<grid, th, smem, s>>>(d, tab); break;
        case 4: k_ace<T, 4, NP><<<grid, th, smem, s>>>(d, tab); break;
        case 5: k_ace<T, 5, NP><<<grid, th, smem, s>>>(d, tab); break;
        case 6: k_ace<T, 6, NP><<<grid, th, smem, s>>>(d, tab); break;
    }
}

template <typename T>
inline void ace_launch_t(const Dev& d, const AceTab<T>& tab, int L, size_t smem, int grid, int wn, cudaStream_t s) {
    if (tab.np == 4) ace_launch_l<T, 4>(d, tab, L, smem, grid, wn, s);
    else if (tab.np == 8) ace_launch_l<T, 8>(d, tab, L, smem, grid, wn, s);
    else if (tab.np == 12) ace_launch_l<T, 12>(d, tab, L, smem, grid, wn, s);
    else ace_launch_l<T, 16>(d, tab, L, smem, grid, wn, s);
}

template <typename T, int NP>
inline void ace_batch_launch_l(const AceBatch<T>& b, int L, size_t smem, int grid, cudaStream_t s) {
    switch (L) {
        case 0: kb_ace<T, 0, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(b); break;
        case 1: kb_ace<T, 1, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(b); break;
        case 2: kb_ace<T, 2, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(b); break;
        case 3: kb_ace<T, 3, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(b); break;
        case 4: kb_ace<T, 4, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(b); break;
        case 5: kb_ace<T, 5, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(b); break;
        case 6: kb_ace<T, 6, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(b); break;
    }
}

template <typename T>
inline void ace_batch_launch_t(const AceBatch<T>& b, int n, int L, size_t smem, int grid, cudaStream_t s) {
    if (n <= 4) ace_batch_launch_l<T, 4>(b, L, smem, grid, s);
    else if (n <= 8) ace_batch_launch_l<T, 8>(b, L, smem, grid, s);
    else if (n <= 12) ace_batch_launch_l<T, 12>(b, L, smem, grid, s);
    else ace_batch_launch_l<T, 16>(b, L, smem, grid, s);
}

}  // namespace mixd
