// Expensive potential (templates): a linear atomic cluster expansion evaluated on the
// compacted list of atoms in Lambda_exp plus its buffer (Sec. 4.5, Alg. 4).
//
// One CTA (4 warps) per evaluated atom, persistent over the list:
//   1. neighbours inside the cutoff, compacted in slot order (FP64 pair
//      vectors, rounded once to T);
//   2. density A[lm][q] = sum_k R_q(r_k) Y_lm(u_k), neighbours in chunks:
//      R (Chebyshev recurrence x (1 - (r/rc)^2)^3) and Y (associated-Legendre
//      recurrence in z times Re/Im (x + iy)^m) go to shared memory, each thread
//      keeps fixed outputs in registers;
//   3. nu <= 2 readout; omega = dE/dA initialised;
//   4. nu = 3, the l-triples split over the warps (balanced on the host), each
//      warp with its own omega copy, so the loop needs no block barrier:
//        U[q1 q2][m3] = sum_q3 W[q1 q2 q3] A[l3 m3][q3]
//        Z[q1 q2][m3] = sum_(m1 m2) G A[l1 m1][q1] A[l2 m2][q2]   (Gaunt-sparse)
//        E += sum Z U;  omega3 += W^T Z;  omega1 += G A2 U;  omega2 += G A1 U;
//      in the U/Z pass a lane owns one q1 and a block of qb consecutive q2
//      (the W rows of that block sit in registers), so each Gaunt entry costs
//      one packed table load, one scalar A1 load and one vector A2 load for qb
//      accumulations; omega3 = W^T Z with a lane per output; where
//      two l's coincide W is symmetrised on the host, the adjoints through the
//      coinciding factors are equal, and one of them is computed and scaled
//      (omega2 only for distinct l's, omega1 not when all three are equal);
//   5. omega = sum of the warp copies (fixed order);
//   6. pair gradients dE_i/dr_ij = u sum_lm sigma_lm Y_lm
//        + (grad_u p - u (u . grad_u p)) / r,  rho = omega R, sigma = omega R',
//      R, R', Y recomputed per neighbour in registers, the lm sum split over
//      pairs of warps; written per list slot, to the atom's own row and to the
//      partner's incoming row (slot rev, stamped with the evaluation count).
// Per-atom arrays are stored transposed ([lm][q], q padded to NP = 4k with
// zeros) so that the inner products run over 4-wide vector loads with no index
// division.  Site energy partial sums are kept in T per thread and reduced in
// float64 once per atom in a fixed order.
#pragma once

#include "mix_launch.h"

namespace mixd {

constexpr int ACE_CH = 64;               // neighbours per density chunk

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
template <typename T>
__device__ __forceinline__ V4<T> ldg4(const T* p);
template <>
__device__ __forceinline__ V4<float> ldg4<float>(const float* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {v.x, v.y, v.z, v.w};
}
template <>
__device__ __forceinline__ V4<double> ldg4<double>(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}

// one Gaunt entry through the read-only path (one 8- or 16-byte load)
__device__ __forceinline__ void ld_gent(const GEnt<float>* p, int& pk, float& g) {
    const int2 v = __ldg(reinterpret_cast<const int2*>(p));
    pk = v.x;
    g = __int_as_float(v.y);
}
__device__ __forceinline__ void ld_gent(const GEnt<double>* p, int& pk, double& g) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(p));
    pk = v.x;
    g = __hiloint2double(v.w, v.z);
}

// QB consecutive values from shared memory (QB in {1, 2, 4}, aligned to QB)
template <typename T, int QB>
__device__ __forceinline__ void ld_blk(const T* p, T* out) {
    if constexpr (QB == 4) {
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

__host__ __device__ constexpr int ace_pad(int x) { return (x + 3) & ~3; }

// shared-memory layout (element offsets), shared by host sizing and the kernel
// The density chunk buffers (R, Y of up to ACE_CH neighbours) and the per-warp
// nu = 3 scratch are never live together and share one region.
struct AceSmem {
    int o_u, o_At, o_om, o_gp, o_w, o_cR, o_cY, ws, total;
    __host__ __device__ AceSmem(int cap, int n, int nq, int L, int NP, int W) {
        const int nlm = (L + 1) * (L + 1);
        const int D = 2 * L + 1;
        o_u = 0;
        o_At = ace_pad(4 * cap);
        o_om = o_At + nlm * NP;
        o_gp = o_om + nlm * NP;
        o_w = o_gp + 2 * (16 * W) * 4;         // gradient partials: 2 halves x 16 W neighbours
        o_cR = o_w;
        o_cY = o_cR + ACE_CH * NP;
        ws = D * n * NP + D * nq + nlm * NP;   // per warp: U, ZT, omega copy
        const int chunk = ACE_CH * NP + ace_pad(ACE_CH * nlm);
        const int wsall = W * ws;
        total = o_w + (chunk > wsall ? chunk : wsall);
    }
};

// nu = 3, U and Z of one l-triple for this warp.  Lane units are (q1, block of
// QB consecutive q2); the m3 loop is uniform over the warp so every Gaunt
// entry and A3 row load is a broadcast.
//   U[m3][q1][q2] = sum_q3 W[q1 q2][q3] A3[m3][q3]      (stored, q2 padded to NP)
//   Z[m3][q1 n + q2] = sum_(m1 m2) G A1[m1][q1] A2[m2][q2]
//   ep += sum U Z
// Without U (all three l's equal: no adjoint needs U) only Z is formed and the
// energy is taken in the omega3 pass as sum A3 (W^T Z), the same sum reordered.
template <typename T, int NP, int QB, bool WITHU>
__device__ __forceinline__ void nu3_uz(const T* __restrict__ W, const T* A1, const T* A2, const T* A3,
                                       const int* g3o, const GEnt<T>* __restrict__ gent, int n, int nq, int d3,
                                       int lane, T* U1, T* ZT, T& ep) {
    constexpr int nqb = NP / QB;
    const int units = n * nqb;
    for (int u0 = 0; u0 < units; u0 += 32) {
        const int u = u0 + lane;
        const bool uv = u < units;
        const int uu = uv ? u : 0;
        const int q1 = uu / nqb;
        const int q2 = (uu - q1 * nqb) * QB;
        T w[QB][NP];
#pragma unroll
        for (int r = 0; r < QB; ++r) {
            if (!WITHU) break;
            const bool ok = uv && q2 + r < n;
            const T* wr = W + (q1 * n + (ok ? q2 + r : 0)) * NP;
#pragma unroll
            for (int p = 0; p < NP; p += 4) {
                V4<T> v = ldg4<T>(wr + p);
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
            if (WITHU) {
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
            for (int e = g3o[m3]; e < e1; ++e) {
                int pk;
                T g;
                ld_gent(gent + e, pk, g);
                const T ga = g * A1[(pk & 255) * NP + q1];
                T a2[QB];
                ld_blk<T, QB>(A2 + (pk >> 8) * NP + q2, a2);
#pragma unroll
                for (int r = 0; r < QB; ++r) z[r] += ga * a2[r];
            }
            if (uv) {
#pragma unroll
                for (int r = 0; r < QB; ++r) {
                    if (WITHU) U1[(m3 * n + q1) * NP + q2 + r] = uo[r];
                    if (q2 + r < n) {
                        ZT[m3 * nq + q1 * n + q2 + r] = z[r];
                        if (WITHU) ep += uo[r] * z[r];
                    }
                }
            }
        }
    }
}

// One evaluated atom (index a of the system's expensive list), by the whole CTA.
template <typename T, int L, int NP>
__device__ __forceinline__ void ace_atom(const Dev& d, const AceTab<T>& tab, int a, unsigned char* smem_raw,
                                         int* s_slot, int* s_wcnt, double* s_red) {
    constexpr int WN = ace_warps<T>();
    constexpr int NT = WN * 32;
    constexpr int NLM = (L + 1) * (L + 1);
    constexpr int D = 2 * L + 1;
    constexpr int NOUT = (NLM * NP + NT - 1) / NT;
    constexpr int QM = sizeof(T) == 4 ? 4 : 2;     // largest q2 block of the U/Z pass
    constexpr int PER = 16 * WN;                   // neighbours per gradient pass
    using V = typename Vec4<T>::type;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = tab.n, nq = tab.nq, cap = d.cap;
    const AceSmem lay(cap, n, nq, L, NP, WN);
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* s_u = sm + lay.o_u;
    T* s_At = sm + lay.o_At;
    T* s_om = sm + lay.o_om;
    T* s_cR = sm + lay.o_cR;
    T* s_cY = sm + lay.o_cY;
    T* s_gp = sm + lay.o_gp;
    T* U1 = sm + lay.o_w + warp * lay.ws;   // U[m3][q1][q2]
    T* ZT = U1 + D * n * NP;                // Z[m3][q1 q2]
    T* omw = ZT + D * nq;

    V* GE = reinterpret_cast<V*>(d.ge);
    V* GIN = reinterpret_cast<V*>(d.ge_in);
    const int stamp = d.status[SW_EPOCH];
    const T rc2 = (T)d.rce2;
    const T rc = (T)tab.rc;
    const T invrc = T(1) / rc;
    const T invh = T(13) / rc;
    const unsigned lt = (1u << lane) - 1u;
    {
        const int i = d.act_e[a];
        const PairFrame<T> pf(d, i);
        const int m = d.nnb[i];
        const int* row = d.nbr + (int64_t)i * cap;
        const int* rvr = d.rev + (int64_t)i * cap;
        V* grow = GE + (int64_t)i * cap;

        // 1. neighbours inside the cutoff, ordered compaction
        int nb = 0;
        for (int base = 0; base < m; base += NT) {
            const int s = base + tid;
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
            if (lane == 0) s_wcnt[warp] = __popc(bal);
            __syncthreads();
            int off = nb, tot = 0;
#pragma unroll
            for (int w = 0; w < WN; ++w) {
                if (w < warp) off += s_wcnt[w];
                tot += s_wcnt[w];
            }
            if (ok) {
                const int k = off + __popc(bal & lt);
                const T r = sqrt(r2), ir = T(1) / r;
                s_slot[k] = s;
                s_u[4 * k + 0] = dv[0] * ir;
                s_u[4 * k + 1] = dv[1] * ir;
                s_u[4 * k + 2] = dv[2] * ir;
                s_u[4 * k + 3] = r;
            }
            nb += tot;
            __syncthreads();
        }

        // 2. density, neighbours in chunks
        T ep = T(0);
        T acc[NOUT];
#pragma unroll
        for (int j = 0; j < NOUT; ++j) acc[j] = T(0);
        for (int k0 = 0; k0 < nb; k0 += ACE_CH) {
            const int kc = nb - k0 < ACE_CH ? nb - k0 : ACE_CH;
            for (int kl = tid; kl < kc; kl += NT) {
                const int k = k0 + kl;
                const T r = s_u[4 * k + 3];
                T R[NP], dR[NP];
                radial<T, NP>(r, invrc, n, R, dR);
#pragma unroll
                for (int p = 0; p < NP; ++p) s_cR[kl * NP + p] = R[p];
                ylm_eval<T, L>(s_u[4 * k], s_u[4 * k + 1], s_u[4 * k + 2], tab.ylmk, s_cY + kl * NLM);
                if (tab.has_pair) {
                    T v, dv;
                    spline16<T>(tab.pair, invh, r, v, dv);
                    ep += T(0.5) * v;
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < NOUT; ++j) {
                const int o = tid + j * NT;
                if (o < NLM * NP) {
                    const int lm = o / NP, q = o - lm * NP;
                    T s = acc[j];
                    for (int kl = 0; kl < kc; ++kl) s += s_cR[kl * NP + q] * s_cY[kl * NLM + lm];
                    acc[j] = s;
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < NOUT; ++j) {
            const int o = tid + j * NT;
            if (o < NLM * NP) s_At[o] = acc[j];
        }
        // the density chunks are dead: zero this warp's scratch (its padding,
        // q >= n and q1 q2 >= n*n, is read as zeros below and never written)
        for (int k = lane; k < lay.ws; k += 32) U1[k] = T(0);
        __syncthreads();

        // 3. nu = 1 and nu = 2; initialises omega
#pragma unroll
        for (int j = 0; j < NOUT; ++j) {
            const int o = tid + j * NT;
            if (o < NLM * NP) {
                const int lm = o / NP, q = o - lm * NP;
                T val = T(0);
                if (q < n) {
                    int l = 0;
                    while ((l + 1) * (l + 1) <= lm) ++l;
                    if (tab.nu >= 2) {
                        const T* S2 = tab.S2 + ((int64_t)l * n + q) * n;
                        const T* Ar = s_At + lm * NP;
                        for (int q2 = 0; q2 < n; ++q2) val += S2[q2] * Ar[q2];
                    }
                    const T av = s_At[o];
                    ep += T(0.5) * av * val;
                    if (lm == 0) {
                        const T c = tab.c1[q];
                        ep += c * av;
                        val += c;
                    }
                }
                s_om[o] = val;
            }
        }

        // 4. nu = 3: this warp's l-triples
        for (int it = tab.wt_off[warp]; it < tab.wt_off[warp + 1]; ++it) {
            const int t = tab.wt_list[it];
            const int l1 = tab.tau[4 * t], l2 = tab.tau[4 * t + 1], l3 = tab.tau[4 * t + 2];
            const int gb = tab.tau[4 * t + 3];
            // coinciding l's (W symmetrised on the host): scale instead of recompute
            const int mode = tab.tmode[t];
            const T mult1 = mode == 1 ? T(2) : T(1);
            const T mult3 = mode == 3 ? T(3) : (mode == 2 ? T(2) : T(1));
            const int d1 = 2 * l1 + 1, d2 = 2 * l2 + 1, d3 = 2 * l3 + 1;
            const T* A1 = s_At + l1 * l1 * NP;
            const T* A2 = s_At + l2 * l2 * NP;
            const T* A3 = s_At + l3 * l3 * NP;
            const int* g3o = tab.goff + gb;
            const int* g1o = g3o + d3 + 1;
            const int* g2o = g1o + d1 + 1;
            const T* W = tab.W3 + (int64_t)t * n * n * NP;
            const T* WT = tab.WT3 + (int64_t)t * n * nq;
            if (mode == 3) nu3_uz<T, NP, QM, false>(W, A1, A2, A3, g3o, tab.gent, n, nq, d3, lane, U1, ZT, ep);
            else if (tab.qb == QM) nu3_uz<T, NP, QM, true>(W, A1, A2, A3, g3o, tab.gent, n, nq, d3, lane, U1, ZT, ep);
            else nu3_uz<T, NP, QM / 2, true>(W, A1, A2, A3, g3o, tab.gent, n, nq, d3, lane, U1, ZT, ep);
            __syncwarp();
            // omega3 += W^T Z
            for (int o = lane; o < n * d3; o += 32) {
                const int q3 = o / d3, m3 = o - q3 * d3;
                const T* wr = WT + q3 * nq;
                const T* zr = ZT + m3 * nq;
                T s = T(0);
                for (int p = 0; p < nq; p += 4) {
                    const V4<T> a4 = ldg4<T>(wr + p);
                    const V4<T> b4 = ld4<T>(zr + p);
                    s += a4.x * b4.x + a4.y * b4.y + a4.z * b4.z + a4.w * b4.w;
                }
                omw[(l3 * l3 + m3) * NP + q3] += mult3 * s;
                if (mode == 3) ep += A3[m3 * NP + q3] * s;
            }
            __syncwarp();
            // omega1 += G A2 U (equal to omega3 when all three l's coincide)
            // (lanes in m1-major order: lanes sharing m1 share the Gaunt loop and its loads)
            if (mode != 3) for (int o = lane; o < n * d1; o += 32) {
                const int m1 = o / n, q1 = o - m1 * n;
                T accv = T(0);
                for (int e = g1o[m1]; e < g1o[m1 + 1]; ++e) {
                    int pk;
                    T gv;
                    ld_gent(tab.gent + e, pk, gv);
                    const T* ar = A2 + (pk & 255) * NP;
                    const T* ur = U1 + ((pk >> 8) * n + q1) * NP;
                    T s = T(0);
#pragma unroll
                    for (int p = 0; p < NP; p += 4) {
                        const V4<T> a4 = ld4<T>(ar + p);
                        const V4<T> b4 = ld4<T>(ur + p);
                        s += a4.x * b4.x + a4.y * b4.y + a4.z * b4.z + a4.w * b4.w;
                    }
                    accv += gv * s;
                }
                omw[(l1 * l1 + m1) * NP + q1] += mult1 * accv;
            }
            __syncwarp();
            // omega2 += G A1 U, needed only when the three l's are distinct
            // (otherwise it equals omega1 or omega3, already scaled in)
            if (mode == 0) for (int o = lane; o < n * d2; o += 32) {
                const int m2 = o / n, q2 = o - m2 * n;
                T accv = T(0);
                for (int e = g2o[m2]; e < g2o[m2 + 1]; ++e) {
                    int pk;
                    T gv;
                    ld_gent(tab.gent + e, pk, gv);
                    const T* ar = A1 + (pk & 255) * NP;
                    const T* ur = U1 + (pk >> 8) * n * NP + q2;
                    T s = T(0);
                    for (int q1 = 0; q1 < n; ++q1) s += ar[q1] * ur[q1 * NP];
                    accv += gv * s;
                }
                omw[(l2 * l2 + m2) * NP + q2] += accv;
            }
            __syncwarp();
        }
        __syncthreads();

        // 5. omega = nu<=2 part + the warp copies, in a fixed order
        for (int o = tid; o < NLM * NP; o += NT) {
            T s = s_om[o];
#pragma unroll
            for (int w = 0; w < WN; ++w) s += sm[lay.o_w + w * lay.ws + D * n * NP + D * nq + o];
            s_om[o] = s;
        }
        __syncthreads();

        // 6. pair gradients: warp pair (2s, 2s+1) takes neighbours k0 + 32 s .. k0 + 32 s + 31;
        //    the two warps of a pair split the lm sum by parity
        const int half = warp & 1, sub = warp >> 1;
        for (int k0 = 0; k0 < nb; k0 += PER) {
            const int kl = sub * 32 + lane;
            const int k = k0 + kl;
            T sy = T(0), Gx = T(0), Gy = T(0), Gz = T(0);
            if (k < nb) {
                const T x = s_u[4 * k], y = s_u[4 * k + 1], z = s_u[4 * k + 2], r = s_u[4 * k + 3];
                T R[NP], dR[NP];
                radial<T, NP>(r, invrc, n, R, dR);
                T Pi[(L + 1) * (L + 2) / 2], C[L + 1], S[L + 1];
                legendre_tables<T, L>(x, y, z, Pi, C, S);
                const T* K = tab.ylmk;
#pragma unroll
                for (int l = 0; l <= L; ++l) {
                    const int pl = l * (l + 1) / 2;
#pragma unroll
                    for (int mm = -l; mm <= l; ++mm) {
                        const int lm = l * l + l + mm;
                        if ((lm & 1) != half) continue;
                        const T* orow = s_om + lm * NP;
                        T rho = T(0), sig = T(0);
#pragma unroll
                        for (int p = 0; p < NP; p += 4) {
                            const V4<T> o4 = ld4<T>(orow + p);
                            rho += o4.x * R[p] + o4.y * R[p + 1] + o4.z * R[p + 2] + o4.w * R[p + 3];
                            sig += o4.x * dR[p] + o4.y * dR[p + 1] + o4.z * dR[p + 2] + o4.w * dR[p + 3];
                        }
                        const int mu = mm < 0 ? -mm : mm;
                        const T kk = K[lm];
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
            }
            T* gp = s_gp + (half * PER + kl) * 4;
            gp[0] = sy;
            gp[1] = Gx;
            gp[2] = Gy;
            gp[3] = Gz;
            __syncthreads();
            if (tid < PER && k0 + tid < nb) {
                const int kk = k0 + tid;
                const T* g0 = s_gp + tid * 4;
                const T* g1 = s_gp + (PER + tid) * 4;
                const T x = s_u[4 * kk], y = s_u[4 * kk + 1], z = s_u[4 * kk + 2], r = s_u[4 * kk + 3];
                const T syt = g0[0] + g1[0];
                const T gxt = g0[1] + g1[1], gyt = g0[2] + g1[2], gzt = g0[3] + g1[3];
                const T ug = x * gxt + y * gyt + z * gzt;
                const T ir = T(1) / r;
                T g[3] = {syt * x + (gxt - x * ug) * ir, syt * y + (gyt - y * ug) * ir, syt * z + (gzt - z * ug) * ir};
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
                const int slot = s_slot[kk];
                grow[slot] = gv;
                gv.w = stamp_as(T(0), stamp);
                GIN[(int64_t)row[slot] * cap + rvr[slot]] = gv;
            }
            __syncthreads();
        }

        // site energy (float64, fixed reduction order)
        const auto e = warp_sum(ep);   // fixed order; compensated for float
        if constexpr (sizeof(T) == 4) {
            // float64 conversion and the sum over warps happen in the gather
            if (lane == 0) d.epark_e[(int64_t)i * WN + warp] = make_float2(e.s, e.c);
        } else {
            if (lane == 0) s_red[warp] = lane0_double(e);
            __syncthreads();
            if (tid == 0) {
                double es = 0.0;
                for (int w = 0; w < WN; ++w) es += s_red[w];
                d.esite_e[i] = es;
            }
        }
        __syncthreads();
    }
}

template <typename T, int L, int NP>
__global__ void __launch_bounds__(ace_warps<T>() * 32, ace_min_ctas<T>()) k_ace(Dev d, AceTab<T> tab) {
    constexpr int WN = ace_warps<T>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_slot[MAX_CAP];
    __shared__ int s_wcnt[WN];
    __shared__ double s_red[WN];
    const int count = d.status[SW_NEXP];
    for (int a = blockIdx.x; a < count; a += gridDim.x) ace_atom<T, L, NP>(d, tab, a, smem_raw, s_slot, s_wcnt, s_red);
}

// Many systems: walks the flattened list {system, index in its expensive list}
// of one group of systems sharing (T, L, NP); the CTA reloads the system's Dev
// and tables into shared memory when the system changes.
template <typename T>
struct AceBatch {
    const Dev* devs;
    const AceTab<T>* tabs;
    const int2* list;
    const int* count;
};

template <typename T, int L, int NP>
__global__ void __launch_bounds__(ace_warps<T>() * 32, ace_min_ctas<T>()) kb_ace(AceBatch<T> b) {
    constexpr int WN = ace_warps<T>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_slot[MAX_CAP];
    __shared__ int s_wcnt[WN];
    __shared__ double s_red[WN];
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
        ace_atom<T, L, NP>(s_dev, s_tab, e.y, smem_raw, s_slot, s_wcnt, s_red);
    }
}

template <typename T, int L, int NP>
inline cudaError_t ace_cfg(int n, int cap, size_t* smem, int* grid) {
    const int nq = (n * n + 3) & ~3;
    const AceSmem lay(cap, n, nq, L, NP, ace_warps<T>());
    const size_t bytes = (size_t)lay.total * sizeof(T);
    cudaError_t e = raise_smem_limit((const void*)k_ace<T, L, NP>, bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ace<T, L, NP>, ace_warps<T>() * 32, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *smem = bytes;
    *grid = per_sm * sm_count();
    return cudaSuccess;
}

template <typename T, int NP>
inline cudaError_t ace_cfg_l(int L, int n, int cap, size_t* smem, int* grid) {
    switch (L) {
        case 0: return ace_cfg<T, 0, NP>(n, cap, smem, grid);
        case 1: return ace_cfg<T, 1, NP>(n, cap, smem, grid);
        case 2: return ace_cfg<T, 2, NP>(n, cap, smem, grid);
        case 3: return ace_cfg<T, 3, NP>(n, cap, smem, grid);
        case 4: return ace_cfg<T, 4, NP>(n, cap, smem, grid);
        case 5: return ace_cfg<T, 5, NP>(n, cap, smem, grid);
        case 6: return ace_cfg<T, 6, NP>(n, cap, smem, grid);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
inline cudaError_t ace_cfg_t(int L, int n, int cap, size_t* smem, int* grid) {
    if (n <= 4) return ace_cfg_l<T, 4>(L, n, cap, smem, grid);
    if (n <= 8) return ace_cfg_l<T, 8>(L, n, cap, smem, grid);
    if (n <= 12) return ace_cfg_l<T, 12>(L, n, cap, smem, grid);
    return ace_cfg_l<T, 16>(L, n, cap, smem, grid);
}

template <typename T, int NP>
inline void ace_launch_l(const Dev& d, const AceTab<T>& tab, int L, size_t smem, int grid, cudaStream_t s) {
    switch (L) {
        case 0: k_ace<T, 0, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(d, tab); break;
        case 1: k_ace<T, 1, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(d, tab); break;
        case 2: k_ace<T, 2, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(d, tab); break;
        case 3: k_ace<T, 3, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(d, tab); break;
        case 4: k_ace<T, 4, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(d, tab); break;
        case 5: k_ace<T, 5, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(d, tab); break;
        case 6: k_ace<T, 6, NP><<<grid, ace_warps<T>() * 32, smem, s>>>(d, tab); break;
    }
}

// multi-system launches of one (T, L, NP) group
template <typename T, int L, int NP>
inline cudaError_t ace_batch_cfg(int n, int cap, size_t* smem, int* grid) {
    const int nq = (n * n + 3) & ~3;
    const AceSmem lay(cap, n, nq, L, NP, ace_warps<T>());
    const size_t bytes = (size_t)lay.total * sizeof(T);
    cudaError_t e = raise_smem_limit((const void*)kb_ace<T, L, NP>, bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_ace<T, L, NP>, ace_warps<T>() * 32, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *smem = bytes;
    *grid = per_sm * sm_count();
    return cudaSuccess;
}

template <typename T, int NP>
inline cudaError_t ace_batch_cfg_l(int L, int n, int cap, size_t* smem, int* grid) {
    switch (L) {
        case 0: return ace_batch_cfg<T, 0, NP>(n, cap, smem, grid);
        case 1: return ace_batch_cfg<T, 1, NP>(n, cap, smem, grid);
        case 2: return ace_batch_cfg<T, 2, NP>(n, cap, smem, grid);
        case 3: return ace_batch_cfg<T, 3, NP>(n, cap, smem, grid);
        case 4: return ace_batch_cfg<T, 4, NP>(n, cap, smem, grid);
        case 5: return ace_batch_cfg<T, 5, NP>(n, cap, smem, grid);
        case 6: return ace_batch_cfg<T, 6, NP>(n, cap, smem, grid);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
inline cudaError_t ace_batch_cfg_t(int L, int n, int cap, size_t* smem, int* grid) {
    if (n <= 4) return ace_batch_cfg_l<T, 4>(L, n, cap, smem, grid);
    if (n <= 8) return ace_batch_cfg_l<T, 8>(L, n, cap, smem, grid);
    if (n <= 12) return ace_batch_cfg_l<T, 12>(L, n, cap, smem, grid);
    return ace_batch_cfg_l<T, 16>(L, n, cap, smem, grid);
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

template <typename T>
inline void ace_launch_t(const Dev& d, const AceTab<T>& tab, int L, size_t smem, int grid, cudaStream_t s) {
    if (tab.np == 4) ace_launch_l<T, 4>(d, tab, L, smem, grid, s);
    else if (tab.np == 8) ace_launch_l<T, 8>(d, tab, L, smem, grid, s);
    else if (tab.np == 12) ace_launch_l<T, 12>(d, tab, L, smem, grid, s);
    else ace_launch_l<T, 16>(d, tab, L, smem, grid, s);
}

}  // namespace mixd
