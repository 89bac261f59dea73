// Expensive potential: a linear atomic cluster expansion evaluated on the
// compacted list of atoms in Lambda_exp plus its buffer (Sec. 4.5, Alg. 4).
//
// One CTA per evaluated atom (persistent grid-stride over the list):
//   1. neighbours inside the cutoff, compacted in slot order (FP64 pair vectors);
//   2. per neighbour R_n(r), R_n'(r) (Chebyshev x (1 - (r/rc)^2)^3) and Y_lm(u)
//      (associated-Legendre recurrence in z times Re/Im (x + iy)^m);
//   3. density A[n][lm] = sum_k R[k][n] Y[k][lm];
//   4. readout and its adjoint omega = dE/dA:
//      nu<=2 through S2_l = W2_l + W2_l^T; nu = 3 per l-triple (l1, l2, l3):
//        U[n1 n2 m3] = sum_n3 W[n1 n2 n3] A[n3, l3 m3]
//        Z[n1 n2 m3] = sum_(m1 m2) G A[n1, l1 m1] A[n2, l2 m2]   (Gaunt-sparse)
//        E += sum Z U;  omega3 += W^T Z;  omega1, omega2 from G A U;
//   5. pair gradients dE_i/dr_ij = u sum_lm sigma_lm Y_lm
//        + (grad_u p - u (u . grad_u p)) / r,  p = sum_lm rho_lm Y_lm,
//      rho = sum_n omega R_n, sigma = sum_n omega R_n', written per list slot.
// The site energy is summed in float64 whatever the element type T.
#include "mix_launch.h"

namespace mixd {

constexpr int ACE_NT = 128;   // threads per CTA
constexpr int ACE_CH = 32;    // neighbours per gradient chunk

template <typename T> __device__ __forceinline__ T tsqrt(T x);
template <> __device__ __forceinline__ double tsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float tsqrt<float>(float x) { return sqrtf(x); }

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

// g = u sum_lm sig_lm Y_lm + (G - u (u.G)) / r,  G = sum_lm rho_lm grad_u p_lm(u)
template <typename T, int L>
__device__ __forceinline__ void ace_pair_grad(const T* __restrict__ u4, const T* __restrict__ Y,
                                              const T* __restrict__ rho, const T* __restrict__ sig,
                                              const T* __restrict__ K, T g[3]) {
    const T x = u4[0], y = u4[1], z = u4[2], r = u4[3];
    T Pi[(L + 1) * (L + 2) / 2], C[L + 1], S[L + 1];
    legendre_tables<T, L>(x, y, z, Pi, C, S);
    T sy = T(0), Gx = T(0), Gy = T(0), Gz = T(0);
#pragma unroll
    for (int l = 0; l <= L; ++l) {
        const int o = l * l + l;
        const int pl = l * (l + 1) / 2;
        sy += sig[o] * Y[o];
        if (l >= 1) Gz += rho[o] * K[o] * Pi[pl + 1];
#pragma unroll
        for (int m = 1; m <= l; ++m) {
            const T p = Pi[pl + m];
            const T pz = (m < l) ? Pi[pl + m + 1] : T(0);
            const T kc = K[o + m] * rho[o + m];
            const T ks = K[o - m] * rho[o - m];
            sy += sig[o + m] * Y[o + m] + sig[o - m] * Y[o - m];
            // p_{l,m} = K Pi C_m:   d/dx = K Pi m C_{m-1}, d/dy = -K Pi m S_{m-1}, d/dz = K Pi' C_m
            // p_{l,-m} = K Pi S_m:  d/dx = K Pi m S_{m-1}, d/dy =  K Pi m C_{m-1}, d/dz = K Pi' S_m
            const T fm = T(m) * p;
            Gx += fm * (kc * C[m - 1] + ks * S[m - 1]);
            Gy += fm * (ks * C[m - 1] - kc * S[m - 1]);
            Gz += pz * (kc * C[m] + ks * S[m]);
        }
    }
    const T ug = x * Gx + y * Gy + z * Gz;
    const T ir = T(1) / r;
    g[0] = sy * x + (Gx - x * ug) * ir;
    g[1] = sy * y + (Gy - y * ug) * ir;
    g[2] = sy * z + (Gz - z * ug) * ir;
}

// uniform cubic B-spline with 16 coefficients on knots (a - 3) h
template <typename T>
__device__ __forceinline__ void spline16(const T* __restrict__ c, T invh, T r, T& v, T& dv) {
    T x = r * invh;
    int q = (int)floor((double)x);
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
struct AceSmem {
    int o_u, o_R, o_dR, o_Y, o_A, o_om, o_work, total_elems;
    __host__ __device__ AceSmem(int cap, int n, int L) {
        const int nlm = (L + 1) * (L + 1);
        const int d3 = 2 * L + 1;
        o_u = 0;
        o_R = o_u + ace_pad(4 * cap);
        o_dR = o_R + ace_pad(cap * n);
        o_Y = o_dR + ace_pad(cap * n);
        o_A = o_Y + ace_pad(cap * nlm);
        o_om = o_A + ace_pad(n * nlm);
        o_work = o_om + ace_pad(n * nlm);
        const int uz = 2 * ace_pad(n * n * d3);
        const int rs = 2 * ace_pad(ACE_CH * nlm);
        total_elems = o_work + (uz > rs ? uz : rs);
    }
};

template <typename T, int L>
__global__ void __launch_bounds__(ACE_NT) k_ace(Dev d, AceTab<T> tab) {
    constexpr int NLM = (L + 1) * (L + 1);
    using V = typename Vec4<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_slot[MAX_CAP];
    __shared__ int s_wcnt[ACE_NT / 32];
    __shared__ double s_red[ACE_NT / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = tab.n, cap = d.cap;
    const AceSmem lay(cap, n, L);
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* s_u = sm + lay.o_u;
    T* s_R = sm + lay.o_R;
    T* s_dR = sm + lay.o_dR;
    T* s_Y = sm + lay.o_Y;
    T* s_A = sm + lay.o_A;
    T* s_om = sm + lay.o_om;
    T* s_work = sm + lay.o_work;

    V* GE = reinterpret_cast<V*>(d.ge);
    const double rc2 = d.rce2;
    const T rc = (T)tab.rc;
    const T invrc = T(1) / rc;
    const T invh = T(13) / rc;
    const int count = d.status[SW_NEXP];
    const unsigned lt = (1u << lane) - 1u;

    for (int a = blockIdx.x; a < count; a += gridDim.x) {
        const int i = d.act_e[a];
        const double4 xi = d.x[i];
        const int m = d.nnb[i];
        const int* row = d.nbr + (int64_t)i * cap;
        V* grow = GE + (int64_t)a * cap;

        // 1. neighbours inside the cutoff, ordered compaction
        int nb = 0;
        for (int base = 0; base < m; base += ACE_NT) {
            const int s = base + tid;
            bool ok = false;
            double dd[3] = {0, 0, 0}, r2 = 0;
            if (s < m) {
                const double4 xj = d.x[row[s]];
                dd[0] = xj.x - xi.x;
                dd[1] = xj.y - xi.y;
                dd[2] = xj.z - xi.z;
                for (int k = 0; k < 3; ++k)
                    if (d.box.per[k]) dd[k] -= d.box.L[k] * rint(dd[k] * d.box.invL[k]);
                r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
                ok = r2 < rc2;
                if (!ok) {
                    V z;
                    z.x = z.y = z.z = z.w = T(0);
                    grow[s] = z;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            if (lane == 0) s_wcnt[warp] = __popc(bal);
            __syncthreads();
            int off = nb, tot = 0;
            for (int w = 0; w < ACE_NT / 32; ++w) {
                if (w < warp) off += s_wcnt[w];
                tot += s_wcnt[w];
            }
            if (ok) {
                const int k = off + __popc(bal & lt);
                const double r = sqrt(r2), ir = 1.0 / r;
                s_slot[k] = s;
                s_u[4 * k + 0] = (T)(dd[0] * ir);
                s_u[4 * k + 1] = (T)(dd[1] * ir);
                s_u[4 * k + 2] = (T)(dd[2] * ir);
                s_u[4 * k + 3] = (T)r;
            }
            nb += tot;
            __syncthreads();
        }

        // 2. radial functions, spherical harmonics, pair term
        double epart = 0.0;
        for (int k = tid; k < nb; k += ACE_NT) {
            const T r = s_u[4 * k + 3];
            const T sc = T(2) * r * invrc - T(1);
            const T q = r * invrc;
            const T om1 = T(1) - q * q;
            const T fc = om1 * om1 * om1;
            const T dfc = T(-6) * r * invrc * invrc * om1 * om1;
            T t0 = T(1), t1 = sc, dt0 = T(0), dt1 = T(1);
            T* R = s_R + k * n;
            T* dR = s_dR + k * n;
            R[0] = fc;
            dR[0] = dfc;
            if (n > 1) {
                R[1] = sc * fc;
                dR[1] = T(2) * invrc * fc + sc * dfc;
            }
            for (int p = 2; p < n; ++p) {
                const T t2 = T(2) * sc * t1 - t0;
                const T dt2 = T(2) * t1 + T(2) * sc * dt1 - dt0;
                R[p] = t2 * fc;
                dR[p] = dt2 * T(2) * invrc * fc + t2 * dfc;
                t0 = t1;
                t1 = t2;
                dt0 = dt1;
                dt1 = dt2;
            }
            ylm_eval<T, L>(s_u[4 * k], s_u[4 * k + 1], s_u[4 * k + 2], tab.ylmk, s_Y + k * NLM);
            if (tab.has_pair) {
                T v, dv;
                spline16<T>(tab.pair, invh, r, v, dv);
                epart += 0.5 * (double)v;
            }
        }
        __syncthreads();

        // 3. density
        for (int o = tid; o < n * NLM; o += ACE_NT) {
            const int q = o / NLM, lm = o - q * NLM;
            T acc = T(0);
            for (int k = 0; k < nb; ++k) acc += s_R[k * n + q] * s_Y[k * NLM + lm];
            s_A[o] = acc;
        }
        __syncthreads();

        // 4a. nu = 1 and nu = 2; initialises omega
        for (int o = tid; o < n * NLM; o += ACE_NT) {
            const int q = o / NLM, lm = o - q * NLM;
            int l = 0;
            while ((l + 1) * (l + 1) <= lm) ++l;
            T val = T(0);
            if (tab.nu >= 2) {
                const T* S2 = tab.S2 + ((int64_t)l * n + q) * n;
                for (int q2 = 0; q2 < n; ++q2) val += S2[q2] * s_A[q2 * NLM + lm];
            }
            const T av = s_A[o];
            epart += 0.5 * (double)(av * val);
            if (lm == 0) {
                const T c = tab.c1[q];
                epart += (double)(c * av);
                val += c;
            }
            s_om[o] = val;
        }
        __syncthreads();

        // 4b. nu = 3, one l-triple at a time
        for (int t = 0; t < tab.ntau; ++t) {
            const int l1 = tab.tau[4 * t], l2 = tab.tau[4 * t + 1], l3 = tab.tau[4 * t + 2];
            const int gb = tab.tau[4 * t + 3];
            const int d1 = 2 * l1 + 1, d2 = 2 * l2 + 1, d3 = 2 * l3 + 1;
            const int o1 = l1 * l1, o2 = l2 * l2, o3 = l3 * l3;
            const int* g3o = tab.goff + gb;
            const int* g1o = g3o + d3 + 1;
            const int* g2o = g1o + d1 + 1;
            const T* W = tab.W3 + (int64_t)t * n * n * n;
            T* sU = s_work;
            T* sZ = s_work + ace_pad(n * n * d3);
            const int nout = n * n * d3;
            for (int o = tid; o < nout; o += ACE_NT) {
                const int q12 = o / d3, m3 = o - q12 * d3;
                const int q1 = q12 / n, q2 = q12 - q1 * n;
                const T* Wr = W + q12 * n;
                T u = T(0);
                for (int q3 = 0; q3 < n; ++q3) u += Wr[q3] * s_A[q3 * NLM + o3 + m3];
                T z = T(0);
                const T* A1 = s_A + q1 * NLM + o1;
                const T* A2 = s_A + q2 * NLM + o2;
                for (int e = g3o[m3]; e < g3o[m3 + 1]; ++e) {
                    const int pk = tab.gidx[e];
                    z += tab.gval[e] * A1[pk & 255] * A2[pk >> 8];
                }
                sU[o] = u;
                sZ[o] = z;
                epart += (double)(u * z);
            }
            __syncthreads();
            for (int o = tid; o < n * d3; o += ACE_NT) {
                const int q3 = o / d3, m3 = o - q3 * d3;
                T acc = T(0);
                for (int q12 = 0; q12 < n * n; ++q12) acc += W[q12 * n + q3] * sZ[q12 * d3 + m3];
                s_om[q3 * NLM + o3 + m3] += acc;
            }
            __syncthreads();
            for (int o = tid; o < n * d1; o += ACE_NT) {
                const int q1 = o / d1, m1 = o - q1 * d1;
                T acc = T(0);
                for (int e = g1o[m1]; e < g1o[m1 + 1]; ++e) {
                    const int pk = tab.gidx[e];
                    const int m2 = pk & 255, m3 = pk >> 8;
                    T s = T(0);
                    for (int q2 = 0; q2 < n; ++q2) s += s_A[q2 * NLM + o2 + m2] * sU[(q1 * n + q2) * d3 + m3];
                    acc += tab.gval[e] * s;
                }
                s_om[q1 * NLM + o1 + m1] += acc;
            }
            __syncthreads();
            for (int o = tid; o < n * d2; o += ACE_NT) {
                const int q2 = o / d2, m2 = o - q2 * d2;
                T acc = T(0);
                for (int e = g2o[m2]; e < g2o[m2 + 1]; ++e) {
                    const int pk = tab.gidx[e];
                    const int m1 = pk & 255, m3 = pk >> 8;
                    T s = T(0);
                    for (int q1 = 0; q1 < n; ++q1) s += s_A[q1 * NLM + o1 + m1] * sU[(q1 * n + q2) * d3 + m3];
                    acc += tab.gval[e] * s;
                }
                s_om[q2 * NLM + o2 + m2] += acc;
            }
            __syncthreads();
        }

        // 5. pair gradients, in chunks of neighbours
        T* s_rho = s_work;
        T* s_sig = s_work + ace_pad(ACE_CH * NLM);
        for (int k0 = 0; k0 < nb; k0 += ACE_CH) {
            const int kc = nb - k0 < ACE_CH ? nb - k0 : ACE_CH;
            for (int o = tid; o < kc * NLM; o += ACE_NT) {
                const int kl = o / NLM, lm = o - kl * NLM;
                const int k = k0 + kl;
                T rho = T(0), sig = T(0);
                for (int q = 0; q < n; ++q) {
                    const T w = s_om[q * NLM + lm];
                    rho += w * s_R[k * n + q];
                    sig += w * s_dR[k * n + q];
                }
                s_rho[o] = rho;
                s_sig[o] = sig;
            }
            __syncthreads();
            for (int kl = tid; kl < kc; kl += ACE_NT) {
                const int k = k0 + kl;
                T g[3];
                ace_pair_grad<T, L>(s_u + 4 * k, s_Y + k * NLM, s_rho + kl * NLM, s_sig + kl * NLM, tab.ylmk, g);
                if (tab.has_pair) {
                    T v, dv;
                    spline16<T>(tab.pair, invh, s_u[4 * k + 3], v, dv);
                    const T hp = T(0.5) * dv;
                    g[0] += hp * s_u[4 * k];
                    g[1] += hp * s_u[4 * k + 1];
                    g[2] += hp * s_u[4 * k + 2];
                }
                V gv;
                gv.x = g[0];
                gv.y = g[1];
                gv.z = g[2];
                gv.w = T(0);
                grow[s_slot[k]] = gv;
            }
            __syncthreads();
        }

        // site energy (float64, fixed reduction order)
        for (int o = 16; o > 0; o >>= 1) epart += __shfl_down_sync(0xffffffffu, epart, o);
        if (lane == 0) s_red[warp] = epart;
        __syncthreads();
        if (tid == 0) {
            double e = 0.0;
            for (int w = 0; w < ACE_NT / 32; ++w) e += s_red[w];
            d.esite_e[i] = e;
        }
        __syncthreads();
    }
}

template <typename T, int L>
static cudaError_t ace_cfg(int n, int cap, size_t* smem, int* grid) {
    const AceSmem lay(cap, n, L);
    const size_t bytes = (size_t)lay.total_elems * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_ace<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ace<T, L>, ACE_NT, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *smem = bytes;
    *grid = per_sm * sm_count();
    return cudaSuccess;
}

template <typename T>
static cudaError_t ace_cfg_t(int L, int n, int cap, size_t* smem, int* grid) {
    switch (L) {
        case 0: return ace_cfg<T, 0>(n, cap, smem, grid);
        case 1: return ace_cfg<T, 1>(n, cap, smem, grid);
        case 2: return ace_cfg<T, 2>(n, cap, smem, grid);
        case 3: return ace_cfg<T, 3>(n, cap, smem, grid);
        case 4: return ace_cfg<T, 4>(n, cap, smem, grid);
        case 5: return ace_cfg<T, 5>(n, cap, smem, grid);
        case 6: return ace_cfg<T, 6>(n, cap, smem, grid);
    }
    return cudaErrorInvalidValue;
}

cudaError_t ace_configure(int precision, int L, int n, int cap, size_t* smem, int* grid) {
    if (cap > MAX_CAP) return cudaErrorInvalidValue;
    return precision == MIX_FP64 ? ace_cfg_t<double>(L, n, cap, smem, grid) : ace_cfg_t<float>(L, n, cap, smem, grid);
}

template <typename T>
static void ace_launch_t(const Dev& d, const AceTab<T>& tab, int L, size_t smem, int grid, cudaStream_t s) {
    switch (L) {
        case 0: k_ace<T, 0><<<grid, ACE_NT, smem, s>>>(d, tab); break;
        case 1: k_ace<T, 1><<<grid, ACE_NT, smem, s>>>(d, tab); break;
        case 2: k_ace<T, 2><<<grid, ACE_NT, smem, s>>>(d, tab); break;
        case 3: k_ace<T, 3><<<grid, ACE_NT, smem, s>>>(d, tab); break;
        case 4: k_ace<T, 4><<<grid, ACE_NT, smem, s>>>(d, tab); break;
        case 5: k_ace<T, 5><<<grid, ACE_NT, smem, s>>>(d, tab); break;
        case 6: k_ace<T, 6><<<grid, ACE_NT, smem, s>>>(d, tab); break;
    }
}

void launch_ace(const Dev& d, const void* tab, int precision, int L, size_t smem, int grid, cudaStream_t s) {
    if (precision == MIX_FP64) ace_launch_t<double>(d, *static_cast<const AceTab<double>*>(tab), L, smem, grid, s);
    else ace_launch_t<float>(d, *static_cast<const AceTab<float>*>(tab), L, smem, grid, s);
}

}  // namespace mixd
