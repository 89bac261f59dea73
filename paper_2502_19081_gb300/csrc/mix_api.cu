// Host side of the C ABI declared in include/mix.h: argument checking, the
// potential tables, the workspace layout and the launch sequence of one force
// evaluation / velocity-Verlet step.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "mix_launch.h"
#include "tc.cuh"

using namespace mixd;

namespace {

// kernels per evaluation: displacement 1, lists 5, sets 4, expensive 1, cheap 1, gather 1
// (13 with geometric regions; the seed-atom modes add one or two)
constexpr int LAUNCHES_PER_EVAL = 13;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------
// real spherical harmonics on the host (same recurrence as the kernels) and
// Gauss-Legendre quadrature, used to tabulate the Gaunt coefficients

void host_ylm(int L, double x, double y, double z, std::vector<double>& Y) {
    const int nlm = (L + 1) * (L + 1);
    Y.assign(nlm, 0.0);
    std::vector<double> Pi((L + 1) * (L + 2) / 2 + 1, 0.0), C(L + 1), S(L + 1);
    auto P = [&](int l, int m) -> double& { return Pi[l * (l + 1) / 2 + m]; };
    P(0, 0) = 1.0;
    for (int m = 1; m <= L; ++m) P(m, m) = (2.0 * m - 1.0) * P(m - 1, m - 1);
    for (int m = 0; m < L; ++m) P(m + 1, m) = (2.0 * m + 1.0) * z * P(m, m);
    for (int m = 0; m <= L; ++m)
        for (int l = m + 2; l <= L; ++l)
            P(l, m) = ((2.0 * l - 1.0) * z * P(l - 1, m) - (l + m - 1.0) * P(l - 2, m)) / (double)(l - m);
    C[0] = 1.0;
    S[0] = 0.0;
    for (int m = 1; m <= L; ++m) {
        C[m] = x * C[m - 1] - y * S[m - 1];
        S[m] = x * S[m - 1] + y * C[m - 1];
    }
    for (int l = 0; l <= L; ++l) {
        const int o = l * l + l;
        for (int m = 0; m <= l; ++m) {
            double f = 1.0;
            for (int k = l - m + 1; k <= l + m; ++k) f *= (double)k;   // (l+m)!/(l-m)!
            const double N = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) / f);
            if (m == 0) {
                Y[o] = N * P(l, 0);
            } else {
                Y[o + m] = std::sqrt(2.0) * N * P(l, m) * C[m];
                Y[o - m] = std::sqrt(2.0) * N * P(l, m) * S[m];
            }
        }
    }
}

double ylm_norm(int l, int m) {
    const int mu = m < 0 ? -m : m;
    double f = 1.0;
    for (int k = l - mu + 1; k <= l + mu; ++k) f *= (double)k;
    const double N = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) / f);
    return m == 0 ? N : std::sqrt(2.0) * N;
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
            const double dp = n * (z * pn - pm) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        const double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
        const double dp = n * (z * pn - pm) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// The real Gaunt coefficients G[m1][m2][m3] of every l-triple l1 >= l2 >= l3
// with l1 <= MIX_MAX_LMAX (the kernels' order of the factors: the third, of
// smallest l, is contracted densely), by quadrature exact for the degree of
// the product (Gauss-Legendre in cos(theta) times a uniform grid in phi).  One
// set serves every potential: the coefficients depend on the l's alone.  Also
// the ordering the expensive kernels read from constant memory: by m3, m1
// ascending within a row (m1 | m2 << 8, GE_RUN_END on the last entry of each
// run of equal m1), with the row offsets of each triple.
struct GauntAll {
    std::vector<int> l1, l2, l3;             // the triples
    std::vector<std::vector<double>> G;      // [t][(m1 d2 + m2) d3 + m3]
    std::vector<int> row0;                   // [t] first row offset of triple t in rows
    std::vector<int> rows;                   // entry offsets, 2 l3 + 2 per triple (the last: the end)
    std::vector<GEnt<float>> ent_f;
    int index(int a, int b, int c) const {
        for (size_t t = 0; t < l1.size(); ++t)
            if (l1[t] == a && l2[t] == b && l3[t] == c) return (int)t;
        return -1;
    }
};

const GauntAll& gaunt_all() {
    static const GauntAll tab = [] {
        GauntAll g;
        const int L = MIX_MAX_LMAX, deg = 3 * L;
        const int nz = deg / 2 + 2, nphi = deg + 2;
        std::vector<double> gz, gw;
        gauss_legendre(nz, gz, gw);
        std::vector<std::vector<double>> Yq;
        std::vector<double> wq;
        for (int iz = 0; iz < nz; ++iz)
            for (int ip = 0; ip < nphi; ++ip) {
                const double ph = 2.0 * M_PI * ip / nphi;
                const double s = std::sqrt(std::max(0.0, 1.0 - gz[iz] * gz[iz]));
                std::vector<double> Y;
                host_ylm(L, s * std::cos(ph), s * std::sin(ph), gz[iz], Y);
                Yq.push_back(Y);
                wq.push_back(gw[iz] * 2.0 * M_PI / nphi);
            }
        for (int l3 = 0; l3 <= L; ++l3)
            for (int l2 = l3; l2 <= L; ++l2)
                for (int l1 = l2; l1 <= L; ++l1) {
                    if (((l1 + l2 + l3) & 1) || l1 > l2 + l3) continue;
                    const int d1 = 2 * l1 + 1, d2 = 2 * l2 + 1, d3 = 2 * l3 + 1;
                    std::vector<double> G((size_t)d1 * d2 * d3, 0.0);
                    for (size_t k = 0; k < wq.size(); ++k) {
                        const std::vector<double>& Y = Yq[k];
                        for (int m1 = 0; m1 < d1; ++m1)
                            for (int m2 = 0; m2 < d2; ++m2) {
                                const double y12 = wq[k] * Y[l1 * l1 + m1] * Y[l2 * l2 + m2];
                                for (int m3 = 0; m3 < d3; ++m3) G[((size_t)m1 * d2 + m2) * d3 + m3] += y12 * Y[l3 * l3 + m3];
                            }
                    }
                    g.l1.push_back(l1);
                    g.l2.push_back(l2);
                    g.l3.push_back(l3);
                    g.row0.push_back((int)g.rows.size());
                    for (int m3 = 0; m3 < d3; ++m3) {
                        g.rows.push_back((int)g.ent_f.size());
                        for (int m1 = 0; m1 < d1; ++m1) {
                            int last = -1;
                            for (int m2 = 0; m2 < d2; ++m2) {
                                const double v = G[((size_t)m1 * d2 + m2) * d3 + m3];
                                if (std::fabs(v) <= GAUNT_ZERO) continue;
                                last = (int)g.ent_f.size();
                                GEnt<float> ef;
                                std::memset(&ef, 0, sizeof ef);
                                ef.pk = m1 | (m2 << 8);
                                ef.g = (float)v;
                                g.ent_f.push_back(ef);
                            }
                            if (last >= 0) g.ent_f[last].pk |= GE_RUN_END;
                        }
                    }
                    g.rows.push_back((int)g.ent_f.size());
                    g.G.push_back(std::move(G));
                }
        // one zero entry past the last, which the kernels' prefetch may read
        GEnt<float> ef;
        std::memset(&ef, 0, sizeof ef);
        g.ent_f.push_back(ef);
        return g;
    }();
    return tab;
}

// Copies the table into the constant memory of each float kernel module on
// the current device, once per device.
int gaunt_upload() {
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MIX_ECUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return MIX_OK;
    const GauntAll& g = gaunt_all();
    if ((int)g.ent_f.size() > GAUNT_ENT_CAP || (int)g.rows.size() > GAUNT_ROW_CAP) return MIX_EINVAL;
    const cudaError_t e = ace_gaunt_upload(g.ent_f.data(), (int)g.ent_f.size(), g.rows.data(), (int)g.rows.size());
    if (e != cudaSuccess) return MIX_ECUDA;
    done.push_back(dev);
    return MIX_OK;
}

// byte arena for the tables uploaded into the workspace
struct Arena {
    std::vector<unsigned char> bytes;
    template <typename T>
    size_t put(const std::vector<T>& v) {
        const size_t off = align256(bytes.size());
        bytes.resize(off + std::max<size_t>(v.size() * sizeof(T), 16));
        if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
};

template <typename T>
std::vector<T> conv(const std::vector<double>& v) {
    return std::vector<T>(v.begin(), v.end());
}

// bf16 bit pattern of a float, rounded to nearest (ties to even)
uint16_t bf16_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
}

// The nu = 3 tables as one tile per l-triple (layout in AceTileHdr): W3 holds
// the symmetrised coefficients [t][q1 q2][q3], tau the triples (l1, l2, l3,
// first offset row), tcg each triple's first row in the constant-memory
// Gaunt table, goff/gidx/gval the Gaunt entries in three orderings (the tile
// takes the one by m2).
// tcm (tensor-core readout): 1 appends W as the bf16 B operand, 2 also its
// bf16 remainders; tiles are then 128-byte multiples.
template <typename T>
std::vector<unsigned char> ace_tiles(int n, int np, const std::vector<int>& tau, const std::vector<int>& tmode,
                                     const std::vector<int>& tcg, const std::vector<int>& goff,
                                     const std::vector<int>& gidx, const std::vector<double>& gval,
                                     const std::vector<double>& W3, std::vector<int>& off, int& tile_max,
                                     int tcm = 0) {
    const int kp = (n * n + 15) & ~15;
    const int sbo_b = (kp / 8) * TC_LBO_B;   // 8 rows of B; two such groups hold the 16 q3 rows
    const int ntau = (int)(tau.size() / 4);
    std::vector<unsigned char> out;
    off.assign(ntau + 1, 0);
    tile_max = 0;
    for (int t = 0; t < ntau; ++t) {
        const int l1 = tau[4 * t], l2 = tau[4 * t + 1], l3 = tau[4 * t + 2], gb = tau[4 * t + 3];
        // the ordering by m2 only (the kernels read the ordering by m3 from the
        // constant-memory table): its 2 l2 + 2 offset rows follow the 2 l3 + 2
        // of the ordering by m3 and the 2 l1 + 2 of the ordering by m1
        const int r2 = gb + (2 * l3 + 2) + (2 * l1 + 2), rows = 2 * l2 + 2;
        const int e0 = goff[r2], ne = goff[r2 + rows - 1] - e0;
        AceTileHdr h;
        std::memset(&h, 0, sizeof h);
        h.l1 = l1;
        h.l2 = l2;
        h.l3 = l3;
        h.mode = tmode[t];
        h.cg = tcg[t];
        size_t o = sizeof(AceTileHdr) + (size_t)n * n * np * sizeof(T);
        h.o_ge = (int)o;
        o += (size_t)ne * sizeof(GEnt<T>);
        h.o_go = (int)o;
        o += (size_t)rows * sizeof(int);
        o = (o + 15) & ~(size_t)15;
        h.o_wb = 0;
        if (tcm) {
            o = (o + 127) & ~(size_t)127;
            h.o_wb = (int)o;
            o += (size_t)(tcm == 2 ? 2 : 1) * 2 * sbo_b;
            o = (o + 127) & ~(size_t)127;
        }
        h.bytes = (int)o;
        std::vector<unsigned char> tile(o, 0);
        std::memcpy(tile.data(), &h, sizeof h);
        T* W = reinterpret_cast<T*>(tile.data() + sizeof(AceTileHdr));
        for (int q12 = 0; q12 < n * n; ++q12)
            for (int q3 = 0; q3 < n; ++q3) W[(size_t)q12 * np + q3] = (T)W3[((size_t)t * n * n + q12) * n + q3];
        for (int k = 0; k < ne; ++k) {
            GEnt<T> g;
            std::memset(&g, 0, sizeof g);
            g.pk = gidx[e0 + k];
            g.g = (T)gval[e0 + k];
            std::memcpy(tile.data() + h.o_ge + (size_t)k * sizeof g, &g, sizeof g);
        }
        for (int r = 0; r < rows; ++r) {
            const int v = goff[r2 + r] - e0;
            std::memcpy(tile.data() + h.o_go + (size_t)r * sizeof(int), &v, sizeof v);
        }
        if (sizeof(T) == 8) {
            // the ordering by m3, with the run-end flags of the constant table
            const int r3 = 2 * l3 + 2, f0 = goff[gb], nf = goff[gb + r3 - 1] - f0;
            size_t o3 = tile.size();
            h.o_ge3 = (int)o3;
            o3 += (size_t)nf * sizeof(GEnt<T>);
            h.o_go3 = (int)o3;
            o3 += (size_t)r3 * sizeof(int);
            o3 = (o3 + 15) & ~(size_t)15;
            tile.resize(o3, 0);
            h.bytes = (int)o3;
            std::memcpy(tile.data(), &h, sizeof h);
            for (int r = 0; r + 1 < r3; ++r)
                for (int k = goff[gb + r] - f0; k < goff[gb + r + 1] - f0; ++k) {
                    GEnt<T> g;
                    std::memset(&g, 0, sizeof g);
                    const int m1 = gidx[f0 + k] & 255;
                    const bool last = k + 1 >= goff[gb + r + 1] - f0 || (gidx[f0 + k + 1] & 255) != m1;
                    g.pk = gidx[f0 + k] | (last ? GE_RUN_END : 0);
                    g.g = (T)gval[f0 + k];
                    std::memcpy(tile.data() + h.o_ge3 + (size_t)k * sizeof g, &g, sizeof g);
                }
            for (int r = 0; r < r3; ++r) {
                const int v = goff[gb + r] - f0;
                std::memcpy(tile.data() + h.o_go3 + (size_t)r * sizeof(int), &v, sizeof v);
            }
        }
        if (tcm) {
            // B[q3][k] = W[k][q3], k = q1 n + q2 (zero padding stays zero)
            for (int k = 0; k < n * n; ++k)
                for (int q3 = 0; q3 < n; ++q3) {
                    const double w = W3[((size_t)t * n * n + k) * n + q3];
                    const uint16_t hi = bf16_bits((float)w);
                    const size_t at = (size_t)h.o_wb + (size_t)tc_off(q3, k, TC_LBO_B, sbo_b);
                    std::memcpy(tile.data() + at, &hi, 2);
                    if (tcm == 2) {
                        const uint16_t lo = bf16_bits((float)(w - bf16_value(hi)));
                        std::memcpy(tile.data() + at + 2 * sbo_b, &lo, 2);
                    }
                }
        }
        off[t] = (int)out.size();
        out.insert(out.end(), tile.begin(), tile.end());
        tile_max = std::max(tile_max, (int)tile.size());
    }
    off[ntau] = (int)out.size();
    return out;
}

}  // namespace

struct mix_ctx {
    mix_system sys;
    mix_options opt;
    int precision;
    // expensive
    double ace_rc;
    int n, L, nu;
    bool has_pair;
    // cheap
    double spl_rc, spl_rc3;
    // regions
    Regions regions;
    SeedRule seedrule;
    cudaStream_t stream;
    Dev dev;
    double rlist;
    int cap;
    // tables (offsets in the arena) and their element-type views
    Arena arena;
    size_t o_c1, o_S2, o_tiles, o_toff, o_ylmk, o_pair, o_sc2, o_sc3;
    int ntau, np, qb, tile_max;
    AceTab<double> ace64;
    AceTab<float> ace32;
    SplTab<double> spl64;
    SplTab<float> spl32;
    // workspace
    size_t ws_bytes;
    size_t off_tab;
    size_t o_status, o_xb, o_xf, o_xr, o_cell3, o_cell_of, o_cell_count, o_cell_start, o_cell_fill, o_cell_atoms, o_nnb, o_nbr, o_rev,
        o_lam, o_wgt, o_flags, o_act_e, o_act_c, o_pos_e, o_pos_c, o_blk_e, o_blk_c, o_ge, o_gc, o_gei, o_gci, o_ee, o_ec, o_pe, o_pc,
        o_seed, o_core, o_zsum;
    size_t ace_smem, spl_smem;
    int ace_grid, spl_grid;
    int ace_wn;                       // warps (atoms) a CTA of the CUDA-core expensive kernel
    int ace_tcm;                      // 0: CUDA-core nu = 3; 1, 2: tensor-core readout (bf16, bf16 hi/lo)
    int ace_nbuf;                     // tile buffers of the tensor-core kernel
    int spl_lpa;                      // lanes per atom of the cheap kernel (32, 16 or 8)
    bool spl_bulk;                    // periodic in every dimension (narrow lane groups allowed)
    bool spl_lpa_settled;             // the lane groups were narrowed or widened once
    int ace_grid_max, spl_grid_max;   // resident CTAs at full occupancy
    int64_t gaunt_nnz, tau_d3_sum, basis_size;
    double nu3_flops, nu3_flops_ref;
    int64_t launches;
    bool profiling;
    bool opt_graphs;
    int order;                 // MIX_ORDER_* of the two potential kernels
    cudaStream_t cap_stream;
    cudaStream_t aux;          // second branch of an evaluation: the cheap potential
    cudaEvent_t ev_fork, ev_join;
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    double graph_dt;
    bool graph_prof;
    int64_t graph_regions, regions_version;
    cudaEvent_t ev[MIX_PHASES + 1];
    double prof_total[MIX_PHASES], prof_last[MIX_PHASES];
    int64_t prof_evals;
    bool bound;
    bool need_build;
    bool forces_valid;
    int64_t steps;
    int* pinned;
    std::string err;
};

namespace {

int fail(mix_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_fail(mix_ctx* c, cudaError_t e, const char* what) {
    return fail(c, MIX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Build the element-type independent tables (in double) and pack them.
int build_tables(mix_ctx* c, const mix_ace* a, const mix_spline* sp) {
    const int n = a->n_rad, L = a->l_max, L1 = L + 1, nlm = L1 * L1;
    std::vector<double> c1(a->c1, a->c1 + n);
    std::vector<double> S2((size_t)L1 * n * n, 0.0);
    if (a->nu_max >= 2)
        for (int l = 0; l <= L; ++l)
            for (int p = 0; p < n; ++p)
                for (int q = 0; q < n; ++q) {
                    const double* C2 = a->c2 + (size_t)l * n * n;
                    const double wpq = p <= q ? C2[p * n + q] : 0.0;
                    const double wqp = q <= p ? C2[q * n + p] : 0.0;
                    S2[((size_t)l * n + p) * n + q] = wpq + wqp;
                }
    // l-triples and masked nu = 3 coefficients
    std::vector<int> tau;
    std::vector<double> W3;
    std::vector<int> goff, gidx;
    std::vector<double> gval;
    std::vector<int> tcg;   // per triple: its first row in the constant-memory table
    if (a->nu_max >= 3) {
        const GauntAll& ga = gaunt_all();
        // The potential indexes its coefficients by the ascending triple
        // la <= lb <= lc.  The kernel contracts the third factor densely
        // (U = W A3 and omega3 = W^T Z cost (2 l3 + 1) n^3 each) and the first
        // two through the Gaunt-sparse products, and the sum is the same for
        // any order of the factors, so it takes them in descending order
        // (l1, l2, l3) = (lc, lb, la): the dense factor has the smallest l.
        for (int la = 0; la <= L; ++la)
            for (int lb = la; lb <= L; ++lb)
                for (int lc = lb; lc <= L; ++lc) {
                    if (((la + lb + lc) & 1) || lc > la + lb) continue;
                    const int l1 = lc, l2 = lb, l3 = la;
                    const int d1 = 2 * l1 + 1, d2 = 2 * l2 + 1, d3 = 2 * l3 + 1;
                    const int tg = ga.index(l1, l2, l3);
                    if (tg < 0) return fail(c, MIX_EINVAL, "l-triple beyond the Gaunt table");
                    const std::vector<double>& G = ga.G[tg];
                    tcg.push_back(ga.row0[tg]);
                    auto nz_ = [&](int m1, int m2, int m3) { return std::fabs(G[((size_t)m1 * d2 + m2) * d3 + m3]) > GAUNT_ZERO; };
                    auto gv = [&](int m1, int m2, int m3) { return G[((size_t)m1 * d2 + m2) * d3 + m3]; };
                    const int t = (int)(tau.size() / 4);
                    (void)t;
                    tau.push_back(l1);
                    tau.push_back(l2);
                    tau.push_back(l3);
                    tau.push_back((int)goff.size());
                    // ordering by m3 (entries m1 | m2 << 8)
                    for (int m3 = 0; m3 < d3; ++m3) {
                        goff.push_back((int)gidx.size());
                        for (int m1 = 0; m1 < d1; ++m1)
                            for (int m2 = 0; m2 < d2; ++m2)
                                if (nz_(m1, m2, m3)) {
                                    gidx.push_back(m1 | (m2 << 8));
                                    gval.push_back(gv(m1, m2, m3));
                                }
                    }
                    goff.push_back((int)gidx.size());
                    // ordering by m1 (entries m2 | m3 << 8)
                    for (int m1 = 0; m1 < d1; ++m1) {
                        goff.push_back((int)gidx.size());
                        for (int m2 = 0; m2 < d2; ++m2)
                            for (int m3 = 0; m3 < d3; ++m3)
                                if (nz_(m1, m2, m3)) {
                                    gidx.push_back(m2 | (m3 << 8));
                                    gval.push_back(gv(m1, m2, m3));
                                }
                    }
                    goff.push_back((int)gidx.size());
                    // ordering by m2 (entries m1 | m3 << 8)
                    for (int m2 = 0; m2 < d2; ++m2) {
                        goff.push_back((int)gidx.size());
                        for (int m1 = 0; m1 < d1; ++m1)
                            for (int m3 = 0; m3 < d3; ++m3)
                                if (nz_(m1, m2, m3)) {
                                    gidx.push_back(m1 | (m3 << 8));
                                    gval.push_back(gv(m1, m2, m3));
                                }
                    }
                    goff.push_back((int)gidx.size());
                    // masked coefficients c[qa][qb][qc] of the ascending triple
                    // (zero where la == lb and qb < qa, or lb == lc and qc < qb),
                    // stored as W[q1 q2][q3] with (q1, q2, q3) = (qc, qb, qa)
                    const size_t id = ((size_t)la * L1 + lb) * L1 + lc;
                    const double* C3 = a->c3 + id * n * n * n;
                    for (int q1 = 0; q1 < n; ++q1)
                        for (int q2 = 0; q2 < n; ++q2)
                            for (int q3 = 0; q3 < n; ++q3) {
                                const int qa = q3, qb = q2, qc = q1;
                                bool ok = true;
                                if (la == lb && qb < qa) ok = false;
                                if (lb == lc && qc < qb) ok = false;
                                W3.push_back(ok ? C3[((size_t)qa * n + qb) * n + qc] : 0.0);
                            }
                }
    }
    c->ntau = (int)(tau.size() / 4);
    c->gaunt_nnz = 0;
    c->tau_d3_sum = 0;
    int64_t nb3 = 0;
    for (int t = 0; t < c->ntau; ++t) {
        const int l1 = tau[4 * t], l2 = tau[4 * t + 1], l3 = tau[4 * t + 2];
        const int gb = tau[4 * t + 3];
        c->gaunt_nnz += goff[gb + 2 * l3 + 1] - goff[gb];
        c->tau_d3_sum += 2 * l3 + 1;
        const int64_t nn = n;
        nb3 += (l1 == l2 && l2 == l3) ? nn * (nn + 1) * (nn + 2) / 6
               : (l1 == l2 || l2 == l3) ? nn * nn * (nn + 1) / 2 : nn * nn * nn;
    }
    c->basis_size = n + (a->nu_max >= 2 ? (int64_t)L1 * n * (n + 1) / 2 : 0) + nb3;
    // padded layout of the nu = 3 coefficients: W[q1 q2][q3] rows of np (zeros
    // in the padding)
    const int np = (n + 3) & ~3;
    c->np = np;
    // Where two l's of a triple coincide the Gaunt factor is symmetric in the
    // matching (l, m) pairs, so the energy only sees the part of W symmetric in
    // the matching n indices.  Symmetrising W there leaves E unchanged and makes
    // the adjoints through the coinciding factors equal (the kernel then
    // computes one and scales it): tau[4t+3] keeps the Gaunt offset row, the
    // mode goes to tmode[t]: 0 distinct, 1 l1 == l2, 2 l2 == l3, 3 all equal.
    std::vector<int> tmode(c->ntau, 0);
    for (int t = 0; t < c->ntau; ++t) {
        const int l1 = tau[4 * t], l2 = tau[4 * t + 1], l3 = tau[4 * t + 2];
        const int mode = (l1 == l2 && l2 == l3) ? 3 : (l1 == l2 ? 1 : (l2 == l3 ? 2 : 0));
        tmode[t] = mode;
        // the kernel keeps U for distinct l's only, sized for l3 <= L - 2
        if (mode == 0 && 2 * l3 + 1 > std::max(2 * L - 3, 1)) return fail(c, MIX_EINVAL, "l-triple order");
        double* Wt = W3.data() + (size_t)t * n * n * n;
        std::vector<double> S(Wt, Wt + (size_t)n * n * n);
        auto at = [&](int a, int b, int cc) -> double { return Wt[((size_t)a * n + b) * n + cc]; };
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b)
                for (int cc = 0; cc < n; ++cc) {
                    double v = at(a, b, cc);
                    if (mode == 1) v = 0.5 * (at(a, b, cc) + at(b, a, cc));
                    else if (mode == 2) v = 0.5 * (at(a, b, cc) + at(a, cc, b));
                    else if (mode == 3)
                        v = (at(a, b, cc) + at(a, cc, b) + at(b, a, cc) + at(b, cc, a) + at(cc, a, b) + at(cc, b, a)) / 6.0;
                    S[((size_t)a * n + b) * n + cc] = v;
                }
        std::copy(S.begin(), S.end(), Wt);
    }
    c->nu3_flops = 0.0;
    c->nu3_flops_ref = 0.0;
    for (int t = 0; t < c->ntau; ++t) {
        const int l3 = tau[4 * t + 2], gb = tau[4 * t + 3];
        const double nnz = goff[gb + 2 * l3 + 1] - goff[gb], d3 = 2 * l3 + 1, nn = n;
        double f = 4.0 * d3 * nn * nn * nn + 2.0 * nnz * nn * nn + 2.0 * d3 * nn * nn;
        if (tmode[t] != 3) f += 2.0 * nnz * nn * nn;
        if (tmode[t] == 0) f += 2.0 * nnz * nn * nn;
        c->nu3_flops += f;
        // the same count with the factors in ascending order: the dense factor
        // is then the one of largest l (l1 here), and the coincidences swap
        const double d1 = 2 * tau[4 * t] + 1;
        const int mref = tmode[t] == 1 ? 2 : (tmode[t] == 2 ? 1 : tmode[t]);
        double fr = 4.0 * d1 * nn * nn * nn + 2.0 * nnz * nn * nn + 2.0 * d1 * nn * nn;
        if (mref != 3) fr += 2.0 * nnz * nn * nn;
        if (mref == 0) fr += 2.0 * nnz * nn * nn;
        c->nu3_flops_ref += fr;
    }
    // q2 block of a lane unit (q1, qb consecutive q2) in the nu = 3 pass: every
    // pass of the warp over its units repeats the per-m3 work (a warp-wide
    // reduction among it), so choose the block with the least estimated work,
    // passes x (2 qb np multiply-adds + ~120 instructions of per-m3 overhead):
    // 4 or 2 (and for float 6 as well where np = 12: n = 12 gives 24 units in
    // one pass instead of 36 in two)
    {
        std::vector<int> cand = {4, 2};
        if (c->precision != MIX_FP64 && np == 12) cand.push_back(6);
        double best = 0.0;
        for (int qb : cand) {
            const int units = n * (np / qb);
            const double cost = (double)((units + 31) / 32) * (2.0 * qb * np + 120.0);
            if (qb == cand[0] || cost < best - 1e-9) {
                best = cost;
                c->qb = qb;
            }
        }
    }
    std::vector<double> ylmk(nlm);
    for (int l = 0; l <= L; ++l)
        for (int m = -l; m <= l; ++m) ylmk[l * l + l + m] = ylm_norm(l, m);
    std::vector<double> pair(16, 0.0);
    if (a->pair) pair.assign(a->pair, a->pair + 16);
    // cheap-potential coefficient windows (the kernel reads each interval's four
    // control points as one aligned vector)
    std::vector<double> sc2(SPL_W2 * 4), sc3(64 * SPL_W3 * 4);
    for (int q = 0; q < SPL_W2; ++q)
        for (int k = 0; k < 4; ++k) sc2[q * 4 + k] = sp->c2[q + k];
    for (int ab = 0; ab < 64; ++ab)
        for (int z = 0; z < SPL_W3; ++z)
            for (int k = 0; k < 4; ++k) sc3[(ab * SPL_W3 + z) * 4 + k] = sp->c3[ab * 8 + z + k];

    std::vector<int> toff;
    Arena& A = c->arena;
    A.bytes.clear();
    if (c->precision == MIX_FP64) {
        c->o_c1 = A.put(c1);
        c->o_S2 = A.put(S2);
        c->o_tiles = A.put(ace_tiles<double>(n, np, tau, tmode, tcg, goff, gidx, gval, W3, toff, c->tile_max));
        c->o_ylmk = A.put(ylmk);
        c->o_pair = A.put(pair);
        c->o_sc2 = A.put(sc2);
        c->o_sc3 = A.put(sc3);
    } else {
        c->o_c1 = A.put(conv<float>(c1));
        c->o_S2 = A.put(conv<float>(S2));
        c->ace_tcm = c->ntau == 0 ? 0 : (c->precision == MIX_BF16 ? 1 : (c->precision == MIX_BF16_SPLIT ? 2 : 0));
        c->o_tiles = A.put(ace_tiles<float>(n, np, tau, tmode, tcg, goff, gidx, gval, W3, toff, c->tile_max, c->ace_tcm));
        c->o_ylmk = A.put(conv<float>(ylmk));
        c->o_pair = A.put(conv<float>(pair));
        c->o_sc2 = A.put(conv<float>(sc2));
        c->o_sc3 = A.put(conv<float>(sc3));
    }
    c->o_toff = A.put(toff);
    A.bytes.resize(align256(A.bytes.size()));
    return MIX_OK;
}

template <typename T>
void fill_tabs(mix_ctx* c, unsigned char* base, AceTab<T>& at, SplTab<T>& st) {
    at.n = c->n;
    at.L = c->L;
    at.nu = c->nu;
    at.nlm = (c->L + 1) * (c->L + 1);
    at.ntau = c->ntau;
    at.np = c->np;
    at.rc = c->ace_rc;
    at.c1 = reinterpret_cast<const T*>(base + c->o_c1);
    at.S2 = reinterpret_cast<const T*>(base + c->o_S2);
    at.tiles = base + c->o_tiles;
    at.tile_off = reinterpret_cast<const int*>(base + c->o_toff);
    at.tile_max = c->tile_max;
    at.qb = c->qb;
    at.ylmk = reinterpret_cast<const T*>(base + c->o_ylmk);
    at.pair = reinterpret_cast<const T*>(base + c->o_pair);
    at.has_pair = c->has_pair ? 1 : 0;
    st.rc = c->spl_rc;
    st.rc3 = c->spl_rc3;
    st.c2w = reinterpret_cast<const T*>(base + c->o_sc2);
    st.c3w = reinterpret_cast<const T*>(base + c->o_sc3);
    st.rc2 = (T)(c->dev.rcc2);
    st.rc32 = (T)(c->spl_rc3 * c->spl_rc3);
    st.invh2 = (T)(13.0 / c->spl_rc);
    st.invh3 = (T)(5.0 / c->spl_rc3);
    st.invhc = (T)(5.0 / (2.0 * c->spl_rc3));
}

void layout(mix_ctx* c) {
    const size_t N = (size_t)c->sys.n_atoms, cap = (size_t)c->cap, nc = (size_t)c->dev.cells.ncell;
    const size_t v4 = c->precision == MIX_FP64 ? sizeof(double4) : sizeof(float4);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align256(o + std::max<size_t>(bytes, 1));
        return at;
    };
    c->o_status = take(SW_COUNT * sizeof(int));
    c->o_xb = take(N * sizeof(double4));
    c->o_xf = take(N * sizeof(float4));
    c->o_xr = take(N * sizeof(float4));
    c->o_cell3 = take(N * sizeof(int));
    c->o_cell_of = take(N * 4);
    c->o_cell_count = take(nc * 4);
    c->o_cell_start = take((nc + 1) * 4);
    c->o_cell_fill = take(nc * 4);
    c->o_cell_atoms = take(N * 4);
    c->o_nnb = take(N * 4);
    c->o_nbr = take(N * cap * 4);
    c->o_rev = take(N * cap * 4);
    c->o_lam = take(N * 8);
    c->o_wgt = take(N * 8);
    c->o_flags = take(N);
    c->o_act_e = take(N * 4);
    c->o_act_c = take(N * 4);
    c->o_pos_e = take(N * 4);
    c->o_pos_c = take(N * 4);
    c->o_blk_e = take((size_t)c->dev.nblk * 4);
    c->o_blk_c = take((size_t)c->dev.nblk * 4);
    c->o_ge = take(N * cap * v4);
    c->o_gc = take(N * cap * v4);
    c->o_gei = take(N * cap * v4);
    c->o_gci = take(N * cap * v4);
    c->o_ee = take(N * 8);
    c->o_ec = take(N * 8);
    c->o_pe = take(N * sizeof(float2));
    c->o_pc = take(N * sizeof(float2));
    c->o_seed = take(N);
    c->o_core = take(N);
    c->o_zsum = take(N * 4);
    c->off_tab = take(c->arena.bytes.size());
    c->ws_bytes = o;
}

int check_stream_error(mix_ctx* c, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    return MIX_OK;
}

int evals_launches(const mix_ctx* c) { return LAUNCHES_PER_EVAL - 4 + sets_launches(c->seedrule); }

// the kernels of one evaluation, in order, on stream s (events between the
// phases when profiling)
// (captured = true: the events become record nodes of the graph being captured)
void enqueue_evaluation(mix_ctx* c, cudaStream_t s, int integrate, double dt, int force_rebuild, bool prof,
                        bool captured = false) {
    const double h = half_kick(dt, c->sys.mass);
    const unsigned ef = captured ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (prof) cudaEventRecordWithFlags(c->ev[0], s, ef);
    launch_disp(c->dev, s, integrate, dt, h, force_rebuild);
    if (prof) cudaEventRecordWithFlags(c->ev[1], s, ef);
    launch_build(c->dev, s);
    if (prof) cudaEventRecordWithFlags(c->ev[2], s, ef);
    launch_sets(c->dev, c->regions, c->seedrule, s);
    if (prof) cudaEventRecordWithFlags(c->ev[3], s, ef);
    const void* at = c->precision == MIX_FP64 ? (const void*)&c->ace64 : (const void*)&c->ace32;
    const void* st = c->precision == MIX_FP64 ? (const void*)&c->spl64 : (const void*)&c->spl32;
    auto exp_kernel = [&]() {
        if (c->ace_tcm) launch_ace_tc(c->dev, at, c->ace_tcm, c->L, c->ace_smem, c->ace_grid, c->ace_nbuf, s);
        else launch_ace(c->dev, at, c->precision, c->L, c->ace_smem, c->ace_grid, c->ace_wn, s);
    };
    if (c->order == MIX_ORDER_SERIAL) {
        // each kernel has the whole GPU: when the expensive set alone fills
        // every SM, running the two side by side only delays the expensive one
        exp_kernel();
        if (prof) cudaEventRecordWithFlags(c->ev[4], s, ef);
        launch_spline(c->dev, st, c->precision, c->spl_lpa, c->spl_smem, c->spl_grid, s);
        if (prof) cudaEventRecordWithFlags(c->ev[5], s, ef);
    } else {
        // the two potentials write disjoint arrays: the cheap one runs on a
        // second branch, launched before the expensive kernel (so that it takes
        // the SMs a small expensive set leaves idle) or after it (so that it
        // fills the expensive kernel's last wave)
        cudaEventRecord(c->ev_fork, s);
        if (c->order == MIX_ORDER_EXP_FIRST) exp_kernel();
        cudaStreamWaitEvent(c->aux, c->ev_fork, 0);
        launch_spline(c->dev, st, c->precision, c->spl_lpa, c->spl_smem, c->spl_grid, c->aux);
        cudaEventRecord(c->ev_join, c->aux);
        if (c->order == MIX_ORDER_CHEAP_FIRST) exp_kernel();
        if (prof) cudaEventRecordWithFlags(c->ev[4], s, ef);
        cudaStreamWaitEvent(s, c->ev_join, 0);
        if (prof) cudaEventRecordWithFlags(c->ev[5], s, ef);
    }
    launch_gather(c->dev, c->precision, integrate, h, s);
    if (prof) cudaEventRecordWithFlags(c->ev[6], s, ef);
}

void drop_graph(mix_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
}

// Capture one velocity-Verlet step (all its kernels, plus the profiling events
// when enabled) into a CUDA graph on a private stream; replayed by
// cudaGraphLaunch on the context stream.
int capture_step(mix_ctx* c, double dt) {
    drop_graph(c);
    if (!c->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(c, e, "capture stream");
    }
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
    enqueue_evaluation(c, c->cap_stream, 1, dt, 0, c->profiling, true);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    c->graph = g;
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    if (e != cudaSuccess) {
        drop_graph(c);
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    c->graph_dt = dt;
    c->graph_prof = c->profiling;
    c->graph_regions = c->regions_version;
    return MIX_OK;
}

// one force evaluation; integrate = 1 wraps it in a velocity-Verlet step
int evaluate(mix_ctx* c, int integrate, double dt) {
    cudaStream_t s = c->stream;
    const bool prof = c->profiling;
    const bool use_graph = c->opt_graphs && integrate && !c->need_build;
    if (use_graph) {
        if (!c->gexec || c->graph_dt != dt || c->graph_prof != prof || c->graph_regions != c->regions_version) {
            int st = capture_step(c, dt);
            if (st) return st;
        }
        cudaError_t e = cudaGraphLaunch(c->gexec, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
    } else {
        enqueue_evaluation(c, s, integrate, dt, c->need_build ? 1 : 0, prof);
    }
    c->need_build = false;
    c->launches += evals_launches(c);
    int rc = check_stream_error(c, "kernel launch");
    if (rc || !prof) return rc;
    cudaError_t e = cudaEventSynchronize(c->ev[MIX_PHASES]);
    if (e != cudaSuccess) return cuda_fail(c, e, "profile event");
    for (int p = 0; p < MIX_PHASES; ++p) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[p], c->ev[p + 1]);
        c->prof_last[p] = ms;
        c->prof_total[p] += ms;
    }
    c->prof_evals++;
    return MIX_OK;
}

int read_status(mix_ctx* c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
    e = cudaMemcpy(c->pinned, c->dev.status, SW_COUNT * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "status read");
    const int st = c->pinned[SW_STATUS];
    if (st & ST_NBR_OVERFLOW)
        return fail(c, MIX_EOVERFLOW, "neighbour list overflow: %d neighbours, capacity %d", c->pinned[SW_MAXNB], c->cap);
    if (st & ST_NB3_OVERFLOW) {
        const int seen = c->pinned[SW_NB3MAX], lim = spline_nb3(c->spl_lpa), lpa = c->spl_lpa;
        if (lpa < 32 && seen <= spline_nb3(32)) {
            // the cheap kernel's narrow lane groups were chosen from the mean
            // density and this system has denser spots: widen them to a warp for
            // the evaluations that follow (this one is incomplete), clear the flag
            // and make any batch holding the context re-plan
            size_t smem = 0;
            int grid = 0;
            if (spline_configure(c->precision, 32, &smem, &grid) == cudaSuccess) {
                c->spl_lpa = 32;
                c->spl_lpa_settled = true;
                c->spl_smem = smem;
                c->spl_grid = c->spl_grid_max = grid;
                drop_graph(c);
                c->regions_version++;
                int w[2] = {st & ~ST_NB3_OVERFLOW, 0};
                cudaMemcpy(c->dev.status + SW_STATUS, &w[0], sizeof(int), cudaMemcpyHostToDevice);
                cudaMemcpy(c->dev.status + SW_NB3MAX, &w[1], sizeof(int), cudaMemcpyHostToDevice);
                return fail(c, MIX_EOVERFLOW,
                            "three-body neighbours %d exceeded the %d of %d-lane groups; the context now "
                            "evaluates the cheap potential with a warp per atom: repeat the evaluation",
                            seen, lim, lpa);
            }
        }
        return fail(c, MIX_EOVERFLOW, "three-body neighbours %d exceed %d", seen, lim);
    }
    if (st & ST_NONFINITE) return fail(c, MIX_ENUMERIC, "non-finite position or force");
    if (st & ST_OUT_OF_BOX) return fail(c, MIX_EBOX, "an atom left the box in a non-periodic dimension");
    if (st & ST_REV_MISSING) return fail(c, MIX_EINVAL, "asymmetric neighbour list");
    if (st & ST_TC_TIMEOUT) return fail(c, MIX_ETIMEOUT, "a wait for the tensor-core readout gave up");
    // The uniform-density estimate behind the initial lane groups overstates
    // open lattices (diamond holds half of it inside 3.4 A).  Once an
    // evaluation has measured the largest 3-body count, a periodic bulk moves
    // to the narrowest group whose on-chip slots hold twice that count.  No
    // result depends on the width (every sum keeps its order), and an overflow
    // widens the groups again; this happens once per context.
    if (!c->spl_lpa_settled && c->spl_bulk && c->spl_lpa > 8 && c->pinned[SW_NB3MAX] > 0) {
        c->spl_lpa_settled = true;
        const int seen = c->pinned[SW_NB3MAX];
        int want = c->spl_lpa;
        for (int l : {16, 8})
            if (l < want && 2 * seen <= spline_nb3(l)) want = l;
        size_t smem = 0;
        int grid = 0;
        if (want < c->spl_lpa && spline_configure(c->precision, want, &smem, &grid) == cudaSuccess) {
            c->spl_lpa = want;
            c->spl_smem = smem;
            c->spl_grid = c->spl_grid_max = grid;
            drop_graph(c);
            c->regions_version++;   // any batch holding the context re-plans
        }
    }
    return MIX_OK;
}

int copy_out(mix_ctx* c, void* dst, const void* src, size_t bytes) {
    if (!dst || bytes == 0) return MIX_OK;
    cudaError_t e = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy D2H");
    return MIX_OK;
}

}  // namespace

extern "C" {

int mix_init(const mix_system* sys, const mix_ace* a, const mix_spline* sp, const mix_options* opt,
             void* cuda_stream, mix_ctx** out) {
    if (!out) return MIX_EINVAL;
    *out = nullptr;
    if (!sys || !a || !sp || !opt) return MIX_EINVAL;
    mix_ctx* c = new (std::nothrow) mix_ctx();
    if (!c) return MIX_ENOMEM;
    auto bad = [&](const char* msg) {
        delete c;
        (void)msg;
        return MIX_EINVAL;
    };
    if (sys->n_atoms < 0 || sys->n_atoms > (int64_t)INT32_MAX / MAX_CAP) return bad("n_atoms");
    if (!(sys->mass > 0)) return bad("mass");
    if (a->n_rad < 1 || a->n_rad > MIX_MAX_NRAD || a->l_max < 0 || a->l_max > MIX_MAX_LMAX || a->nu_max < 1 ||
        a->nu_max > 3 || !(a->r_cut > 0) || !a->c1 || (a->nu_max >= 2 && !a->c2) || (a->nu_max >= 3 && !a->c3))
        return bad("expensive potential");
    if (!(sp->r_cut > 0) || !(sp->r_cut3 > 0) || sp->r_cut3 > sp->r_cut || !sp->c2 || !sp->c3)
        return bad("cheap potential");
    for (int p = 0; p < 8; ++p)
        for (int q = 0; q < 8; ++q)
            for (int r = 0; r < 8; ++r)
                if (sp->c3[(p * 8 + q) * 8 + r] != sp->c3[(q * 8 + p) * 8 + r]) return bad("c3 not symmetric");
    if (opt->precision != MIX_FP64 && opt->precision != MIX_FP32 && opt->precision != MIX_BF16 &&
        opt->precision != MIX_BF16_SPLIT)
        return bad("precision");
    if (!(opt->skin > 0)) return bad("skin");
    if (opt->blend != MIX_BLEND_LINEAR && opt->blend != MIX_BLEND_CUBIC) return bad("blend");
    c->sys = *sys;
    c->opt = *opt;
    c->opt_graphs = opt->no_graphs == 0;
    if (opt->potential_order < MIX_ORDER_CHEAP_FIRST || opt->potential_order > MIX_ORDER_SERIAL)
        return bad("potential_order");
    c->order = opt->potential_order;
    c->precision = opt->precision;
    c->ace_rc = a->r_cut;
    c->n = a->n_rad;
    c->L = a->l_max;
    c->nu = a->nu_max;
    c->has_pair = a->pair != nullptr;
    c->spl_rc = sp->r_cut;
    c->spl_rc3 = sp->r_cut3;
    c->stream = (cudaStream_t)cuda_stream;
    const double rcmax = std::max(a->r_cut, sp->r_cut);
    c->rlist = rcmax + opt->skin;
    const double bufe = opt->buffer_exp > 0 ? opt->buffer_exp : a->r_cut;
    const double bufc = opt->buffer_cheap > 0 ? opt->buffer_cheap : sp->r_cut;
    if (bufe > rcmax || bufc > rcmax) return bad("buffer radius beyond the neighbour range");

    Dev& d = c->dev;
    std::memset(&d, 0, sizeof d);
    d.n = sys->n_atoms;
    d.mass = sys->mass;
    double vol = 1.0;
    for (int k = 0; k < 3; ++k) {
        if (!(sys->box_len[k] > 0)) return bad("box");
        d.box.lo[k] = sys->box_lo[k];
        d.box.L[k] = sys->box_len[k];
        d.box.invL[k] = 1.0 / sys->box_len[k];
        d.box.per[k] = sys->periodic[k] ? 1 : 0;
        // checked as a double before it becomes an int (at most 1023 cells a dimension)
        if (!(sys->box_len[k] / c->rlist < 1024.0)) return bad("more than 1023 cells along one dimension");
        int ncd = (int)std::floor(sys->box_len[k] / c->rlist);
        if (d.box.per[k]) {
            if (sys->box_lo[k] != 0.0) return bad("periodic box_lo must be 0");
            if (ncd < 3 || sys->box_len[k] < 2.0 * c->rlist) return bad("periodic box too small");
        } else if (ncd < 1) {
            ncd = 1;
        }
        d.cells.nc[k] = ncd;
        d.cells.invh[k] = (double)ncd / sys->box_len[k];
        d.cells.h[k] = sys->box_len[k] / (double)ncd;
        d.cells.hf[k] = (float)d.cells.h[k];
        if (ncd > 1023) return bad("more than 1023 cells along one dimension");
        vol *= sys->box_len[k];
    }
    const int64_t ncell = (int64_t)d.cells.nc[0] * d.cells.nc[1] * d.cells.nc[2];
    if (ncell > (1 << 26)) return bad("too many cells");
    d.cells.ncell = (int)ncell;
    const double rho_mean = vol > 0 ? (double)sys->n_atoms / vol : 0.0;
    const double expect = rho_mean * 4.0 / 3.0 * M_PI * c->rlist * c->rlist * c->rlist;
    // gather lane groups from the mean list length (not the capacity, so that the
    // order of every sum, and with it every result, is independent of it)
    d.gat_lpa = expect <= 40.0 ? 8 : (expect <= 80.0 ? 16 : 32);
    if (opt->nbr_cap > 0) {
        c->cap = opt->nbr_cap;
    } else {
        int cap = (int)std::ceil(1.4 * expect + 16.0);
        cap = std::max(cap, 64);
        c->cap = ((cap + 31) / 32) * 32;
    }
    if (c->cap > MAX_CAP) c->cap = MAX_CAP;
    if (c->cap < 1) return bad("nbr_cap");
    d.cap = c->cap;
    d.rlist2 = c->rlist * c->rlist;
    d.half_skin2 = 0.25 * opt->skin * opt->skin;
    d.rce = a->r_cut;
    d.rce2 = a->r_cut * a->r_cut;
    d.rcc = sp->r_cut;
    d.rcc2 = sp->r_cut * sp->r_cut;
    d.rc3 = sp->r_cut3;
    d.bufe2 = bufe * bufe;
    d.bufc2 = bufc * bufc;
    d.bufe = bufe;
    d.bufc = bufc;
    d.bufe2_lo = (float)(d.bufe2 - 1e-3);
    d.bufe2_hi = (float)(d.bufe2 + 1e-3);
    d.bufc2_lo = (float)(d.bufc2 - 1e-3);
    d.bufc2_hi = (float)(d.bufc2 + 1e-3);
    double extent = 0.0;
    for (int k = 0; k < 3; ++k) extent = std::max(extent, std::fabs(sys->box_lo[k]) + sys->box_len[k]);
    d.exact_lists = extent > 2000.0 ? 1 : 0;
    const int64_t nblk = (sys->n_atoms + SCAN_BLOCK - 1) / SCAN_BLOCK;
    d.nblk = (int)(nblk > 0 ? nblk : 1);
    std::memset(&c->regions, 0, sizeof c->regions);
    c->regions.blend = opt->blend;
    int st = build_tables(c, a, sp);
    if (st == MIX_OK && c->ntau > 0) st = gaunt_upload();
    if (st) {
        delete c;
        return st;
    }
    layout(c);
    // large float systems: CTAs of 4 warps share the coefficient tiles between
    // twice the atoms, so more warps fit an SM (their expensive sets are many
    // waves large); small sets keep groups of 2, which spread them more evenly
    c->ace_wn = (c->precision != MIX_FP64 && sys->n_atoms >= 50000) ? ACE_MAX_WARPS : ACE_GROUP;
    cudaError_t e = c->ace_tcm
                        ? ace_tc_configure(c->ace_tcm, c->L, c->n, c->cap, c->tile_max, c->qb, &c->ace_smem,
                                           &c->ace_grid, &c->ace_nbuf)
                        : ace_configure(c->precision, c->L, c->n, c->cap, c->tile_max, c->qb, &c->ace_smem,
                                        &c->ace_grid, c->ace_wn);
    if (e != cudaSuccess) {
        delete c;
        return e == cudaErrorInvalidValue ? MIX_EINVAL : MIX_ECUDA;
    }
    // Fewer lanes per cheap atom where atoms have few neighbours: in a periodic
    // bulk whose mean count inside the 3-body cutoff is at most a third of what
    // the group holds on chip, a quarter warp (16 slots) up to 5.3 or half a warp
    // (24 slots) up to 8; a warp (32 slots) otherwise.  Si has about 5, bcc Fe 12.
    {
        bool bulk = vol > 0;
        for (int k = 0; k < 3; ++k) bulk = bulk && sys->periodic[k];
        const double rho = vol > 0 ? (double)sys->n_atoms / vol : 0.0;
        const double n3 = rho * 4.0 / 3.0 * M_PI * sp->r_cut3 * sp->r_cut3 * sp->r_cut3;
        c->spl_lpa = !bulk ? 32 : (n3 * 3.0 <= spline_nb3(8) ? 8 : (n3 * 3.0 <= spline_nb3(16) ? 16 : 32));
        c->spl_bulk = bulk;
    }
    e = spline_configure(c->precision, c->spl_lpa, &c->spl_smem, &c->spl_grid);
    c->ace_grid_max = c->ace_grid;
    c->spl_grid_max = c->spl_grid;
    if (e != cudaSuccess) {
        delete c;
        return MIX_ECUDA;
    }
    e = cudaMallocHost((void**)&c->pinned, SW_COUNT * sizeof(int));
    if (e != cudaSuccess) {
        delete c;
        return MIX_ECUDA;
    }
    e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaFreeHost(c->pinned);
        delete c;
        return MIX_ECUDA;
    }
    c->bound = false;
    c->need_build = true;
    c->forces_valid = false;
    c->steps = 0;
    *out = c;
    return MIX_OK;
}

int mix_workspace_bytes(const mix_ctx* c, size_t* bytes) {
    if (!c || !bytes) return MIX_EINVAL;
    *bytes = c->ws_bytes;
    return MIX_OK;
}

int mix_bind(mix_ctx* c, double* x, double* v, double* f, void* ws) {
    if (!c) return MIX_EINVAL;
    if (c->sys.n_atoms > 0 && (!x || !v || !f)) return fail(c, MIX_EINVAL, "null state buffer");
    if (!ws) return fail(c, MIX_EINVAL, "null workspace");
    if (((uintptr_t)x | (uintptr_t)v | (uintptr_t)f) & 15) return fail(c, MIX_EINVAL, "state buffers must be 16-byte aligned");
    if ((uintptr_t)ws & 255) return fail(c, MIX_EINVAL, "workspace must be 256-byte aligned");
    unsigned char* w = static_cast<unsigned char*>(ws);
    Dev& d = c->dev;
    d.x = reinterpret_cast<double4*>(x);
    d.v = reinterpret_cast<double4*>(v);
    d.f = reinterpret_cast<double4*>(f);
    d.status = reinterpret_cast<int*>(w + c->o_status);
    d.xb = reinterpret_cast<double4*>(w + c->o_xb);
    d.xf = reinterpret_cast<float4*>(w + c->o_xf);
    d.xr = reinterpret_cast<float4*>(w + c->o_xr);
    d.cell3 = reinterpret_cast<int*>(w + c->o_cell3);
    d.cell_of = reinterpret_cast<int*>(w + c->o_cell_of);
    d.cell_count = reinterpret_cast<int*>(w + c->o_cell_count);
    d.cell_start = reinterpret_cast<int*>(w + c->o_cell_start);
    d.cell_fill = reinterpret_cast<int*>(w + c->o_cell_fill);
    d.cell_atoms = reinterpret_cast<int*>(w + c->o_cell_atoms);
    d.nnb = reinterpret_cast<int*>(w + c->o_nnb);
    d.nbr = reinterpret_cast<int*>(w + c->o_nbr);
    d.rev = reinterpret_cast<int*>(w + c->o_rev);
    d.lam = reinterpret_cast<double*>(w + c->o_lam);
    d.wgt = reinterpret_cast<double*>(w + c->o_wgt);
    d.flags = reinterpret_cast<uint8_t*>(w + c->o_flags);
    d.act_e = reinterpret_cast<int*>(w + c->o_act_e);
    d.act_c = reinterpret_cast<int*>(w + c->o_act_c);
    d.pos_e = reinterpret_cast<int*>(w + c->o_pos_e);
    d.pos_c = reinterpret_cast<int*>(w + c->o_pos_c);
    d.blk_e = reinterpret_cast<int*>(w + c->o_blk_e);
    d.blk_c = reinterpret_cast<int*>(w + c->o_blk_c);
    d.ge = w + c->o_ge;
    d.gc = w + c->o_gc;
    d.ge_in = w + c->o_gei;
    d.gc_in = w + c->o_gci;
    d.esite_e = reinterpret_cast<double*>(w + c->o_ee);
    d.esite_c = reinterpret_cast<double*>(w + c->o_ec);
    d.epark_e = reinterpret_cast<float2*>(w + c->o_pe);
    d.epark_c = reinterpret_cast<float2*>(w + c->o_pc);
    d.seed = reinterpret_cast<uint8_t*>(w + c->o_seed);
    d.core = reinterpret_cast<uint8_t*>(w + c->o_core);
    d.zsum = reinterpret_cast<int*>(w + c->o_zsum);
    unsigned char* tb = w + c->off_tab;
    fill_tabs<double>(c, tb, c->ace64, c->spl64);
    fill_tabs<float>(c, tb, c->ace32, c->spl32);
    cudaError_t e = cudaMemsetAsync(d.status, 0, SW_COUNT * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.cell_count, 0, (size_t)d.cells.ncell * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.seed, 0, (size_t)d.n, c->stream);
    // incoming rows carry the epoch of the evaluation that wrote them; zero is never current
    if (e == cudaSuccess) e = cudaMemsetAsync(d.ge_in, 0, c->o_gci - c->o_gei, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.gc_in, 0, c->o_gci - c->o_gei, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tb, c->arena.bytes.data(), c->arena.bytes.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mix_bind");
    drop_graph(c);
    c->bound = true;
    c->regions_version++;      // batches holding this context re-read its buffers
    c->need_build = true;
    c->forces_valid = false;
    c->steps = 0;
    c->launches = 0;
    return MIX_OK;
}

int mix_set_regions(mix_ctx* c, const mix_region* r, int n) {
    if (!c) return MIX_EINVAL;
    if (n < 0 || n > MIX_MAX_REGIONS || (n > 0 && !r)) return fail(c, MIX_EINVAL, "region count");
    Regions R;
    std::memset(&R, 0, sizeof R);
    R.n = n;
    R.blend = c->opt.blend;
    for (int k = 0; k < n; ++k) {
        if (r[k].kind != MIX_REGION_SPHERE && r[k].kind != MIX_REGION_CYLINDER)
            return fail(c, MIX_EINVAL, "region kind");
        if (!(r[k].r_core >= 0) || !(r[k].ramp >= 0)) return fail(c, MIX_EINVAL, "region radii");
        double* q = R.r[k];
        q[0] = r[k].kind;
        q[1] = r[k].centre[0];
        q[2] = r[k].centre[1];
        q[3] = r[k].centre[2];
        const double ax = r[k].axis[0], ay = r[k].axis[1], az = r[k].axis[2];
        const double nrm = std::sqrt(ax * ax + ay * ay + az * az);
        if (r[k].kind == MIX_REGION_CYLINDER && !(nrm > 0)) return fail(c, MIX_EINVAL, "cylinder axis");
        q[4] = nrm > 0 ? ax / nrm : ax;
        q[5] = nrm > 0 ? ay / nrm : ay;
        q[6] = nrm > 0 ? az / nrm : az;
        q[7] = r[k].r_core;
        q[8] = r[k].ramp;
        for (int t = 0; t < 3; ++t) {
            R.cf[k][t] = (float)q[1 + t];
            R.cf[k][3 + t] = (float)q[4 + t];
        }
        const double far = r[k].r_core + r[k].ramp + c->dev.bufe + std::sqrt(c->dev.half_skin2) + 0.01;
        R.far2[k] = (float)(far * far);
    }
    R.screen = c->dev.exact_lists ? 0 : 1;
    for (int t = 0; t < 3; ++t) {
        R.Lf[t] = (float)c->dev.box.L[t];
        R.iLf[t] = (float)c->dev.box.invL[t];
    }
    c->regions = R;
    c->seedrule.mode = 0;
    c->regions_version++;
    c->forces_valid = false;
    return MIX_OK;
}

int mix_forces(mix_ctx* c) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "mix_forces before mix_bind");
    int st = evaluate(c, 0, 0.0);
    if (st) return st;
    c->forces_valid = true;
    return MIX_OK;
}

int mix_step(mix_ctx* c, double dt, int nsteps) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "mix_step before mix_bind");
    if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt)) return fail(c, MIX_EINVAL, "dt / nsteps");
    if (!c->forces_valid) {
        int st = evaluate(c, 0, 0.0);
        if (st) return st;
        c->forces_valid = true;
    }
    for (int s = 0; s < nsteps; ++s) {
        int st = evaluate(c, 1, dt);
        if (st) return st;
        c->steps++;
    }
    return MIX_OK;
}

int mix_step_host(mix_ctx* c, double* xh, double* vh, double* fh, double dt, int nsteps) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "mix_step_host before mix_bind");
    const size_t bytes = (size_t)c->sys.n_atoms * sizeof(double4);
    if (bytes && (!xh || !vh)) return fail(c, MIX_EINVAL, "null host buffer");
    cudaError_t e = cudaMemcpyAsync(c->dev.x, xh, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->dev.v, vh, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && fh) e = cudaMemcpyAsync(c->dev.f, fh, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mix_step_host upload");
    c->forces_valid = fh != nullptr;
    int st = mix_step(c, dt, nsteps);
    if (st) return st;
    e = cudaMemcpyAsync(xh, c->dev.x, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vh, c->dev.v, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && fh) e = cudaMemcpyAsync(fh, c->dev.f, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mix_step_host download");
    return read_status(c);
}

int mix_sync(mix_ctx* c) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return MIX_OK;
    return read_status(c);
}

int mix_get_stats(mix_ctx* c, mix_stats* s) {
    if (!c || !s) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "not bound");
    int st = read_status(c);
    const int* p = c->pinned;
    s->n_core = p[SW_NCORE];
    s->n_ramp = p[SW_NRAMP];
    s->n_exp = p[SW_NEXP];
    s->n_cheap = p[SW_NCHEAP];
    s->rebuilds = p[SW_REBUILDS];
    s->steps = c->steps;
    s->max_neighbours = p[SW_MAXNB];
    s->status_bits = p[SW_STATUS];
    return st;
}

int mix_get_cells(mix_ctx* c, int* ncell3, int* cell_of) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "not bound");
    int st = read_status(c);
    if (st) return st;
    if (ncell3)
        for (int k = 0; k < 3; ++k) ncell3[k] = c->dev.cells.nc[k];
    return copy_out(c, cell_of, c->dev.cell_of, (size_t)c->sys.n_atoms * 4);
}

int mix_get_neighbours(mix_ctx* c, int* cap_out, int* nnb, int* nbr, int* rev) {
    if (!c) return MIX_EINVAL;
    if (cap_out) *cap_out = c->cap;
    if (!c->bound) return fail(c, MIX_ESTATE, "not bound");
    int st = read_status(c);
    if (st) return st;
    const size_t N = (size_t)c->sys.n_atoms;
    st = copy_out(c, nnb, c->dev.nnb, N * 4);
    if (!st) st = copy_out(c, nbr, c->dev.nbr, N * c->cap * 4);
    if (!st) st = copy_out(c, rev, c->dev.rev, N * c->cap * 4);
    return st;
}

int mix_get_lambda(mix_ctx* c, double* lam, double* w) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "not bound");
    int st = read_status(c);
    if (st) return st;
    const size_t N = (size_t)c->sys.n_atoms;
    st = copy_out(c, lam, c->dev.lam, N * 8);
    if (!st) st = copy_out(c, w, c->dev.wgt, N * 8);
    return st;
}

int mix_get_sets(mix_ctx* c, uint8_t* flags, int* act_e, int64_t* n_e, int* act_c, int64_t* n_c) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "not bound");
    int st = read_status(c);
    if (st) return st;
    const size_t N = (size_t)c->sys.n_atoms;
    const int ne = c->pinned[SW_NEXP], nch = c->pinned[SW_NCHEAP];
    if (n_e) *n_e = ne;
    if (n_c) *n_c = nch;
    st = copy_out(c, flags, c->dev.flags, N);
    if (!st) st = copy_out(c, act_e, c->dev.act_e, (size_t)ne * 4);
    if (!st) st = copy_out(c, act_c, c->dev.act_c, (size_t)nch * 4);
    return st;
}

int mix_get_site_energies(mix_ctx* c, double* ee, double* ec) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "not bound");
    int st = read_status(c);
    if (st) return st;
    const size_t N = (size_t)c->sys.n_atoms;
    st = copy_out(c, ee, c->dev.esite_e, N * 8);
    if (!st) st = copy_out(c, ec, c->dev.esite_c, N * 8);
    return st;
}

int mix_get_state(mix_ctx* c, double* x, double* v, double* f, int64_t* step) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "not bound");
    int st = read_status(c);
    const size_t bytes = (size_t)c->sys.n_atoms * sizeof(double4);
    int s2 = copy_out(c, x, c->dev.x, bytes);
    if (!s2) s2 = copy_out(c, v, c->dev.v, bytes);
    if (!s2) s2 = copy_out(c, f, c->dev.f, bytes);
    if (step) *step = c->steps;
    return st ? st : s2;
}

int mix_set_state(mix_ctx* c, const double* x, const double* v, const double* f, int64_t step, int forces_valid) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "not bound");
    const size_t bytes = (size_t)c->sys.n_atoms * sizeof(double4);
    cudaError_t e = cudaSuccess;
    if (x) e = cudaMemcpyAsync(c->dev.x, x, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && v) e = cudaMemcpyAsync(c->dev.v, v, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && f) e = cudaMemcpyAsync(c->dev.f, f, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mix_set_state");
    c->steps = step;
    c->need_build = true;
    c->forces_valid = forces_valid && f;
    return MIX_OK;
}

int mix_destroy(mix_ctx* c) {
    if (!c) return MIX_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    drop_graph(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->profiling)
        for (int p = 0; p <= MIX_PHASES; ++p) cudaEventDestroy(c->ev[p]);
    delete c;
    return MIX_OK;
}

int mix_get_info(const mix_ctx* c, mix_info* info) {
    if (!c || !info) return MIX_EINVAL;
    info->nbr_cap = c->cap;
    info->n_tau = c->ntau;
    info->gaunt_nnz = c->gaunt_nnz;
    info->tau_dim3_sum = c->tau_d3_sum;
    info->basis_size = c->basis_size;
    info->nu3_flops_per_atom = c->nu3_flops;
    info->workspace_bytes = c->ws_bytes;
    info->exp_smem_bytes = c->ace_smem;
    info->exp_grid = c->ace_grid;
    info->exp_threads = 32 * (c->ace_tcm ? TC_ACE_WARPS : c->ace_wn);
    info->cheap_smem_bytes = c->spl_smem;
    info->cheap_grid = c->spl_grid;
    info->launches_per_evaluation = evals_launches(c);
    info->launches = c->launches;
    info->gather_grid = c->dev.grid_gather;
    info->build_grid = c->dev.grid_build;
    info->buffer_grid = c->dev.grid_buffer;
    info->exp_tensor_cores = c->ace_tcm ? 1 : 0;
    info->tc_flops_per_atom = c->ace_tcm ? 2.0 * (double)c->tau_d3_sum * c->n * c->n * c->n : 0.0;
    info->cheap_lanes = c->spl_lpa;
    info->nu3_flops_ref_per_atom = c->nu3_flops_ref;
    info->potential_order = c->order;
    return MIX_OK;
}

int mix_profile(mix_ctx* c, int enable) {
    if (!c) return MIX_EINVAL;
    if ((enable != 0) != c->profiling) {
        cudaStreamSynchronize(c->stream);
        drop_graph(c);
    }
    if (enable && !c->profiling) {
        for (int p = 0; p <= MIX_PHASES; ++p) {
            cudaError_t e = cudaEventCreate(&c->ev[p]);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventCreate");
        }
        c->profiling = true;
    } else if (!enable && c->profiling) {
        cudaStreamSynchronize(c->stream);
        for (int p = 0; p <= MIX_PHASES; ++p) cudaEventDestroy(c->ev[p]);
        c->profiling = false;
    }
    for (int p = 0; p < MIX_PHASES; ++p) c->prof_total[p] = c->prof_last[p] = 0.0;
    c->prof_evals = 0;
    return MIX_OK;
}

int mix_get_profile(mix_ctx* c, double* total_ms, double* last_ms, int64_t* evaluations) {
    if (!c) return MIX_EINVAL;
    for (int p = 0; p < MIX_PHASES; ++p) {
        if (total_ms) total_ms[p] = c->prof_total[p];
        if (last_ms) last_ms[p] = c->prof_last[p];
    }
    if (evaluations) *evaluations = c->prof_evals;
    return MIX_OK;
}

int mix_fma_peak(int precision, void* stream, double* flops) {
    if (!flops || (precision != MIX_FP64 && precision != MIX_FP32)) return MIX_EINVAL;
    return fma_peak(precision, (cudaStream_t)stream, flops);
}

int mix_tc_selftest(const void* a_dev, const void* b_dev, int m, int n, int k, float* d_dev, int* status_dev,
                    void* stream) {
    if (!a_dev || !b_dev || !d_dev || !status_dev) return MIX_EINVAL;
    if ((m != 64 && m != 128) || n < 16 || n > 256 || n % 16 || k < 16 || k > 160 || k % 16) return MIX_EINVAL;
    const cudaError_t e = tc_selftest(static_cast<const uint16_t*>(a_dev), static_cast<const uint16_t*>(b_dev), m,
                                      n, k, d_dev, status_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? MIX_OK : MIX_ECUDA;
}

const char* mix_strerror(int code) {
    switch (code) {
        case MIX_OK: return "ok";
        case MIX_EINVAL: return "invalid argument";
        case MIX_ENOMEM: return "out of memory";
        case MIX_ECUDA: return "CUDA error";
        case MIX_EOVERFLOW: return "capacity overflow";
        case MIX_ETIMEOUT: return "device wait timed out";
        case MIX_ENUMERIC: return "non-finite value";
        case MIX_ESTATE: return "call out of order";
        case MIX_EBOX: return "atom outside a non-periodic box dimension";
    }
    return "unknown status";
}

const char* mix_last_error(const mix_ctx* c) { return c ? c->err.c_str() : ""; }

}  // extern "C"

// ---------------------------------------------------------------------------
// autotuning and batches

namespace {

// One force evaluation captured as a graph: the form in which mix_step replays
// its steps, so that the tuner times the candidates as they will run (the
// order in which the two potential kernels reach the SMs differs between
// graph replays and launches on streams).
int capture_eval(mix_ctx* c, cudaGraphExec_t* out) {
    *out = nullptr;
    if (!c->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(c, e, "capture stream");
    }
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
    enqueue_evaluation(c, c->cap_stream, 0, 0.0, 0, false, true);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    return MIX_OK;
}

// median duration (ms) of `reps` force evaluations at the current positions
// (integrate = 0 leaves x, v and f as they are), after one untimed evaluation;
// with graphs enabled each is a replay of one captured evaluation
int time_force_evals(mix_ctx* c, int reps, float* ms) {
    int st = evaluate(c, 0, 0.0);
    if (st) return st;
    c->forces_valid = true;
    cudaGraphExec_t gx = nullptr;
    if (c->opt_graphs) {
        st = capture_eval(c, &gx);
        if (st) return st;
        cudaError_t e = cudaGraphLaunch(gx, c->stream);   // once untimed
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(gx);
            return cuda_fail(c, e, "tuning");
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (gx) cudaGraphExecDestroy(gx);
        return fail(c, MIX_ECUDA, "event");
    }
    std::vector<float> v;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, c->stream);
        if (gx) cudaGraphLaunch(gx, c->stream);
        else enqueue_evaluation(c, c->stream, 0, 0.0, 0, false);
        cudaEventRecord(e1, c->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (gx) cudaGraphExecDestroy(gx);
            return cuda_fail(c, e, "tuning");
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        v.push_back(t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (gx) cudaGraphExecDestroy(gx);
    std::sort(v.begin(), v.end());
    *ms = v.empty() ? 0.f : v[v.size() / 2];
    return check_stream_error(c, "tuning");
}

// Coordinate descent over candidate values of one launch parameter.
int tune_param(mix_ctx* c, int reps, int* param, const std::vector<int>& cand) {
    int best = *param;
    float tbest = 1e30f;
    for (int v : cand) {
        if (v < 1) continue;
        *param = v;
        float t = 0.f;
        int st = time_force_evals(c, reps, &t);
        if (st) return st;
        if (t < tbest) {
            tbest = t;
            best = v;
        }
    }
    *param = best;
    return MIX_OK;
}

// The cheap kernel's lane groups: besides the current width, each narrower
// group whose on-chip 3-body slots the largest count measured so far fills to
// at most two thirds (so a local rise of half that count still fits; beyond
// it the evaluation reports MIX_EOVERFLOW and the groups widen again), in any
// system, periodic or not; the fastest is kept.  The forces do not depend on
// the width (every per-slot sum keeps its order).
int tune_cheap_lanes(mix_ctx* c, int reps) {
    const int seen = c->pinned[SW_NB3MAX], lpa0 = c->spl_lpa;
    if (seen <= 0) return MIX_OK;
    std::vector<int> lanes = {lpa0};
    for (int l : {16, 8})
        if (l < lpa0 && 3 * seen <= 2 * spline_nb3(l)) lanes.push_back(l);
    if (lanes.size() < 2) return MIX_OK;
    const size_t smem0 = c->spl_smem;
    const int grid0 = c->spl_grid, gmax0 = c->spl_grid_max;
    int best = lpa0;
    float tbest = 1e30f;
    for (int l : lanes) {
        size_t smem = 0;
        int grid = 0;
        if (spline_configure(c->precision, l, &smem, &grid) != cudaSuccess) continue;
        c->spl_lpa = l;
        c->spl_smem = smem;
        c->spl_grid = c->spl_grid_max = grid;
        float t = 0.f;
        const int st = time_force_evals(c, reps, &t);
        if (st) return st;
        if (t < tbest) {
            tbest = t;
            best = l;
        }
    }
    if (best == lpa0) {
        c->spl_lpa = lpa0;
        c->spl_smem = smem0;
        c->spl_grid = grid0;
        c->spl_grid_max = gmax0;
        return MIX_OK;
    }
    size_t smem = 0;
    int grid = 0;
    cudaError_t e = spline_configure(c->precision, best, &smem, &grid);
    if (e != cudaSuccess) return cuda_fail(c, e, "cheap kernel shape");
    c->spl_lpa = best;
    c->spl_smem = smem;
    c->spl_grid = c->spl_grid_max = grid;
    c->spl_lpa_settled = true;
    c->regions_version++;   // any batch holding the context re-plans
    return MIX_OK;
}

void set_grid_divisor(mix_ctx* c, int div) {
    c->ace_grid = std::max(1, c->ace_grid_max / div);
    c->spl_grid = std::max(1, c->spl_grid_max / div);
    c->dev.grid_gather = std::max(1, sm_count() * 8 / div);
    c->dev.grid_buffer = std::max(1, sm_count() * 8 / div);
    drop_graph(c);
}

// Seed state advanced by every evaluation under the coordination rule; the
// tuners' extra evaluations must leave it as they found it.
struct SeedSave {
    bool active = false;
    std::vector<uint8_t> seed;
    std::vector<int> zsum;
    int evals = 0;
};

int seed_save(mix_ctx* c, SeedSave* s) {
    s->active = c->seedrule.mode == 2;
    if (!s->active) return MIX_OK;
    const size_t N = (size_t)c->sys.n_atoms;
    s->seed.resize(N);
    s->zsum.resize(N);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && N) e = cudaMemcpy(s->seed.data(), c->dev.seed, N, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && N) e = cudaMemcpy(s->zsum.data(), c->dev.zsum, N * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&s->evals, c->dev.status + SW_EVALS, 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MIX_OK : cuda_fail(c, e, "seed state save");
}

int seed_restore(mix_ctx* c, const SeedSave& s) {
    if (!s.active) return MIX_OK;
    const size_t N = (size_t)c->sys.n_atoms;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && N) e = cudaMemcpy(c->dev.seed, s.seed.data(), N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && N) e = cudaMemcpy(c->dev.zsum, s.zsum.data(), N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->dev.status + SW_EVALS, &s.evals, 4, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? MIX_OK : cuda_fail(c, e, "seed state restore");
}

// one member evaluation captured into a (not instantiated) graph
int member_graph(mix_ctx* c, int integrate, double dt, cudaGraph_t* g) {
    if (!c->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(c, e, "capture stream");
    }
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
    enqueue_evaluation(c, c->cap_stream, integrate, dt, 0, false, true);
    e = cudaStreamEndCapture(c->cap_stream, g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    return MIX_OK;
}

}  // namespace

struct mix_batch {
    std::vector<mix_ctx*> m;
    std::vector<int64_t> regions_seen;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double dt = 0.0;
    int divisor = 1;
    std::string err;
    // fused multi-system step: one launch per kernel for all members
    int want_fused = 1;              // use it whenever the members allow
    bool graph_fused = false;        // the current graph is the fused step
    cudaStream_t cap_stream = nullptr;
    unsigned char* dmem = nullptr;   // plan arrays (device)
    BatchPlan plan{};
    int precision = 0;
    struct Group {
        int L, n, cap, tile_max, qb;   // qb: the smallest unit block of the members
        size_t base, smem;
        int grid;
    };
    std::vector<Group> groups;
    const Dev* ddevs = nullptr;
    const void* dace = nullptr;
    const void* dspl = nullptr;
    size_t spl_smem = 0;
    int spl_grid = 0;
    int spl_uniform = 0;             // every member has the same cheap coefficient tables
    int spl_lpa = 32;                // lanes per atom of the fused cheap kernel
    int64_t launches = 0;            // kernels launched by fused steps
    cudaStream_t aux = nullptr;      // second branch (cheap potential) of the fused step
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

int bfail(mix_batch* b, int code, const std::string& msg) {
    b->err = msg;
    return code;
}

void batch_drop(mix_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// parent graph with one independent child graph per member
int batch_graph(mix_batch* b, int integrate, double dt, cudaGraph_t* graph, cudaGraphExec_t* exec) {
    cudaGraph_t parent = nullptr;
    cudaError_t e = cudaGraphCreate(&parent, 0);
    if (e != cudaSuccess) return bfail(b, MIX_ECUDA, "cudaGraphCreate");
    for (size_t k = 0; k < b->m.size(); ++k) {
        mix_ctx* c = b->m[k];
        cudaGraph_t g = nullptr;
        int st = member_graph(c, integrate, dt, &g);
        if (st) {
            cudaGraphDestroy(parent);
            return bfail(b, st, "member " + std::to_string(k) + ": " + c->err);
        }
        cudaGraphNode_t node;
        e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, g);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGraphDestroy(parent);
            return bfail(b, MIX_ECUDA, std::string("cudaGraphAddChildGraphNode: ") + cudaGetErrorString(e));
        }
    }
    e = cudaGraphInstantiate(exec, parent, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(parent);
        return bfail(b, MIX_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    *graph = parent;
    return MIX_OK;
}

// --- fused multi-system step ------------------------------------------------

// The fused step needs one arithmetic for all members and the geometric form
// of the weights (the seed-atom kernels have no batched version).
bool fused_eligible(const mix_batch* b) {
    if (!b->want_fused || b->m.empty()) return false;
    for (const mix_ctx* c : b->m)
        if (!c->bound || c->precision != b->m[0]->precision || c->seedrule.mode != 0 || c->ace_tcm) return false;
    return true;
}

void fused_free(mix_batch* b) {
    if (b->dmem) cudaFree(b->dmem);
    b->dmem = nullptr;
}

// Host-built plan: per-system parameter arrays, one block table per launch
// granularity, the expensive groups (systems sharing L and the padded radial
// count) and the flattened work lists, all in one device allocation.
int fused_build(mix_batch* b) {
    const int ns = (int)b->m.size();
    b->precision = b->m[0]->precision;
    const bool f64 = b->precision == MIX_FP64;
    std::vector<Dev> devs(ns);
    std::vector<Regions> regs(ns);
    for (int s = 0; s < ns; ++s) {
        devs[s] = b->m[s]->dev;
        regs[s] = b->m[s]->regions;
    }
    // expensive groups
    auto npad = [](int n) { return n <= 4 ? 4 : n <= 8 ? 8 : n <= 12 ? 12 : 16; };
    std::vector<int> egroup(ns), elast(ns, 0);
    b->groups.clear();
    std::vector<int64_t> gatoms;
    for (int s = 0; s < ns; ++s) {
        const mix_ctx* c = b->m[s];
        int g = -1;
        for (size_t k = 0; k < b->groups.size(); ++k)
            if (b->groups[k].L == c->L && npad(b->groups[k].n) == npad(c->n)) g = (int)k;
        if (g < 0) {
            b->groups.push_back({c->L, c->n, c->cap, c->tile_max, c->qb, 0, 0, 0});
            gatoms.push_back(0);
            g = (int)b->groups.size() - 1;
        }
        b->groups[g].n = std::max(b->groups[g].n, c->n);
        b->groups[g].cap = std::max(b->groups[g].cap, c->cap);
        b->groups[g].tile_max = std::max(b->groups[g].tile_max, c->tile_max);
        b->groups[g].qb = std::min(b->groups[g].qb, c->qb);
        gatoms[g] += c->sys.n_atoms;
        egroup[s] = g;
    }
    for (int s = 0; s < ns; ++s) {
        bool last = true;
        for (int t = s + 1; t < ns; ++t)
            if (egroup[t] == egroup[s]) last = false;
        elast[s] = last ? 1 : 0;
    }
    const int ng = (int)b->groups.size();
    std::vector<int> ebase(ng);
    int64_t tot = 0, acc = 0;
    for (int g = 0; g < ng; ++g) {
        ebase[g] = (int)acc;
        b->groups[g].base = (size_t)acc;
        acc += gatoms[g];
    }
    tot = acc;
    if (tot > INT32_MAX / 2) return bfail(b, MIX_EINVAL, "batch too large for one fused step");
    // block tables
    std::vector<std::vector<int4>> tabs(BT_COUNT);
    int capp2 = 32;
    for (int s = 0; s < ns; ++s) {
        const Dev& d = devs[s];
        const int64_t n = d.n;
        auto blocks = [](int64_t units, int64_t per) { return (int)std::max<int64_t>(1, (units + per - 1) / per); };
        const int gx[BT_COUNT] = {blocks(n, 1024), 1, blocks(n, 32), blocks(n, 64),
                                  blocks(n, 256), std::max(1, d.nblk), blocks(n, 256)};
        for (int k = 0; k < BT_COUNT; ++k)
            for (int bx = 0; bx < gx[k]; ++bx) tabs[k].push_back(make_int4(s, bx, gx[k], 0));
        while (capp2 < d.cap) capp2 <<= 1;
    }
    // one device allocation for everything
    const size_t tsz = f64 ? sizeof(AceTab<double>) : sizeof(AceTab<float>);
    const size_t ssz = f64 ? sizeof(SplTab<double>) : sizeof(SplTab<float>);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + std::max<size_t>(bytes, 16));
        return at;
    };
    const size_t o_devs = take(ns * sizeof(Dev)), o_regs = take(ns * sizeof(Regions)), o_ace = take(ns * tsz),
                 o_spl = take(ns * ssz), o_eg = take(ns * 4), o_el = take(ns * 4), o_eb = take(ng * 4),
                 o_cnt = take((ng + 1) * 4), o_le = take(tot * sizeof(int2)), o_lc = take(tot * sizeof(int2));
    size_t o_tab[BT_COUNT];
    for (int k = 0; k < BT_COUNT; ++k) o_tab[k] = take(tabs[k].size() * sizeof(int4));
    fused_free(b);
    cudaError_t e = cudaMalloc(&b->dmem, off);
    if (e != cudaSuccess) {
        b->dmem = nullptr;
        return bfail(b, MIX_ENOMEM, std::string("fused batch arrays: ") + cudaGetErrorString(e));
    }
    std::vector<unsigned char> host(off, 0);
    auto put = [&](size_t o, const void* src, size_t bytes) {
        if (bytes) std::memcpy(host.data() + o, src, bytes);
    };
    put(o_devs, devs.data(), ns * sizeof(Dev));
    put(o_regs, regs.data(), ns * sizeof(Regions));
    for (int s = 0; s < ns; ++s) {
        const mix_ctx* c = b->m[s];
        if (f64) {
            put(o_ace + s * tsz, &c->ace64, tsz);
            put(o_spl + s * ssz, &c->spl64, ssz);
        } else {
            put(o_ace + s * tsz, &c->ace32, tsz);
            put(o_spl + s * ssz, &c->spl32, ssz);
        }
    }
    put(o_eg, egroup.data(), ns * 4);
    put(o_el, elast.data(), ns * 4);
    put(o_eb, ebase.data(), ng * 4);
    for (int k = 0; k < BT_COUNT; ++k) put(o_tab[k], tabs[k].data(), tabs[k].size() * sizeof(int4));
    e = cudaMemcpy(b->dmem, host.data(), off, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bfail(b, MIX_ECUDA, std::string("fused batch upload: ") + cudaGetErrorString(e));
    unsigned char* base = b->dmem;
    BatchPlan& P = b->plan;
    b->ddevs = reinterpret_cast<const Dev*>(base + o_devs);
    b->dace = base + o_ace;
    b->dspl = base + o_spl;
    for (int k = 0; k < BT_COUNT; ++k) {
        P.ba[k].devs = b->ddevs;
        P.ba[k].tab = reinterpret_cast<const int4*>(base + o_tab[k]);
        P.nblk[k] = (int)tabs[k].size();
    }
    P.regions = reinterpret_cast<const Regions*>(base + o_regs);
    P.capp2 = capp2;
    FlatArgs& F = P.flat;
    F.devs = b->ddevs;
    F.nsys = ns;
    F.ngrp = ng;
    F.egroup = reinterpret_cast<const int*>(base + o_eg);
    F.elast = reinterpret_cast<const int*>(base + o_el);
    F.ebase = reinterpret_cast<const int*>(base + o_eb);
    F.list_e = reinterpret_cast<int2*>(base + o_le);
    F.list_c = reinterpret_cast<int2*>(base + o_lc);
    F.counts = reinterpret_cast<int*>(base + o_cnt);
    // launch shapes of the potentials
    for (mix_batch::Group& g : b->groups) {
        e = ace_batch_configure(b->precision, g.L, g.n, g.cap, g.tile_max, g.qb, &g.smem, &g.grid);
        if (e != cudaSuccess) return bfail(b, MIX_ECUDA, std::string("fused expensive kernel: ") + cudaGetErrorString(e));
    }
    // identical cheap tables in every member: the fused kernel stages them once per block
    {
        const size_t tb = f64 ? sizeof(double) : sizeof(float);
        const mix_ctx* c0 = b->m[0];
        b->spl_uniform = 1;
        for (int s = 1; s < ns && b->spl_uniform; ++s) {
            const mix_ctx* c = b->m[s];
            if (std::memcmp(c->arena.bytes.data() + c->o_sc2, c0->arena.bytes.data() + c0->o_sc2,
                            SPL_W2 * 4 * tb) != 0 ||
                std::memcmp(c->arena.bytes.data() + c->o_sc3, c0->arena.bytes.data() + c0->o_sc3,
                            64 * SPL_W3 * 4 * tb) != 0)
                b->spl_uniform = 0;
        }
    }
    // the widest lane group any member needs alone
    b->spl_lpa = 8;
    for (int s = 0; s < ns; ++s) b->spl_lpa = std::max(b->spl_lpa, b->m[s]->spl_lpa);
    e = spline_batch_configure(b->precision, b->spl_lpa, &b->spl_smem, &b->spl_grid);
    if (e != cudaSuccess) return bfail(b, MIX_ECUDA, std::string("fused cheap kernel: ") + cudaGetErrorString(e));
    return MIX_OK;
}

int fused_launches(const mix_batch* b) { return 15 + (int)b->groups.size(); }

// one fused step (or force evaluation) captured on the batch's private stream
int fused_graph(mix_batch* b, int integrate, double dt, cudaGraph_t* graph, cudaGraphExec_t* exec) {
    if (!b->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bfail(b, MIX_ECUDA, "capture stream");
    }
    if (!b->aux) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) return bfail(b, MIX_ECUDA, "second branch stream");
    }
    cudaStream_t s = b->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(b, MIX_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    const BatchPlan& P = b->plan;
    launch_disp_batch(P, s, integrate, dt, 0);
    launch_build_batch(P, s);
    launch_sets_batch(P, s);
    // cheap potential on a second branch, concurrent with the expensive groups
    cudaEventRecord(b->ev_fork, s);
    cudaStreamWaitEvent(b->aux, b->ev_fork, 0);
    launch_spline_batch(b->precision, b->spl_lpa, b->ddevs, b->dspl, P.flat.list_c, P.flat.counts + b->groups.size(),
                        b->spl_uniform, b->spl_smem, b->spl_grid, b->aux);
    cudaEventRecord(b->ev_join, b->aux);
    for (size_t g = 0; g < b->groups.size(); ++g) {
        const mix_batch::Group& G = b->groups[g];
        launch_ace_batch(b->precision, b->ddevs, b->dace, P.flat.list_e + G.base, P.flat.counts + g, G.n, G.L, G.smem,
                         G.grid, s);
    }
    cudaStreamWaitEvent(s, b->ev_join, 0);
    launch_gather_batch(P, b->precision, integrate, dt, s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) return bfail(b, MIX_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return bfail(b, MIX_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    *graph = g;
    return MIX_OK;
}

// evaluate members whose forces or lists are not current, one by one
int batch_prepare(mix_batch* b) {
    for (size_t k = 0; k < b->m.size(); ++k) {
        mix_ctx* c = b->m[k];
        if (!c->bound) return bfail(b, MIX_ESTATE, "member " + std::to_string(k) + " is not bound");
        if (c->need_build || !c->forces_valid) {
            int st = evaluate(c, 0, 0.0);
            if (st) return bfail(b, st, "member " + std::to_string(k) + ": " + c->err);
            c->forces_valid = true;
        }
    }
    return MIX_OK;
}

}  // namespace

extern "C" {

int mix_tune(mix_ctx* c, int reps) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "mix_tune before mix_bind");
    if (reps < 1) reps = 3;
    const int sms = sm_count();
    std::vector<int> ga = {c->ace_grid_max, c->ace_grid_max * 3 / 4, c->ace_grid_max / 2, c->ace_grid_max / 4};
    std::vector<int> gg = {sms * 2, sms * 4, sms * 8, sms * 16};
    SeedSave saved;
    const std::vector<int> orders = {MIX_ORDER_CHEAP_FIRST, MIX_ORDER_EXP_FIRST, MIX_ORDER_SERIAL};
    int st = seed_save(c, &saved);
    if (!st) st = tune_param(c, reps, &c->order, orders);
    if (!st) st = tune_cheap_lanes(c, reps);
    std::vector<int> gs = {c->spl_grid_max, c->spl_grid_max / 2, c->spl_grid_max / 4};
    if (!st) st = tune_param(c, reps, &c->ace_grid, ga);
    if (!st) st = tune_param(c, reps, &c->spl_grid, gs);
    if (!st) st = tune_param(c, reps, &c->dev.grid_gather, gg);
    if (!st) st = tune_param(c, reps, &c->dev.grid_buffer, gg);
    if (!st) st = tune_param(c, reps, &c->order, orders);   // again, at the shapes chosen
    drop_graph(c);
    const int st2 = seed_restore(c, saved);
    return st ? st : st2;
}

int mix_batch_create(mix_ctx* const* members, int n, void* stream, mix_batch** out) {
    if (!out || n < 1 || !members) return MIX_EINVAL;
    *out = nullptr;
    mix_batch* b = new (std::nothrow) mix_batch();
    if (!b) return MIX_ENOMEM;
    b->stream = (cudaStream_t)stream;
    for (int k = 0; k < n; ++k) {
        mix_ctx* c = members[k];
        if (!c || c->stream != b->stream) {
            delete b;
            return MIX_EINVAL;
        }
        b->m.push_back(c);
        b->regions_seen.push_back(c->regions_version);
    }
    *out = b;
    return MIX_OK;
}

int mix_batch_step(mix_batch* b, double dt, int nsteps) {
    if (!b) return MIX_EINVAL;
    if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt)) return bfail(b, MIX_EINVAL, "dt / nsteps");
    int st = batch_prepare(b);
    if (st) return st;
    const bool fused = fused_eligible(b);
    bool stale = !b->exec || b->dt != dt || b->graph_fused != fused;
    for (size_t k = 0; k < b->m.size(); ++k)
        if (b->regions_seen[k] != b->m[k]->regions_version) stale = true;
    if (stale) {
        batch_drop(b);
        if (fused) {
            // the plan snapshots the members' device descriptors: rebuilt with the graph
            st = fused_build(b);
            if (!st) st = fused_graph(b, 1, dt, &b->graph, &b->exec);
        } else {
            st = batch_graph(b, 1, dt, &b->graph, &b->exec);
        }
        if (st) return st;
        b->graph_fused = fused;
        b->dt = dt;
        for (size_t k = 0; k < b->m.size(); ++k) b->regions_seen[k] = b->m[k]->regions_version;
    }
    for (int s = 0; s < nsteps; ++s) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
        if (e != cudaSuccess) return bfail(b, MIX_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    }
    for (mix_ctx* c : b->m) {
        c->steps += nsteps;
        if (!fused) c->launches += (int64_t)evals_launches(c) * nsteps;
    }
    if (fused) b->launches += (int64_t)fused_launches(b) * nsteps;
    return MIX_OK;
}

int mix_batch_sync(mix_batch* b) {
    if (!b) return MIX_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, MIX_ECUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
    for (size_t k = 0; k < b->m.size(); ++k) {
        int st = read_status(b->m[k]);
        if (st) return bfail(b, st, "member " + std::to_string(k) + ": " + b->m[k]->err);
    }
    return MIX_OK;
}

int mix_batch_tune(mix_batch* b, int reps, int* chosen) {
    if (!b) return MIX_EINVAL;
    if (reps < 1) reps = 3;
    int st = batch_prepare(b);
    if (st) return st;
    std::vector<SeedSave> saved(b->m.size());
    for (size_t k = 0; k < b->m.size() && !st; ++k) st = seed_save(b->m[k], &saved[k]);
    if (st) return bfail(b, st, "seed state save");
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, MIX_ECUDA, "event");
    int best = 1;
    float tbest = 1e30f;
    for (int div : {1, 2, 4, 8, 16}) {
        for (mix_ctx* c : b->m) set_grid_divisor(c, div);
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        st = batch_graph(b, 0, 0.0, &g, &x);
        if (st) break;
        std::vector<float> v;
        cudaGraphLaunch(x, b->stream);
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(e0, b->stream);
            cudaGraphLaunch(x, b->stream);
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            v.push_back(t);
        }
        cudaGraphExecDestroy(x);
        cudaGraphDestroy(g);
        std::sort(v.begin(), v.end());
        const float t = v[v.size() / 2];
        if (t < tbest) {
            tbest = t;
            best = div;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (mix_ctx* c : b->m) set_grid_divisor(c, best);
    batch_drop(b);
    b->divisor = best;
    if (chosen) *chosen = best;
    for (size_t k = 0; k < b->m.size(); ++k) {
        const int sr = seed_restore(b->m[k], saved[k]);
        if (!st && sr) st = bfail(b, sr, "seed state restore");
    }
    cudaError_t e = cudaGetLastError();
    if (!st && e != cudaSuccess) st = bfail(b, MIX_ECUDA, cudaGetErrorString(e));
    return st;
}

int mix_batch_destroy(mix_batch* b) {
    if (!b) return MIX_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop(b);
    fused_free(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->aux) cudaStreamDestroy(b->aux);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    delete b;
    return MIX_OK;
}

int mix_batch_set_fused(mix_batch* b, int fused) {
    if (!b) return MIX_EINVAL;
    b->want_fused = fused ? 1 : 0;
    return MIX_OK;
}

int mix_batch_info(const mix_batch* b, int* fused, int* groups, int64_t* launches) {
    if (!b) return MIX_EINVAL;
    if (fused) *fused = b->graph_fused ? 1 : 0;
    if (groups) *groups = (int)b->groups.size();
    if (launches) *launches = b->launches;
    return MIX_OK;
}

const char* mix_batch_last_error(const mix_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"

// ---------------------------------------------------------------------------
// weights from seed atoms (Alg. 1-2)

namespace {

int seed_radii_ok(mix_ctx* c, double a, double b) {
    const double rmax = c->rlist - c->opt.skin;   // pairs closer than this are always in the lists
    if (!(a >= 0) || !(b >= 0) || a > rmax || b > rmax)
        return fail(c, MIX_EINVAL, "seed radii must lie in [0, %.4g] (the largest cutoff)", rmax);
    return MIX_OK;
}

}  // namespace

extern "C" {

int mix_set_seeds(mix_ctx* c, const int* seeds, int n_seeds, double r_core, double r_blend) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "mix_set_seeds before mix_bind");
    if (n_seeds < 0 || (n_seeds > 0 && !seeds)) return fail(c, MIX_EINVAL, "seed list");
    int st = seed_radii_ok(c, r_core, r_blend);
    if (st) return st;
    const int64_t N = c->sys.n_atoms;
    std::vector<uint8_t> mask((size_t)(N > 0 ? N : 1), 0);
    for (int k = 0; k < n_seeds; ++k) {
        if (seeds[k] < 0 || seeds[k] >= N) return fail(c, MIX_EINVAL, "seed index %d out of range", seeds[k]);
        mask[seeds[k]] = 1;
    }
    cudaError_t e = cudaMemcpyAsync(c->dev.seed, mask.data(), (size_t)N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mix_set_seeds");
    SeedRule& r = c->seedrule;
    r = SeedRule();
    r.mode = 1;
    r.blend = c->opt.blend;
    r.rcore2 = r_core * r_core;
    r.rblend2 = r_blend * r_blend;
    r.rblend = r_blend;
    r.period = 1;
    c->regions_version++;
    c->forces_valid = false;
    return MIX_OK;
}

int mix_set_seed_rule(mix_ctx* c, double r_coord, double z_lo, double z_hi, int period, double r_core,
                      double r_blend) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "mix_set_seed_rule before mix_bind");
    if (period < 1 || !(z_lo <= z_hi)) return fail(c, MIX_EINVAL, "period >= 1 and z_lo <= z_hi");
    int st = seed_radii_ok(c, r_core, r_blend);
    if (!st) st = seed_radii_ok(c, r_coord, 0.0);
    if (st) return st;
    const size_t N = (size_t)c->sys.n_atoms;
    cudaError_t e = cudaMemsetAsync(c->dev.zsum, 0, N * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dev.seed, 0, N, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dev.status + SW_EVALS, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mix_set_seed_rule");
    SeedRule& r = c->seedrule;
    r = SeedRule();
    r.mode = 2;
    r.blend = c->opt.blend;
    r.rcore2 = r_core * r_core;
    r.rblend2 = r_blend * r_blend;
    r.rblend = r_blend;
    r.rz2 = r_coord * r_coord;
    r.zlo = z_lo;
    r.zhi = z_hi;
    r.period = period;
    c->regions_version++;
    c->forces_valid = false;
    return MIX_OK;
}

int mix_get_seeds(mix_ctx* c, uint8_t* seed, int64_t* n_seeds) {
    if (!c) return MIX_EINVAL;
    if (!c->bound) return fail(c, MIX_ESTATE, "not bound");
    int st = read_status(c);
    if (st) return st;
    if (n_seeds) *n_seeds = c->pinned[SW_NSEED];
    return copy_out(c, seed, c->dev.seed, (size_t)c->sys.n_atoms);
}

}  // extern "C"
