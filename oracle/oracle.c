/*
 * Plain FP64 CPU oracle for the spatially mixed MD step of arXiv 2502.19081
 * (ML-MIX force mixing).  TEST INFRASTRUCTURE ONLY: the tests, the package's
 * smoke check and the benchmark's CPU-baseline leg call it; the product path
 * never does.  It shares no code with the CUDA library.
 *
 * What it computes, in the paper's order:
 *   - region weights lambda_i (Sec. 4.4, Alg. 1-2, geometric reading);
 *   - the evaluated sets Lambda_k and their buffers (Sec. 4.5, buffer set
 *     equation; Alg. 3);
 *   - forces as sums of site-energy derivatives (Sec. 4.5, force equation)
 *     for each potential restricted to its evaluated set, scaled by the blend
 *     weight and accumulated (Alg. 4);
 *   - the plain definition F = w F_exp,full + (1 - w) F_cheap,full used to
 *     check the above (one-cutoff buffer sufficiency, Sec. 4.5);
 *   - velocity-Verlet NVE steps.
 * Both potentials are synthetic (the paper names the families only: linear ACE
 * and UF3, Sec. 2.1): see the header comment of oracle/__init__.py.
 *
 * Conventions that make sets and lists bit-reproducible: minimum image
 * d - L*rint(d/L) with 1/L precomputed, squared distance dx*dx+dy*dy+dz*dz in
 * that order, strict '<' comparisons, no contraction into FMA (built with
 * -ffp-contract=off).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_EOVERFLOW (-4)

#define MAXREG 16
#define MAXL 8
#define KAPPA 9.6485332e-3 /* (eV / Angstrom / amu) in Angstrom / fs^2 */

/* ------------------------------------------------------------------------- */
/* geometry                                                                   */

typedef struct {
    double lo[3], L[3], invL[3];
    int per[3];
} obox;

static void box_init(obox* b, const double* lo, const double* L, const int* per) {
    for (int d = 0; d < 3; ++d) {
        b->lo[d] = lo[d];
        b->L[d] = L[d];
        b->invL[d] = 1.0 / L[d];
        b->per[d] = per[d];
    }
}

/* d = xj - xi with the minimum-image convention in periodic dimensions */
static void box_delta(const obox* b, const double* xi, const double* xj, double* d) {
    for (int k = 0; k < 3; ++k) {
        double t = xj[k] - xi[k];
        if (b->per[k]) t = t - b->L[k] * rint(t * b->invL[k]);
        d[k] = t;
    }
}

static double norm2(const double* d) { return d[0] * d[0] + d[1] * d[1] + d[2] * d[2]; }

/* ------------------------------------------------------------------------- */
/* cell list and neighbour lists                                             */

typedef struct {
    int nc[3];
    double invh[3];
} ocells;

static int cells_init(const obox* b, double rlist, ocells* c) {
    for (int d = 0; d < 3; ++d) {
        int n = (int)floor(b->L[d] / rlist);
        if (b->per[d]) {
            if (b->lo[d] != 0.0) return OR_EINVAL;
            if (n < 3 || b->L[d] < 2.0 * rlist) return OR_EINVAL;
        } else if (n < 1) {
            n = 1;
        }
        c->nc[d] = n;
        c->invh[d] = (double)n / b->L[d];
    }
    return OR_OK;
}

/* Cell index along d.  In a periodic dimension the coordinate is first folded
 * into [0, L) as x - L floor(x / L): between list rebuilds an atom may sit up
 * to half a skin outside a periodic face, and its cell must be the one its
 * image lies in (clamping it into the edge cell would leave partners more than
 * h - rlist beyond the face outside the 27-cell stencil).  Pair vectors stay
 * minimum images of the raw positions (box_delta). */
static int cell_coord(const obox* b, const ocells* c, const double* x, int d) {
    double t = x[d] - b->lo[d];
    if (b->per[d]) t = t - b->L[d] * floor(t * b->invL[d]);
    double s = t * c->invh[d];
    int q = (int)floor(s);
    if (q < 0) q = 0;
    if (q > c->nc[d] - 1) q = c->nc[d] - 1;
    return q;
}

static int cmp_int(const void* a, const void* b) {
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

/* cell id per atom, c = (cz * ncy + cy) * ncx + cx */
int or_cells(int64_t n, const double* x, const double* lo, const double* L, const int* per,
             double rlist, int* ncell, int* cell_of) {
    obox b;
    ocells c;
    box_init(&b, lo, L, per);
    int st = cells_init(&b, rlist, &c);
    if (st) return st;
    for (int d = 0; d < 3; ++d) ncell[d] = c.nc[d];
    for (int64_t i = 0; i < n; ++i) {
        const double* xi = x + 4 * i;
        int cx = cell_coord(&b, &c, xi, 0), cy = cell_coord(&b, &c, xi, 1), cz = cell_coord(&b, &c, xi, 2);
        cell_of[i] = (cz * c.nc[1] + cy) * c.nc[0] + cx;
    }
    return OR_OK;
}

/* Full neighbour list {j != i : |r_ij|^2 < rlist^2} through a 27-cell stencil,
 * each row sorted ascending.  nnb[i] is the true count even on overflow. */
static int neighbours_cells(const obox* b, int64_t n, const double* x, double rlist, int cap, int* nnb,
                            int* nbr) {
    ocells c;
    int st = cells_init(b, rlist, &c);
    if (st) return st;
    int ncell = c.nc[0] * c.nc[1] * c.nc[2];
    int* head = (int*)malloc(sizeof(int) * (size_t)ncell);
    int* next = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int* cid = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!head || !next || !cid) {
        free(head); free(next); free(cid);
        return OR_ENOMEM;
    }
    for (int k = 0; k < ncell; ++k) head[k] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        const double* xi = x + 4 * i;
        int cx = cell_coord(b, &c, xi, 0), cy = cell_coord(b, &c, xi, 1), cz = cell_coord(b, &c, xi, 2);
        int k = (cz * c.nc[1] + cy) * c.nc[0] + cx;
        cid[i] = k;
        next[i] = head[k];
        head[k] = (int)i;
    }
    double r2max = rlist * rlist;
    int over = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : over)
    for (int64_t i = 0; i < n; ++i) {
        const double* xi = x + 4 * i;
        int k = cid[i];
        int ci[3] = {k % c.nc[0], (k / c.nc[0]) % c.nc[1], k / (c.nc[0] * c.nc[1])};
        int cnt = 0;
        int* row = nbr + (int64_t)cap * i;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int o[3] = {dx, dy, dz}, q[3];
                    int ok = 1;
                    for (int d = 0; d < 3; ++d) {
                        q[d] = ci[d] + o[d];
                        if (b->per[d]) {
                            q[d] = (q[d] + c.nc[d]) % c.nc[d];
                        } else if (q[d] < 0 || q[d] >= c.nc[d]) {
                            ok = 0;
                        }
                    }
                    if (!ok) continue;
                    int kk = (q[2] * c.nc[1] + q[1]) * c.nc[0] + q[0];
                    for (int j = head[kk]; j >= 0; j = next[j]) {
                        if (j == i) continue;
                        double dd[3];
                        box_delta(b, xi, x + 4 * (int64_t)j, dd);
                        if (norm2(dd) < r2max) {
                            if (cnt < cap) row[cnt] = j;
                            cnt++;
                        }
                    }
                }
        nnb[i] = cnt;
        if (cnt > cap) over = 1;
        else qsort(row, (size_t)cnt, sizeof(int), cmp_int);
    }
    free(head); free(next); free(cid);
    return over ? OR_EOVERFLOW : OR_OK;
}

int or_neighbours(int64_t n, const double* x, const double* lo, const double* L, const int* per, double rlist,
                  int cap, int* nnb, int* nbr) {
    obox b;
    box_init(&b, lo, L, per);
    return neighbours_cells(&b, n, x, rlist, cap, nnb, nbr);
}

/* O(N^2) enumeration of the same list; used to pin the cell-list version */
int or_neighbours_brute(int64_t n, const double* x, const double* lo, const double* L, const int* per,
                        double rlist, int cap, int* nnb, int* nbr) {
    obox b;
    box_init(&b, lo, L, per);
    double r2max = rlist * rlist;
    int over = 0;
    for (int64_t i = 0; i < n; ++i) {
        int cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            box_delta(&b, x + 4 * i, x + 4 * j, d);
            if (norm2(d) < r2max) {
                if (cnt < cap) nbr[(int64_t)cap * i + cnt] = (int)j;
                cnt++;
            }
        }
        nnb[i] = cnt;
        if (cnt > cap) over = 1;
    }
    return over ? OR_EOVERFLOW : OR_OK;
}

/* x <- x - L floor(x / L) in periodic dimensions (the fold applied at a rebuild) */
void or_wrap(int64_t n, double* x, const double* L, const int* per) {
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d)
            if (per[d]) {
                double invL = 1.0 / L[d];
                x[4 * i + d] = x[4 * i + d] - L[d] * floor(x[4 * i + d] * invL);
            }
}

/* ------------------------------------------------------------------------- */
/* real spherical harmonics as explicit polynomials                           */
/*   Y_lm(x,y,z) = N_lm s_m Pi_l^|m|(z) T_m(x,y) on the unit sphere, with      */
/*   Pi_l^mu = d^mu P_l / dz^mu (P_l from its explicit coefficient sum),       */
/*   T_m = Re (x+iy)^m (m>0), Im (x+iy)^|m| (m<0), 1 (m=0),                     */
/*   N_lm = sqrt((2l+1)/(4pi) (l-|m|)!/(l+|m|)!), s_m = sqrt2 (m != 0), 1.      */
/*   No Condon-Shortley phase.                                                */

typedef struct {
    int nt;
    int ex[64], ey[64], ez[64];
    double cf[64];
} opoly;

static double fact(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

static double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    return fact(n) / (fact(k) * fact(n - k));
}

static void ylm_poly(int l, int m, opoly* p) {
    int mu = m < 0 ? -m : m;
    /* Legendre coefficients: P_l(z) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) z^(l-2k) */
    double pz[2 * MAXL + 2];
    memset(pz, 0, sizeof(pz));
    for (int k = 0; 2 * k <= l; ++k)
        pz[l - 2 * k] = ldexp(1.0, -l) * ((k & 1) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l);
    /* mu-th derivative */
    double dz[2 * MAXL + 2];
    memset(dz, 0, sizeof(dz));
    for (int e = mu; e <= l; ++e) dz[e - mu] = pz[e] * fact(e) / fact(e - mu);
    /* (x + i y)^mu terms */
    double nlm = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fact(l - mu) / fact(l + mu));
    double sm = (m == 0) ? 1.0 : sqrt(2.0);
    p->nt = 0;
    for (int k = 0; k <= mu; ++k) {
        /* C(mu,k) x^(mu-k) (i y)^k; i^k = 1, i, -1, -i */
        double re = 0.0, im = 0.0;
        switch (k & 3) {
            case 0: re = 1.0; break;
            case 1: im = 1.0; break;
            case 2: re = -1.0; break;
            case 3: im = -1.0; break;
        }
        double t = (m > 0) ? re : (m < 0 ? im : (k == 0 ? 1.0 : 0.0));
        if (m == 0 && k > 0) t = 0.0;
        if (t == 0.0) continue;
        for (int e = 0; e <= l - mu; ++e) {
            if (dz[e] == 0.0) continue;
            p->ex[p->nt] = mu - k;
            p->ey[p->nt] = k;
            p->ez[p->nt] = e;
            p->cf[p->nt] = nlm * sm * binom(mu, k) * t * dz[e];
            p->nt++;
        }
    }
}

static double ipow(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

/* value and gradient (w.r.t. the unit-vector argument) of the polynomial */
static void poly_eval(const opoly* p, const double* u, double* val, double* grad) {
    double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int t = 0; t < p->nt; ++t) {
        int a = p->ex[t], b = p->ey[t], c = p->ez[t];
        double cf = p->cf[t];
        v += cf * ipow(u[0], a) * ipow(u[1], b) * ipow(u[2], c);
        if (a > 0) gx += cf * a * ipow(u[0], a - 1) * ipow(u[1], b) * ipow(u[2], c);
        if (b > 0) gy += cf * b * ipow(u[0], a) * ipow(u[1], b - 1) * ipow(u[2], c);
        if (c > 0) gz += cf * c * ipow(u[0], a) * ipow(u[1], b) * ipow(u[2], c - 1);
    }
    *val = v;
    if (grad) {
        grad[0] = gx;
        grad[1] = gy;
        grad[2] = gz;
    }
}

/* exported for the convention pin against a library implementation */
double or_ylm(int l, int m, const double* u) {
    opoly p;
    ylm_poly(l, m, &p);
    double v;
    poly_eval(&p, u, &v, NULL);
    return v;
}

/* ------------------------------------------------------------------------- */
/* Wigner 3j (Racah formula) and real Gaunt coefficients                     */

static double w3j(int j1, int j2, int j3, int m1, int m2, int m3) {
    if (m1 + m2 + m3 != 0) return 0.0;
    if (j3 < abs(j1 - j2) || j3 > j1 + j2) return 0.0;
    if (abs(m1) > j1 || abs(m2) > j2 || abs(m3) > j3) return 0.0;
    double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
    double pre = sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) * fact(j3 + m3) *
                      fact(j3 - m3));
    double s = 0.0;
    for (int k = 0; k <= j1 + j2 + j3; ++k) {
        int a1 = j3 - j2 + k + m1, a2 = j3 - j1 + k - m2, a3 = j1 + j2 - j3 - k, a4 = j1 - k - m1,
            a5 = j2 - k + m2;
        if (a1 < 0 || a2 < 0 || a3 < 0 || a4 < 0 || a5 < 0) continue;
        double den = fact(k) * fact(a1) * fact(a2) * fact(a3) * fact(a4) * fact(a5);
        s += ((k & 1) ? -1.0 : 1.0) / den;
    }
    int ph = j1 - j2 - m3;
    double sign = ((ph % 2) + 2) % 2 ? -1.0 : 1.0;
    return sign * pre * s;
}

/* integral of three complex Y_l^m (Condon-Shortley phase) over the sphere */
static double gaunt_complex(int l1, int m1, int l2, int m2, int l3, int m3) {
    return sqrt((2.0 * l1 + 1) * (2.0 * l2 + 1) * (2.0 * l3 + 1) / (4.0 * M_PI)) * w3j(l1, l2, l3, 0, 0, 0) *
           w3j(l1, l2, l3, m1, m2, m3);
}

/* coefficient of Y_l^{mp} (complex) in the real Y_lm of this file */
static double complex u_real(int m, int mp) {
    double r2 = 1.0 / sqrt(2.0);
    if (m == 0) return (mp == 0) ? 1.0 : 0.0;
    if (m > 0) {
        if (mp == m) return ((m & 1) ? -1.0 : 1.0) * r2;
        if (mp == -m) return r2;
        return 0.0;
    }
    int mu = -m;
    if (mp == mu) return -I * ((mu & 1) ? -1.0 : 1.0) * r2;
    if (mp == -mu) return I * r2;
    return 0.0;
}

double or_gaunt_real(int l1, int m1, int l2, int m2, int l3, int m3) {
    double complex s = 0.0;
    for (int a = -l1; a <= l1; ++a) {
        double complex ua = u_real(m1, a);
        if (ua == 0.0) continue;
        for (int b = -l2; b <= l2; ++b) {
            double complex ub = u_real(m2, b);
            if (ub == 0.0) continue;
            int c = -a - b;
            if (c < -l3 || c > l3) continue;
            double complex uc = u_real(m3, c);
            if (uc == 0.0) continue;
            s += ua * ub * uc * gaunt_complex(l1, a, l2, b, l3, c);
        }
    }
    return creal(s);
}

/* ------------------------------------------------------------------------- */
/* cubic B-splines on an explicit knot vector (Cox-de Boor)                   */

static double bsp(const double* t, int a, int k, double x) {
    if (k == 0) return (t[a] <= x && x < t[a + 1]) ? 1.0 : 0.0;
    double s = 0.0;
    double d1 = t[a + k] - t[a], d2 = t[a + k + 1] - t[a + 1];
    if (d1 > 0) s += (x - t[a]) / d1 * bsp(t, a, k - 1, x);
    if (d2 > 0) s += (t[a + k + 1] - x) / d2 * bsp(t, a + 1, k - 1, x);
    return s;
}

static double bsp_d(const double* t, int a, int k, double x) {
    double s = 0.0;
    double d1 = t[a + k] - t[a], d2 = t[a + k + 1] - t[a + 1];
    if (d1 > 0) s += k / d1 * bsp(t, a, k - 1, x);
    if (d2 > 0) s -= k / d2 * bsp(t, a + 1, k - 1, x);
    return s;
}

/* uniform knots t_a = (a-3) h, a = 0..nb+3 */
static void uniform_knots(double h, int nb, double* t) {
    for (int a = 0; a < nb + 4; ++a) t[a] = (a - 3) * h;
}

/* V(r) = sum_a c_a B_a(r) and V'(r) */
static void spline1(const double* c, int nb, const double* t, double r, double* v, double* dv) {
    double s = 0.0, ds = 0.0;
    for (int a = 0; a < nb; ++a) {
        if (c[a] == 0.0) continue;
        s += c[a] * bsp(t, a, 3, r);
        ds += c[a] * bsp_d(t, a, 3, r);
    }
    *v = s;
    *dv = ds;
}

/* ------------------------------------------------------------------------- */
/* potentials                                                                 */

typedef struct {
    double rc;
    int n, L, nu;
    double* c1; /* [n] */
    double* c2; /* [L+1][n][n] */
    double* c3; /* [L+1]^3 [n]^3 */
    double pair[16];
    double tpair[20];
    int nlm;
    opoly* poly; /* [nlm] */
    /* Gaunt tables per (l1,l2,l3): nonzero (m1,m2,m3,G) */
    int* gstart; /* [(L+1)^3 + 1] */
    int* gm;     /* [nnz][3] */
    double* gv;  /* [nnz] */
} oace;

typedef struct {
    double rc, rc3;
    double c2[16];
    double c3[8 * 8 * 8];
    double t2[20], t3a[12], t3c[12];
} ospl;

#define LM(l, m) ((l) * (l) + (m) + (l))

static void ace_free(oace* a) {
    if (!a) return;
    free(a->c1); free(a->c2); free(a->c3); free(a->poly); free(a->gstart); free(a->gm); free(a->gv);
    free(a);
}

static oace* ace_new(double rc, int n, int L, int nu, const double* c1, const double* c2, const double* c3,
                     const double* pair) {
    if (L < 0 || L >= MAXL || n < 1 || nu < 1 || nu > 3) return NULL;
    oace* a = (oace*)calloc(1, sizeof(oace));
    a->rc = rc; a->n = n; a->L = L; a->nu = nu;
    int L1 = L + 1;
    a->c1 = (double*)malloc(sizeof(double) * n);
    a->c2 = (double*)malloc(sizeof(double) * L1 * n * n);
    a->c3 = (double*)malloc(sizeof(double) * (size_t)L1 * L1 * L1 * n * n * n);
    memcpy(a->c1, c1, sizeof(double) * n);
    memcpy(a->c2, c2, sizeof(double) * L1 * n * n);
    memcpy(a->c3, c3, sizeof(double) * (size_t)L1 * L1 * L1 * n * n * n);
    for (int k = 0; k < 16; ++k) a->pair[k] = pair ? pair[k] : 0.0;
    uniform_knots(rc / 13.0, 16, a->tpair);
    a->nlm = L1 * L1;
    a->poly = (opoly*)malloc(sizeof(opoly) * a->nlm);
    for (int l = 0; l <= L; ++l)
        for (int m = -l; m <= l; ++m) ylm_poly(l, m, &a->poly[LM(l, m)]);
    int nt = L1 * L1 * L1;
    a->gstart = (int*)calloc((size_t)nt + 1, sizeof(int));
    int cap = 0;
    for (int l1 = 0; l1 <= L; ++l1)
        for (int l2 = 0; l2 <= L; ++l2)
            for (int l3 = 0; l3 <= L; ++l3) cap += (2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1);
    a->gm = (int*)malloc(sizeof(int) * 3 * (size_t)cap);
    a->gv = (double*)malloc(sizeof(double) * (size_t)cap);
    int nnz = 0;
    for (int l1 = 0; l1 <= L; ++l1)
        for (int l2 = 0; l2 <= L; ++l2)
            for (int l3 = 0; l3 <= L; ++l3) {
                int id = (l1 * L1 + l2) * L1 + l3;
                a->gstart[id] = nnz;
                if (nu >= 3 && l1 <= l2 && l2 <= l3)
                    for (int m1 = -l1; m1 <= l1; ++m1)
                        for (int m2 = -l2; m2 <= l2; ++m2)
                            for (int m3 = -l3; m3 <= l3; ++m3) {
                                double g = or_gaunt_real(l1, m1, l2, m2, l3, m3);
                                if (fabs(g) < 1e-14) continue;
                                a->gm[3 * nnz] = m1;
                                a->gm[3 * nnz + 1] = m2;
                                a->gm[3 * nnz + 2] = m3;
                                a->gv[nnz] = g;
                                nnz++;
                            }
                a->gstart[id + 1] = nnz;
            }
    return a;
}

static ospl* spl_new(double rc, double rc3, const double* c2, const double* c3) {
    ospl* s = (ospl*)calloc(1, sizeof(ospl));
    s->rc = rc;
    s->rc3 = rc3;
    memcpy(s->c2, c2, sizeof(double) * 16);
    memcpy(s->c3, c3, sizeof(double) * 512);
    uniform_knots(rc / 13.0, 16, s->t2);
    uniform_knots(rc3 / 5.0, 8, s->t3a);
    uniform_knots(2.0 * rc3 / 5.0, 8, s->t3c);
    return s;
}

/* Chebyshev radial basis R_n(r) = T_n(2r/rc - 1) fc(r), fc = (1 - (r/rc)^2)^3 */
static void radial(const oace* a, double r, double* R, double* dR) {
    double s = 2.0 * r / a->rc - 1.0, ds = 2.0 / a->rc;
    double q = (r / a->rc) * (r / a->rc);
    double fc = (1.0 - q) * (1.0 - q) * (1.0 - q);
    double dfc = 3.0 * (1.0 - q) * (1.0 - q) * (-2.0 * r / (a->rc * a->rc));
    double T[32], dT[32];
    T[0] = 1.0; dT[0] = 0.0;
    if (a->n > 1) { T[1] = s; dT[1] = 1.0; }
    for (int k = 2; k < a->n; ++k) {
        T[k] = 2.0 * s * T[k - 1] - T[k - 2];
        dT[k] = 2.0 * T[k - 1] + 2.0 * s * dT[k - 1] - dT[k - 2];
    }
    for (int k = 0; k < a->n; ++k) {
        R[k] = T[k] * fc;
        dR[k] = dT[k] * ds * fc + T[k] * dfc;
    }
}

/* Basis values and the readout, written out per basis function in the
 * canonical enumeration; returns E_site (many-body part) and omega = dE/dA. */
static double ace_readout(const oace* P, const double* A, double* om, double* basis_out) {
    int n = P->n, L = P->L, L1 = L + 1, nlm = P->nlm;
    double E = 0.0;
    int kb = 0;
    memset(om, 0, sizeof(double) * n * nlm);
    /* nu = 1: A_{n00} */
    for (int q = 0; q < n; ++q) {
        double B = A[q * nlm + 0];
        if (basis_out) basis_out[kb] = B;
        kb++;
        E += P->c1[q] * B;
        om[q * nlm + 0] += P->c1[q];
    }
    if (P->nu >= 2) {
        for (int l = 0; l <= L; ++l)
            for (int n1 = 0; n1 < n; ++n1)
                for (int n2 = n1; n2 < n; ++n2) {
                    double c = P->c2[(l * n + n1) * n + n2];
                    double B = 0.0;
                    for (int m = -l; m <= l; ++m) B += A[n1 * nlm + LM(l, m)] * A[n2 * nlm + LM(l, m)];
                    if (basis_out) basis_out[kb] = B;
                    kb++;
                    E += c * B;
                    for (int m = -l; m <= l; ++m) {
                        om[n1 * nlm + LM(l, m)] += c * A[n2 * nlm + LM(l, m)];
                        om[n2 * nlm + LM(l, m)] += c * A[n1 * nlm + LM(l, m)];
                    }
                }
    }
    if (P->nu >= 3) {
        for (int l1 = 0; l1 <= L; ++l1)
            for (int l2 = l1; l2 <= L; ++l2)
                for (int l3 = l2; l3 <= L; ++l3) {
                    if ((l1 + l2 + l3) & 1) continue;
                    if (l3 > l1 + l2) continue;
                    int id = (l1 * L1 + l2) * L1 + l3;
                    int g0 = P->gstart[id], g1 = P->gstart[id + 1];
                    for (int n1 = 0; n1 < n; ++n1)
                        for (int n2 = (l2 == l1 ? n1 : 0); n2 < n; ++n2)
                            for (int n3 = (l3 == l2 ? n2 : 0); n3 < n; ++n3) {
                                double c = P->c3[(((size_t)id * n + n1) * n + n2) * n + n3];
                                double B = 0.0;
                                for (int t = g0; t < g1; ++t) {
                                    int m1 = P->gm[3 * t], m2 = P->gm[3 * t + 1], m3 = P->gm[3 * t + 2];
                                    double G = P->gv[t];
                                    double a1 = A[n1 * nlm + LM(l1, m1)];
                                    double a2 = A[n2 * nlm + LM(l2, m2)];
                                    double a3 = A[n3 * nlm + LM(l3, m3)];
                                    B += G * a1 * a2 * a3;
                                    om[n1 * nlm + LM(l1, m1)] += c * G * a2 * a3;
                                    om[n2 * nlm + LM(l2, m2)] += c * G * a1 * a3;
                                    om[n3 * nlm + LM(l3, m3)] += c * G * a1 * a2;
                                }
                                if (basis_out) basis_out[kb] = B;
                                kb++;
                                E += c * B;
                            }
                }
    }
    return E;
}

int or_ace_basis_count(const oace* P) {
    int n = P->n, L = P->L, cnt = n;
    if (P->nu >= 2) cnt += (L + 1) * n * (n + 1) / 2;
    if (P->nu >= 3)
        for (int l1 = 0; l1 <= L; ++l1)
            for (int l2 = l1; l2 <= L; ++l2)
                for (int l3 = l2; l3 <= L; ++l3) {
                    if (((l1 + l2 + l3) & 1) || l3 > l1 + l2) continue;
                    for (int n1 = 0; n1 < n; ++n1)
                        for (int n2 = (l2 == l1 ? n1 : 0); n2 < n; ++n2)
                            for (int n3 = (l3 == l2 ? n2 : 0); n3 < n; ++n3) cnt++;
                }
    return cnt;
}

/* Site energy of the expensive potential for one environment; rij[j] = x_j - x_i.
 * g[j] = dE_i / d r_ij.  Neighbours at r >= rc contribute nothing. */
static double ace_site(const oace* P, int nn, const double* rij, double* g, double* basis_out, double* A_out) {
    int n = P->n, nlm = P->nlm;
    double* A = (double*)calloc((size_t)n * nlm, sizeof(double));
    double* om = (double*)calloc((size_t)n * nlm, sizeof(double));
    double* R = (double*)malloc(sizeof(double) * (size_t)(nn > 0 ? nn : 1) * n);
    double* dR = (double*)malloc(sizeof(double) * (size_t)(nn > 0 ? nn : 1) * n);
    double* Y = (double*)malloc(sizeof(double) * (size_t)(nn > 0 ? nn : 1) * nlm);
    double* dY = (double*)malloc(sizeof(double) * (size_t)(nn > 0 ? nn : 1) * nlm * 3);
    double* rr = (double*)malloc(sizeof(double) * (size_t)(nn > 0 ? nn : 1));
    double Epair = 0.0;
    for (int j = 0; j < nn; ++j) {
        const double* d = rij + 3 * j;
        double r = sqrt(norm2(d));
        rr[j] = r;
        if (!(r < P->rc)) continue;
        double u[3] = {d[0] / r, d[1] / r, d[2] / r};
        radial(P, r, R + (size_t)j * n, dR + (size_t)j * n);
        for (int k = 0; k < nlm; ++k) {
            double v, gp[3];
            poly_eval(&P->poly[k], u, &v, gp);
            Y[(size_t)j * nlm + k] = v;
            double ug = u[0] * gp[0] + u[1] * gp[1] + u[2] * gp[2];
            for (int c = 0; c < 3; ++c) dY[((size_t)j * nlm + k) * 3 + c] = (gp[c] - u[c] * ug) / r;
        }
        for (int q = 0; q < n; ++q)
            for (int k = 0; k < nlm; ++k) A[q * nlm + k] += R[(size_t)j * n + q] * Y[(size_t)j * nlm + k];
        double vp, dvp;
        spline1(P->pair, 16, P->tpair, r, &vp, &dvp);
        Epair += 0.5 * vp;
    }
    double E = Epair + ace_readout(P, A, om, basis_out);
    if (A_out) memcpy(A_out, A, sizeof(double) * n * nlm);
    if (g) {
        for (int j = 0; j < nn; ++j) {
            double* gj = g + 3 * j;
            gj[0] = gj[1] = gj[2] = 0.0;
            double r = rr[j];
            if (!(r < P->rc)) continue;
            const double* d = rij + 3 * j;
            double u[3] = {d[0] / r, d[1] / r, d[2] / r};
            double vp, dvp;
            spline1(P->pair, 16, P->tpair, r, &vp, &dvp);
            for (int c = 0; c < 3; ++c) gj[c] += 0.5 * dvp * u[c];
            for (int q = 0; q < n; ++q)
                for (int k = 0; k < nlm; ++k) {
                    double w = om[q * nlm + k];
                    double a = dR[(size_t)j * n + q] * Y[(size_t)j * nlm + k];
                    double b = R[(size_t)j * n + q];
                    for (int c = 0; c < 3; ++c) gj[c] += w * (a * u[c] + b * dY[((size_t)j * nlm + k) * 3 + c]);
                }
        }
    }
    free(A); free(om); free(R); free(dR); free(Y); free(dY); free(rr);
    return E;
}

/* Site energy of the cheap potential:
 * E_i = 1/2 sum_j V2(r_ij) + sum_{j<k; r_ij, r_ik < rc3} V3(r_ij, r_ik, r_jk). */
static double spl_site(const ospl* S, int nn, const double* rij, double* g) {
    double E = 0.0;
    double* rr = (double*)malloc(sizeof(double) * (size_t)(nn > 0 ? nn : 1));
    if (g) memset(g, 0, sizeof(double) * 3 * (size_t)nn);
    for (int j = 0; j < nn; ++j) {
        const double* d = rij + 3 * j;
        double r = sqrt(norm2(d));
        rr[j] = r;
        if (!(r < S->rc)) continue;
        double v, dv;
        spline1(S->c2, 16, S->t2, r, &v, &dv);
        E += 0.5 * v;
        if (g)
            for (int c = 0; c < 3; ++c) g[3 * j + c] += 0.5 * dv * d[c] / r;
    }
    for (int j = 0; j < nn; ++j) {
        if (!(rr[j] < S->rc3)) continue;
        for (int k = j + 1; k < nn; ++k) {
            if (!(rr[k] < S->rc3)) continue;
            const double* dj = rij + 3 * j;
            const double* dk = rij + 3 * k;
            double w[3] = {dk[0] - dj[0], dk[1] - dj[1], dk[2] - dj[2]};
            double r3 = sqrt(norm2(w));
            double ba[8], bb[8], bc[8], dba[8], dbb[8], dbc[8];
            for (int a = 0; a < 8; ++a) {
                ba[a] = bsp(S->t3a, a, 3, rr[j]);
                dba[a] = bsp_d(S->t3a, a, 3, rr[j]);
                bb[a] = bsp(S->t3a, a, 3, rr[k]);
                dbb[a] = bsp_d(S->t3a, a, 3, rr[k]);
                bc[a] = bsp(S->t3c, a, 3, r3);
                dbc[a] = bsp_d(S->t3c, a, 3, r3);
            }
            double V = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
            for (int a = 0; a < 8; ++a)
                for (int b = 0; b < 8; ++b)
                    for (int c = 0; c < 8; ++c) {
                        double cf = S->c3[(a * 8 + b) * 8 + c];
                        if (cf == 0.0) continue;
                        V += cf * ba[a] * bb[b] * bc[c];
                        d1 += cf * dba[a] * bb[b] * bc[c];
                        d2 += cf * ba[a] * dbb[b] * bc[c];
                        d3 += cf * ba[a] * bb[b] * dbc[c];
                    }
            E += V;
            if (g) {
                for (int c = 0; c < 3; ++c) {
                    double uj = dj[c] / rr[j], uk = dk[c] / rr[k], uw = (r3 > 0) ? w[c] / r3 : 0.0;
                    g[3 * j + c] += d1 * uj - d3 * uw;
                    g[3 * k + c] += d2 * uk + d3 * uw;
                }
            }
        }
    }
    free(rr);
    return E;
}

/* ------------------------------------------------------------------------- */
/* model: system + both potentials + regions                                  */

typedef struct {
    int64_t n;
    obox box;
    double mass;
    oace* ace;
    ospl* spl;
    int nreg;
    double reg[MAXREG][9]; /* kind, c[3], axis[3] (unit), r_core, ramp */
    int blend;             /* 0 linear, 1 cubic (smoothstep of the linear ramp) */
    double buf_e, buf_c;
    int atomic;            /* 1: weights from seed atoms (Alg. 1-2) instead of regions */
    uint8_t* seed;         /* [n] seed atoms */
    double a_core, a_blend;
} omodel;

void* or_model_new(int64_t n, const double* lo, const double* L, const int* per, double mass, double ace_rc,
                   int ace_n, int ace_L, int ace_nu, const double* c1, const double* c2, const double* c3,
                   const double* pair, double spl_rc, double spl_rc3, const double* s2, const double* s3,
                   int nreg, const double* regs, int blend, double buf_e, double buf_c) {
    if (nreg < 0 || nreg > MAXREG) return NULL;
    omodel* m = (omodel*)calloc(1, sizeof(omodel));
    m->n = n;
    box_init(&m->box, lo, L, per);
    m->mass = mass;
    m->ace = ace_new(ace_rc, ace_n, ace_L, ace_nu, c1, c2, c3, pair);
    m->spl = spl_new(spl_rc, spl_rc3, s2, s3);
    if (!m->ace || !m->spl) {
        ace_free(m->ace);
        free(m->spl);
        free(m);
        return NULL;
    }
    m->nreg = nreg;
    for (int r = 0; r < nreg; ++r) {
        for (int k = 0; k < 9; ++k) m->reg[r][k] = regs[9 * r + k];
        double* ax = &m->reg[r][4];
        double nrm = sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
        if (nrm > 0) {
            ax[0] = ax[0] / nrm;
            ax[1] = ax[1] / nrm;
            ax[2] = ax[2] / nrm;
        }
    }
    m->blend = blend;
    m->buf_e = buf_e > 0 ? buf_e : ace_rc;
    m->buf_c = buf_c > 0 ? buf_c : spl_rc;
    return m;
}

void or_model_free(void* p) {
    omodel* m = (omodel*)p;
    if (!m) return;
    ace_free(m->ace);
    free(m->spl);
    free(m->seed);
    free(m);
}

int or_model_basis_count(void* p) { return or_ace_basis_count(((omodel*)p)->ace); }

void or_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Region weights (Alg. 2, geometric reading): distance d from the region
 * (sphere: to the centre; cylinder: to the axis line), lambda = 1 for d < r_core,
 * 1 - (d - r_core)/ramp for d < r_core + ramp, else 0; maximum over regions.
 * lam = the linear ramp (defines the sets), w = the blend weight. */
static void lambda_one(const omodel* m, const double* x, double* lam, double* w) {
    double best = 0.0;
    for (int r = 0; r < m->nreg; ++r) {
        const double* R = m->reg[r];
        double v[3];
        box_delta(&m->box, &R[1], x, v);
        double d2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        if ((int)R[0] == 1) {
            double t = v[0] * R[4] + v[1] * R[5] + v[2] * R[6];
            d2 = d2 - t * t;
            if (d2 < 0.0) d2 = 0.0;
        }
        double d = sqrt(d2);
        double rc = R[7], ramp = R[8], lr;
        if (d < rc)
            lr = 1.0;
        else if (ramp > 0.0 && d < rc + ramp)
            lr = 1.0 - (d - rc) / ramp;
        else
            lr = 0.0;
        if (lr > best) best = lr;
    }
    *lam = best;
    if (m->blend == 1)
        *w = best * best * (3.0 - 2.0 * best);
    else
        *w = best;
}

typedef struct {
    int cap;
    int* nnb;
    int* nbr;
} olist;
static int list_build(const omodel* m, const double* x, double rc, olist* L);
static void list_free(olist* L);

/* Weights from seed atoms, Alg. 1 then Alg. 2 as written: every seed and every
 * neighbour of a seed closer than r_core is a core atom with weight 1; then for
 * every core atom i and neighbour j closer than r_blend the weight of j becomes
 * max(weight, 1 - r_ij / r_blend).  Distances compared squared (r2 < r_core^2,
 * r2 < r_blend^2), r = sqrt(r2). */
static int lambda_atomic(const omodel* m, const double* x, double* lam) {
    int64_t n = m->n;
    size_t nz = (size_t)(n > 0 ? n : 1);
    uint8_t* core = (uint8_t*)calloc(nz, 1);
    for (int64_t i = 0; i < n; ++i) lam[i] = 0.0;
    olist L;
    double rmax = m->a_core > m->a_blend ? m->a_core : m->a_blend;
    int st = list_build(m, x, rmax, &L);
    if (st) {
        free(core);
        return st;
    }
    double rc2 = m->a_core * m->a_core, rb2 = m->a_blend * m->a_blend;
    for (int64_t i = 0; i < n; ++i) {
        if (!m->seed[i]) continue;
        core[i] = 1;
        lam[i] = 1.0;
        for (int k = 0; k < L.nnb[i]; ++k) {
            int j = L.nbr[(size_t)L.cap * i + k];
            double d[3];
            box_delta(&m->box, x + 4 * i, x + 4 * (int64_t)j, d);
            if (norm2(d) < rc2) {
                core[j] = 1;
                lam[j] = 1.0;
            }
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        if (!core[i]) continue;
        for (int k = 0; k < L.nnb[i]; ++k) {
            int j = L.nbr[(size_t)L.cap * i + k];
            double d[3];
            box_delta(&m->box, x + 4 * i, x + 4 * (int64_t)j, d);
            double r2 = norm2(d);
            if (r2 < rb2) {
                double v = 1.0 - sqrt(r2) / m->a_blend;
                if (v > lam[j]) lam[j] = v;
            }
        }
    }
    list_free(&L);
    free(core);
    return OR_OK;
}

void or_lambda(void* p, const double* x, double* lam, double* w) {
    omodel* m = (omodel*)p;
    if (m->atomic) {
        lambda_atomic(m, x, lam);
        for (int64_t i = 0; i < m->n; ++i) {
            double b = lam[i];
            w[i] = m->blend == 1 ? b * b * (3.0 - 2.0 * b) : b;
        }
        return;
    }
    for (int64_t i = 0; i < m->n; ++i) lambda_one(m, x + 4 * i, lam + i, w + i);
}

/* Switch the model to seed-atom weights (seed: [n] 0/1, NULL switches back to
 * the geometric regions). */
int or_set_atomic(void* p, const uint8_t* seed, double r_core, double r_blend) {
    omodel* m = (omodel*)p;
    free(m->seed);
    m->seed = NULL;
    m->atomic = 0;
    if (!seed) return OR_OK;
    if (!(r_core >= 0) || !(r_blend >= 0)) return OR_EINVAL;
    m->seed = (uint8_t*)malloc((size_t)(m->n > 0 ? m->n : 1));
    memcpy(m->seed, seed, (size_t)m->n);
    m->a_core = r_core;
    m->a_blend = r_blend;
    m->atomic = 1;
    return OR_OK;
}

/* Coordination: number of neighbours closer than r (strict) of every atom. */
int or_coordination(void* p, const double* x, double r, int* z) {
    omodel* m = (omodel*)p;
    olist L;
    int st = list_build(m, x, r, &L);
    if (st) return st;
    for (int64_t i = 0; i < m->n; ++i) z[i] = L.nnb[i];
    list_free(&L);
    return OR_OK;
}

/* flags bit0: lambda > 0 (Lambda_e), bit1: lambda < 1 (Lambda_c),
 *       bit2: evaluated with the expensive potential (Lambda_e or its buffer),
 *       bit3: evaluated with the cheap potential (Lambda_c or its buffer).
 * Buffer of a set S with radius b: atoms outside S with some member of S
 * closer than b (strict). */
/* environment of atom i: neighbours within rc (from a fresh list) as r_ij vectors */
static int list_build(const omodel* m, const double* x, double rc, olist* L) {
    int64_t n = m->n;
    L->cap = 128;
    for (;;) {
        L->nnb = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
        L->nbr = (int*)malloc(sizeof(int) * (size_t)L->cap * (size_t)(n > 0 ? n : 1));
        if (!L->nnb || !L->nbr) return OR_ENOMEM;
        int st = neighbours_cells(&m->box, n, x, rc, L->cap, L->nnb, L->nbr);
        if (st == OR_EOVERFLOW) {
            free(L->nnb); free(L->nbr);
            L->cap *= 2;
            continue;
        }
        return st;
    }
}

static void list_free(olist* L) {
    free(L->nnb);
    free(L->nbr);
}

int or_sets(void* p, const double* x, uint8_t* flags) {
    omodel* m = (omodel*)p;
    int64_t n = m->n;
    double* lam = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    or_lambda(p, x, lam, w);
    double rb = m->buf_e > m->buf_c ? m->buf_e : m->buf_c;
    olist NL;
    int st = list_build(m, x, rb, &NL);
    if (st) {
        free(lam); free(w);
        return st;
    }
    int cap = NL.cap;
    int* nnb = NL.nnb;
    int* nbr = NL.nbr;
    double be2 = m->buf_e * m->buf_e, bc2 = m->buf_c * m->buf_c;
    for (int64_t i = 0; i < n; ++i) {
        uint8_t f = 0;
        if (lam[i] > 0.0) f |= 1;
        if (lam[i] < 1.0) f |= 2;
        flags[i] = f;
    }
    for (int64_t i = 0; i < n; ++i) {
        uint8_t f = flags[i];
        int ine = (f & 1) != 0, inc = (f & 2) != 0;
        if (ine) f |= 4;
        if (inc) f |= 8;
        for (int k = 0; k < nnb[i] && (!(f & 4) || !(f & 8)); ++k) {
            int j = nbr[(size_t)cap * i + k];
            double d[3];
            box_delta(&m->box, x + 4 * i, x + 4 * (int64_t)j, d);
            double r2 = norm2(d);
            if (!(f & 4) && (flags[j] & 1) && r2 < be2) f |= 4;
            if (!(f & 8) && (flags[j] & 2) && r2 < bc2) f |= 8;
        }
        flags[i] = (uint8_t)((flags[i] & 3) | (f & 12));
    }
    free(lam); free(w); free(nnb); free(nbr);
    return OR_OK;
}

/* which: 0 expensive, 1 cheap.  Site energy and pair gradients of atom i. */
static double site_eval(const omodel* m, int which, const double* x, const olist* L, int64_t i, double* g) {
    int nn = L->nnb[i];
    double* rij = (double*)malloc(sizeof(double) * 3 * (size_t)(nn > 0 ? nn : 1));
    for (int k = 0; k < nn; ++k) {
        int j = L->nbr[(size_t)L->cap * i + k];
        box_delta(&m->box, x + 4 * i, x + 4 * (int64_t)j, rij + 3 * k);
    }
    double E = which == 0 ? ace_site(m->ace, nn, rij, g, NULL, NULL) : spl_site(m->spl, nn, rij, g);
    free(rij);
    return E;
}

/* Forces of one potential with only the atoms in `active` (NULL = all) as
 * centres: Fp_k = -d(sum_{i active} E_i)/dx_k, written as a scatter of the
 * pair gradients (Sec. 4.5 force equation; Alg. 4 "compute()"). */
static int pot_forces(const omodel* m, int which, const double* x, const uint8_t* active, double* Fp,
                      double* Esite) {
    int64_t n = m->n;
    double rc = which == 0 ? m->ace->rc : m->spl->rc;
    olist L;
    int st = list_build(m, x, rc, &L);
    if (st) return st;
    double** gs = (double**)calloc((size_t)(n > 0 ? n : 1), sizeof(double*));
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : err)
    for (int64_t i = 0; i < n; ++i) {
        if (active && !active[i]) {
            if (Esite) Esite[i] = 0.0;
            continue;
        }
        int nn = L.nnb[i];
        gs[i] = (double*)malloc(sizeof(double) * 3 * (size_t)(nn > 0 ? nn : 1));
        if (!gs[i]) { err = 1; continue; }
        double E = site_eval(m, which, x, &L, i, gs[i]);
        if (Esite) Esite[i] = E;
    }
    memset(Fp, 0, sizeof(double) * 4 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        if (!gs[i]) continue;
        for (int k = 0; k < L.nnb[i]; ++k) {
            int j = L.nbr[(size_t)L.cap * i + k];
            for (int c = 0; c < 3; ++c) {
                Fp[4 * (int64_t)j + c] -= gs[i][3 * k + c];
                Fp[4 * i + c] += gs[i][3 * k + c];
            }
        }
        free(gs[i]);
    }
    free(gs);
    list_free(&L);
    return err ? OR_ENOMEM : OR_OK;
}

/* mode 0: force mixing as the method does it (each potential on its evaluated
 *         set = Lambda_k plus buffer, Alg. 4);
 * mode 1: the plain definition w F_exp,full + (1 - w) F_cheap,full;
 * mode 2: pure expensive; mode 3: pure cheap.
 * Ee, Ec (nullable): site energies (0 where not evaluated). */
int or_forces(void* p, const double* x, int mode, double* F, double* Ee, double* Ec) {
    omodel* m = (omodel*)p;
    int64_t n = m->n;
    size_t nz = (size_t)(n > 0 ? n : 1);
    double* Fe = (double*)calloc(4 * nz, sizeof(double));
    double* Fc = (double*)calloc(4 * nz, sizeof(double));
    double* lam = (double*)malloc(sizeof(double) * nz);
    double* w = (double*)malloc(sizeof(double) * nz);
    uint8_t* flags = (uint8_t*)malloc(nz);
    uint8_t* act = (uint8_t*)malloc(nz);
    int st = OR_OK;
    if (mode == 2) {
        st = pot_forces(m, 0, x, NULL, F, Ee);
        if (Ec) memset(Ec, 0, sizeof(double) * nz);
        goto done;
    }
    if (mode == 3) {
        st = pot_forces(m, 1, x, NULL, F, Ec);
        if (Ee) memset(Ee, 0, sizeof(double) * nz);
        goto done;
    }
    or_lambda(p, x, lam, w);
    if (mode == 0) {
        st = or_sets(p, x, flags);
        if (st) goto done;
        for (int64_t i = 0; i < n; ++i) act[i] = (flags[i] & 4) ? 1 : 0;
        st = pot_forces(m, 0, x, act, Fe, Ee);
        if (st) goto done;
        for (int64_t i = 0; i < n; ++i) act[i] = (flags[i] & 8) ? 1 : 0;
        st = pot_forces(m, 1, x, act, Fc, Ec);
        if (st) goto done;
    } else {
        st = pot_forces(m, 0, x, NULL, Fe, Ee);
        if (st) goto done;
        st = pot_forces(m, 1, x, NULL, Fc, Ec);
        if (st) goto done;
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < 3; ++c) F[4 * i + c] = w[i] * Fe[4 * i + c] + (1.0 - w[i]) * Fc[4 * i + c];
        F[4 * i + 3] = 0.0;
    }
done:
    free(Fe); free(Fc); free(lam); free(w); free(flags); free(act);
    return st;
}

/* Mixed forces (method form) on a sample of atoms only: each sampled atom's
 * force needs the site gradients of itself and of its evaluated neighbours. */
int or_forces_sampled(void* p, const double* x, int ns, const int64_t* idx, double* Fs) {
    omodel* m = (omodel*)p;
    int64_t n = m->n;
    size_t nz = (size_t)(n > 0 ? n : 1);
    double* lam = (double*)malloc(sizeof(double) * nz);
    double* w = (double*)malloc(sizeof(double) * nz);
    uint8_t* flags = (uint8_t*)malloc(nz);
    or_lambda(p, x, lam, w);
    int st = or_sets(p, x, flags);
    if (st) {
        free(lam); free(w); free(flags);
        return st;
    }
    for (int which = 0; which < 2; ++which) {
        double rc = which == 0 ? m->ace->rc : m->spl->rc;
        uint8_t bit = which == 0 ? 4 : 8;
        olist L;
        st = list_build(m, x, rc, &L);
        if (st) break;
#pragma omp parallel for schedule(dynamic, 1)
        for (int s = 0; s < ns; ++s) {
            int64_t k = idx[s];
            double acc[3] = {0, 0, 0};
            double wk = which == 0 ? w[k] : 1.0 - w[k];
            if (wk != 0.0) {
                int nn = L.nnb[k];
                double* g = (double*)malloc(sizeof(double) * 3 * (size_t)(L.cap));
                if (flags[k] & bit) {
                    site_eval(m, which, x, &L, k, g);
                    for (int q = 0; q < nn; ++q)
                        for (int c = 0; c < 3; ++c) acc[c] += g[3 * q + c];
                }
                for (int q = 0; q < nn; ++q) {
                    int j = L.nbr[(size_t)L.cap * k + q];
                    if (!(flags[j] & bit)) continue;
                    site_eval(m, which, x, &L, j, g);
                    for (int t = 0; t < L.nnb[j]; ++t)
                        if (L.nbr[(size_t)L.cap * j + t] == (int)k)
                            for (int c = 0; c < 3; ++c) acc[c] -= g[3 * t + c];
                }
                free(g);
            }
            for (int c = 0; c < 3; ++c) {
                double v = wk * acc[c];
                if (which == 0) Fs[4 * s + c] = v;
                else Fs[4 * s + c] += v;
            }
            Fs[4 * s + 3] = 0.0;
        }
        list_free(&L);
    }
    free(lam); free(w); free(flags);
    return st;
}

/* single-environment evaluation, for finite-difference and invariance checks.
 * which: 0 expensive, 1 cheap.  basis (nullable) gets the expensive basis values. */
double or_site(void* p, int which, int nn, const double* rij, double* g, double* basis) {
    omodel* m = (omodel*)p;
    if (which == 0) return ace_site(m->ace, nn, rij, g, basis, NULL);
    return spl_site(m->spl, nn, rij, g);
}

/* atomic density A[n][lm] of one environment */
void or_density(void* p, int nn, const double* rij, double* A) {
    omodel* m = (omodel*)p;
    ace_site(m->ace, nn, rij, NULL, NULL, A);
}

/* Velocity Verlet, nsteps steps of dt fs with forces of the given mode:
 *   v += (dt/2) kappa F / m;  x += dt v;  F = F(x);  v += (dt/2) kappa F / m.
 * F must hold the forces at the incoming x.  epot (nullable, [nsteps]) gets the
 * total site energy of the pure potential in modes 2 and 3. */
int or_md(void* p, double* x, double* v, double* F, double dt, int nsteps, int mode, double* epot) {
    omodel* m = (omodel*)p;
    int64_t n = m->n;
    double h = 0.5 * dt * KAPPA / m->mass;
    double* Es = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int st = OR_OK;
    for (int s = 0; s < nsteps; ++s) {
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) {
                v[4 * i + c] = v[4 * i + c] + h * F[4 * i + c];
                x[4 * i + c] = x[4 * i + c] + dt * v[4 * i + c];
            }
        st = or_forces(p, x, mode, F, mode == 3 ? NULL : Es, mode == 3 ? Es : NULL);
        if (st) break;
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) v[4 * i + c] = v[4 * i + c] + h * F[4 * i + c];
        if (epot) {
            double e = 0.0;
            for (int64_t i = 0; i < n; ++i) e += Es[i];
            epot[s] = e;
        }
    }
    free(Es);
    return st;
}
