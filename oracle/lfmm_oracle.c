/*
 * lfmm_oracle.c -- plain, slow FP64 CPU oracle for the layered-media Laplace
 * potential of Wang, Zhang & Cai, "Fast multipole method for 3-D Laplace
 * equation in layered media" (arXiv 1908.10863).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (all definitions, no fast algorithm):
 *   - reaction densities sigma^{ab}_{l l'}(k) by solving, for each k, the
 *     spectral interface problem of Appendix A (eqs. A.1-A.3) directly as a
 *     2L x 2L linear system (Gaussian elimination, partial pivoting);
 *   - the explicit three-layer densities printed in Appendix A
 *     (densitythreelayer1-3), with the two corrections that the linear solve
 *     fixes (kappa sign, sigma^{22}_{22} numerator), as a cross-check;
 *   - Sommerfeld-type integrals K_{N,mu}(rho,z) = int_0^inf J_mu(k rho) k^N
 *     e^{-kz} sigma(k) dk (the unnormalised form of eq. uniformintegral) by
 *     adaptive Gauss-Kronrod (7/15) on the real axis;
 *   - for three layers, the exact image series obtained by expanding the
 *     closed-form densities as a geometric series in e^{-k(d0-d1)}; every term
 *     integrates to a closed form (Legendre function over a distance power);
 *   - the potential Phi and field E = -grad Phi at target charges by direct
 *     summation over all source charges of the free-space part plus the
 *     reaction components (eqs. potential1, totalinteraction,
 *     generalcomponents, zexponential), with the 1/(4 pi) factor included,
 *     the free-space self term excluded and the reaction self term included.
 *
 * Parity is pinned by the tests (closed forms, two-layer image charge,
 * reciprocity, harmonicity, transmission conditions, sigma==1 identity).
 */
#define _DEFAULT_SOURCE 1 /* j0, j1, jn from the C library */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXL 8 /* interfaces */
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Spectral interface problem (Appendix A).                            */
/* Layer j occupies d_j < z < d_{j-1} (d_{-1}=+inf, d_L=-inf).  In     */
/* layer j the reaction part of the transformed Green's function (times */
/* 2k) is a_j e^{-k(z-d_j)} + b_j e^{-k(d_{j-1}-z)}, with b_0 = a_L = 0. */
/* The source in layer lp contributes e^{-k|z-z'|}; its value at the    */
/* bottom interface d_lp is g1 = e^{-k(z'-d_lp)} and at the top         */
/* interface d_{lp-1} is g2 = e^{-k(d_{lp-1}-z')}.  Interface conditions */
/* (eq. transmissioncond): continuity of u and of eps * du/dz.  With    */
/* g_b = 1 the solution gives sigma^{1b}_{l,lp} = a_l and               */
/* sigma^{2b}_{l,lp} = b_l (eqs. generalcomponents, zexponential).      */
/* ------------------------------------------------------------------ */

static int solve_dense(int n, double* A, double* x) /* A is n x (n+1) */
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * (n + 1) + c]) > fabs(A[piv * (n + 1) + c])) piv = r;
        if (fabs(A[piv * (n + 1) + c]) < 1e-300) return -1;
        if (piv != c)
            for (int j = 0; j <= n; ++j) {
                double t = A[c * (n + 1) + j];
                A[c * (n + 1) + j] = A[piv * (n + 1) + j];
                A[piv * (n + 1) + j] = t;
            }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * (n + 1) + c] / A[c * (n + 1) + c];
            for (int j = c; j <= n; ++j) A[r * (n + 1) + j] -= f * A[c * (n + 1) + j];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = A[r * (n + 1) + n];
        for (int j = r + 1; j < n; ++j) s -= A[r * (n + 1) + j] * x[j];
        x[r] = s / A[r * (n + 1) + r];
    }
    return 0;
}

/* out[(l*2 + a-1)*2 + b-1] = sigma^{ab}_{l,lp}(k); entries of components
 * that do not exist are set to 0.  Returns 0 on success. */
int oracle_sigma(int L, const double* d, const double* eps, double k, int lp, double* out)
{
    if (L < 0 || L > OR_MAXL || lp < 0 || lp > L || k < 0) return -1;
    memset(out, 0, sizeof(double) * 4 * (L + 1));
    if (L == 0) return 0;
    const int n = 2 * L;
    /* unknown index: a_j -> j (j=0..L-1), b_j -> L + j - 1 (j=1..L) */
    for (int b = 1; b <= 2; ++b) {
        if (b == 1 && lp == L) continue; /* no bottom interface */
        if (b == 2 && lp == 0) continue; /* no top interface */
        double A[(2 * OR_MAXL) * (2 * OR_MAXL + 1)];
        double x[2 * OR_MAXL];
        memset(A, 0, sizeof(A));
        for (int j = 0; j < L; ++j) { /* interface d_j: layer j above, j+1 below */
            double* rc = &A[(2 * j) * (n + 1)];     /* continuity */
            double* rf = &A[(2 * j + 1) * (n + 1)]; /* flux */
            /* layer j evaluated at its bottom z = d_j */
            rc[j] += 1.0;
            rf[j] += -eps[j];
            if (j > 0) {
                double e = exp(-k * (d[j - 1] - d[j]));
                rc[L + j - 1] += e;
                rf[L + j - 1] += eps[j] * e;
            }
            /* minus layer j+1 evaluated at its top z = d_j */
            rc[L + j] -= 1.0;
            rf[L + j] -= eps[j + 1];
            if (j + 1 < L) {
                double e = exp(-k * (d[j] - d[j + 1]));
                rc[j + 1] -= e;
                rf[j + 1] -= -eps[j + 1] * e;
            }
            /* free part of the source, moved to the right-hand side.
             * Below the source (z = d_lp < z'): value g1, slope/k = +g1.
             * Above the source (z = d_{lp-1} > z'): value g2, slope/k = -g2. */
            if (b == 1 && j == lp) { rc[n] -= 1.0; rf[n] -= eps[j]; }
            if (b == 2 && j + 1 == lp) { rc[n] -= -1.0; rf[n] -= eps[j + 1]; }
        }
        if (solve_dense(n, A, x)) return -1;
        for (int l = 0; l <= L; ++l) {
            if (l < L) out[(l * 2 + 0) * 2 + (b - 1)] = x[l];
            if (l > 0) out[(l * 2 + 1) * 2 + (b - 1)] = x[L + l - 1];
        }
    }
    return 0;
}

/* Appendix A, explicit three-layer densities (a_l = 1, b_l = eps_l).
 * Written as numerator polynomial (n0 + n1 x + n2 x^2) in x = e^{-k(d0-d1)}
 * over kappa(x) = kappa0 (1 + qq x^2) (the printed forms use d0 = 0, so
 * e^{d1 k} = x).  Two corrections relative to the printed text:
 *   kappa = 1/2[(e0+e1)(e1+e2) + (e0-e1)(e1-e2) x^2]  (printed: (e2-e1)),
 *   sigma^{22}_{22} numerator = (e2-e1)(e0+e1) + (e1-e0)(e1+e2) x^2
 *   (printed with the two eps-products swapped between the x^0 and x^2 terms).
 * Returns 0 and fills num[3] and *den0, *qq such that
 *   sigma = (num0 + num1 x + num2 x^2) / (den0 (1 + qq x^2)),
 * or -1 if the component does not exist. */
int oracle_sigma3_poly(const double* eps, int l, int lp, int a, int b, double* num, double* den0, double* qq)
{
    const double e0 = eps[0], e1 = eps[1], e2 = eps[2];
    const double kap0 = 0.5 * (e0 + e1) * (e1 + e2);
    *qq = (e0 - e1) * (e1 - e2) / ((e0 + e1) * (e1 + e2));
    num[0] = num[1] = num[2] = 0.0;
    *den0 = kap0;
    int key = ((l * 3 + lp) * 2 + (a - 1)) * 2 + (b - 1);
#define KEY(l_, lp_, a_, b_) ((((l_) * 3 + (lp_)) * 2 + ((a_) - 1)) * 2 + ((b_) - 1))
    switch (key) {
    /* source in the top layer (densitythreelayer1) */
    case KEY(0, 0, 1, 1): num[0] = (e0 - e1) * (e1 + e2); num[2] = (e0 + e1) * (e1 - e2); *den0 = 2 * kap0; break;
    case KEY(1, 0, 2, 1): num[0] = e0 * (e1 + e2); break;
    case KEY(1, 0, 1, 1): num[1] = e0 * (e1 - e2); break;
    case KEY(2, 0, 2, 1): num[1] = 2 * e0 * e1; break;
    /* source in the middle layer (densitythreelayer2) */
    case KEY(0, 1, 1, 2): num[0] = e1 * (e1 + e2); break;
    case KEY(0, 1, 1, 1): num[1] = e1 * (e1 - e2); break;
    case KEY(1, 1, 1, 1): num[0] = (e1 - e2) * (e1 + e0); *den0 = 2 * kap0; break;
    case KEY(1, 1, 2, 1): num[1] = (e1 - e2) * (e1 - e0); *den0 = 2 * kap0; break;
    case KEY(1, 1, 1, 2): num[1] = (e1 - e2) * (e1 - e0); *den0 = 2 * kap0; break;
    case KEY(1, 1, 2, 2): num[0] = (e1 + e2) * (e1 - e0); *den0 = 2 * kap0; break;
    case KEY(2, 1, 2, 2): num[1] = e1 * (e1 - e0); break;
    case KEY(2, 1, 2, 1): num[0] = e1 * (e0 + e1); break;
    /* source in the bottom layer (densitythreelayer3) */
    case KEY(0, 2, 1, 2): num[1] = 2 * e1 * e2; break;
    case KEY(1, 2, 2, 2): num[1] = e2 * (e1 - e0); break;
    case KEY(1, 2, 1, 2): num[0] = e2 * (e0 + e1); break;
    case KEY(2, 2, 2, 2): num[0] = (e2 - e1) * (e0 + e1); num[2] = (e1 - e0) * (e1 + e2); *den0 = 2 * kap0; break;
    default: return -1;
    }
#undef KEY
    return 0;
}

int oracle_sigma3_closed(const double* d, const double* eps, double k, int l, int lp, int a, int b, double* out)
{
    double num[3], den0, qq;
    if (oracle_sigma3_poly(eps, l, lp, a, b, num, &den0, &qq)) return -1;
    double x = exp(-k * (d[0] - d[1]));
    *out = (num[0] + num[1] * x + num[2] * x * x) / (den0 * (1.0 + qq * x * x));
    return 0;
}

/* ------------------------------------------------------------------ */
/* Component bookkeeping (eqs. reactioncomponent, zexponential).       */
/* ------------------------------------------------------------------ */
static int comp_exists(int L, int l, int lp, int a, int b)
{
    if (L == 0) return 0;
    if (a == 1 && l == L) return 0;
    if (a == 2 && l == 0) return 0;
    if (b == 1 && lp == L) return 0;
    if (b == 2 && lp == 0) return 0;
    return 1;
}

/* exponent distance of Z^{ab}_{l l'}(z,z') and its derivative d/dz */
static double comp_h(const double* d, int l, int lp, int a, int b, double z, double zp, double* dhdz)
{
    double t = (a == 1) ? (z - d[l]) : (d[l - 1] - z);
    double s = (b == 1) ? (zp - d[lp]) : (d[lp - 1] - zp);
    *dhdz = (a == 1) ? 1.0 : -1.0;
    return t + s;
}

/* ------------------------------------------------------------------ */
/* Adaptive Gauss-Kronrod (7-point Gauss, 15-point Kronrod).           */
/* ------------------------------------------------------------------ */
static const double gk_x[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                               0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                               0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                               0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double gk_wk[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                                0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                                0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                                0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double gk_wg[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                                0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

#define GK_MAXDIM 4
typedef void (*vec_integrand)(double k, const void* ctx, double* f);

static void gk15(vec_integrand fn, const void* ctx, int dim, double a, double b, double* K, double* err)
{
    double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double fc[GK_MAXDIM], f1[GK_MAXDIM], f2[GK_MAXDIM], G[GK_MAXDIM];
    fn(c, ctx, fc);
    for (int i = 0; i < dim; ++i) { K[i] = gk_wk[7] * fc[i]; G[i] = gk_wg[3] * fc[i]; }
    for (int j = 0; j < 7; ++j) {
        fn(c - h * gk_x[j], ctx, f1);
        fn(c + h * gk_x[j], ctx, f2);
        for (int i = 0; i < dim; ++i) {
            K[i] += gk_wk[j] * (f1[i] + f2[i]);
            if (j & 1) G[i] += gk_wg[j / 2] * (f1[i] + f2[i]);
        }
    }
    for (int i = 0; i < dim; ++i) { K[i] *= h; G[i] *= h; err[i] = fabs(K[i] - G[i]); }
}

typedef struct { double a, b, K[GK_MAXDIM], E[GK_MAXDIM]; } gk_panel;

/* Globally adaptive: keep bisecting the panel with the largest error until
 * the summed error is below tol * (sum of |panel integrals|) + floor[c] per
 * component (floor may be NULL: no absolute part).  Returns 0 when that holds.  When the panel budget runs out first it
 * returns 1 and writes NaN to every output, so that an unconverged sum can
 * never pass for a result. */
static int gk_adaptive(vec_integrand fn, const void* ctx, int dim, double a, double b, int npanel0, double tol,
                       const double* floor, double* out)
{
    enum { MAXP = 20000 };
    gk_panel* P = (gk_panel*)malloc(sizeof(gk_panel) * MAXP);
    int np = 0, status = 1;
    if (!P) {
        for (int c = 0; c < dim; ++c) out[c] = NAN;
        return 1;
    }
    if (npanel0 < 1) npanel0 = 1;
    if (npanel0 > MAXP / 2) npanel0 = MAXP / 2;
    for (int i = 0; i < npanel0; ++i) {
        P[np].a = a + (b - a) * i / npanel0;
        P[np].b = a + (b - a) * (i + 1) / npanel0;
        gk15(fn, ctx, dim, P[np].a, P[np].b, P[np].K, P[np].E);
        ++np;
    }
    for (;;) {
        double tot[GK_MAXDIM] = {0}, scale[GK_MAXDIM] = {0}, errs[GK_MAXDIM] = {0};
        for (int i = 0; i < np; ++i)
            for (int c = 0; c < dim; ++c) { tot[c] += P[i].K[c]; scale[c] += fabs(P[i].K[c]); errs[c] += P[i].E[c]; }
        int done = 1;
        for (int c = 0; c < dim; ++c)
            if (!(errs[c] <= tol * scale[c] + (floor ? floor[c] : 0.0) + 1e-300)) done = 0;
        if (done) {
            for (int c = 0; c < dim; ++c) out[c] = tot[c];
            status = 0;
            break;
        }
        if (np >= MAXP - 1) {
            for (int c = 0; c < dim; ++c) out[c] = NAN;
            break;
        }
        /* bisect the worst panel (worst relative to its component scale) */
        int w = 0;
        double wv = -1.0;
        for (int i = 0; i < np; ++i) {
            double v = 0;
            for (int c = 0; c < dim; ++c) {
                double r = P[i].E[c] / (scale[c] + 1e-300);
                if (r > v) v = r;
            }
            if (v > wv) { wv = v; w = i; }
        }
        double m = 0.5 * (P[w].a + P[w].b);
        P[np].a = m; P[np].b = P[w].b;
        P[w].b = m;
        gk15(fn, ctx, dim, P[w].a, P[w].b, P[w].K, P[w].E);
        gk15(fn, ctx, dim, P[np].a, P[np].b, P[np].K, P[np].E);
        ++np;
    }
    free(P);
    return status;
}

/* ------------------------------------------------------------------ */
/* Sommerfeld-type integral K_{N,mu}(rho, z) (eq. uniformintegral       */
/* without the 1/sqrt((N+mu)!(N-mu)!) normalisation).                  */
/* ------------------------------------------------------------------ */
typedef struct {
    int L;
    const double *d, *eps;
    int l, lp, a, b, N, mu, sigma_mode;
    double rho, z;
} knm_ctx;

static double sigma_one(const knm_ctx* c, double k)
{
    if (c->sigma_mode == 1) return 1.0;
    double s[4 * (OR_MAXL + 1)];
    if (oracle_sigma(c->L, c->d, c->eps, k, c->lp, s)) return NAN;
    return s[(c->l * 2 + c->a - 1) * 2 + c->b - 1];
}

static void knm_integrand(double k, const void* vctx, double* f)
{
    const knm_ctx* c = (const knm_ctx*)vctx;
    double j = (c->mu == 0) ? j0(k * c->rho) : (c->mu == 1) ? j1(k * c->rho) : jn(c->mu, k * c->rho);
    f[0] = j * pow(k, c->N) * exp(-k * c->z) * sigma_one(c, k);
}

/* sigma_mode: 0 = density from the spectral solve, 1 = sigma == 1. */
double oracle_sommerfeld_K(int L, const double* d, const double* eps, int l, int lp, int a, int b, int N, int mu,
                           double rho, double z, int sigma_mode, double tol)
{
    if (z <= 0 || N < 0 || mu < 0 || mu > N) return NAN;
    if (sigma_mode == 0 && !comp_exists(L, l, lp, a, b)) return NAN;
    knm_ctx c = {L, d, eps, l, lp, a, b, N, mu, sigma_mode, rho, z};
    /* integrand ~ k^N e^{-kz}: negligible beyond (N + 50)/z */
    double kmax = (N + 50.0 + 2.0 * sqrt((double)N + 1.0) * 6.0) / z;
    int np = 8 + (int)ceil(kmax * rho / OR_PI);
    double out;
    gk_adaptive(knm_integrand, &c, 1, 0.0, kmax, np, tol, NULL, &out); /* NaN if unconverged */
    return out;
}

/* Associated Legendre function without the Condon-Shortley phase,
 * Pbar_n^m(x) = (1-x^2)^{m/2} d^m P_n / dx^m, by the textbook upward
 * recurrence in n. */
static double legendre_nocs(int n, int m, double x)
{
    double s = sqrt(fmax(0.0, (1.0 - x) * (1.0 + x)));
    double pmm = 1.0;
    for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * s;
    if (n == m) return pmm;
    double p1 = x * (2.0 * m + 1.0) * pmm;
    if (n == m + 1) return p1;
    double p0 = pmm;
    for (int k = m + 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k + m - 1.0) * p0) / (k - m);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

double oracle_legendre_nocs(int n, int m, double x) { return legendre_nocs(n, m, x); }

/* Closed form int_0^inf J_mu(k rho) k^N e^{-k Z} dk = (N-mu)! Pbar_N^mu(Z/R) / R^{N+1}. */
static double free_K(int N, int mu, double rho, double Z)
{
    double R = sqrt(rho * rho + Z * Z);
    double f = 1.0;
    for (int i = 2; i <= N - mu; ++i) f *= i;
    return f * legendre_nocs(N, mu, Z / R) / pow(R, N + 1);
}

/* Three-layer image series of K_{N,mu}: sigma = sum_i c_i x^i, x = e^{-kD}. */
double oracle_sommerfeld_K_images(const double* d, const double* eps, int l, int lp, int a, int b, int N, int mu,
                                  double rho, double z)
{
    double num[3], den0, qq;
    if (oracle_sigma3_poly(eps, l, lp, a, b, num, &den0, &qq)) return NAN;
    const double D = d[0] - d[1];
    double nmax = fmax(fabs(num[0]), fmax(fabs(num[1]), fabs(num[2])));
    double sum = 0.0, g = 1.0; /* g = (-qq)^j */
    for (int j = 0; j < 100000; ++j) {
        for (int t = 0; t < 3; ++t)
            if (num[t] != 0.0) sum += g * num[t] / den0 * free_K(N, mu, rho, z + (2 * j + t) * D);
        g *= -qq;
        if (fabs(g) * nmax / (1.0 - fabs(qq)) < 1e-18 * nmax) break;
    }
    return sum;
}

/* ------------------------------------------------------------------ */
/* Direct summation of Phi and E (eqs. potential1, totalinteraction).  */
/* ------------------------------------------------------------------ */
typedef struct {
    int L;
    const double *d, *eps;
    int l, lp;
    double rho, z, zp;
    int sigma_mode; /* 0 spectral solve, 1 sigma==1 (fake density for tests) */
    const double* s_inf; /* sigma(k -> inf) per component, subtracted (mode 0) */
} pair_ctx;

/* With s(k) = sigma(k) - sigma_inf (mode 0) or s = 1 (mode 1):
 * f[0] = sum_ab e^{-k h} s J0(k rho)
 * f[1] = d/dz of the same
 * f[2] = d/drho of the same */
static void pair_integrand(double k, const void* vctx, double* f)
{
    const pair_ctx* c = (const pair_ctx*)vctx;
    double s[4 * (OR_MAXL + 1)];
    if (c->sigma_mode == 0) {
        if (oracle_sigma(c->L, c->d, c->eps, k, c->lp, s)) { f[0] = f[1] = f[2] = NAN; return; }
    }
    double J0 = j0(k * c->rho), J1 = j1(k * c->rho);
    double F = 0.0, Fz = 0.0;
    for (int a = 1; a <= 2; ++a)
        for (int b = 1; b <= 2; ++b) {
            if (!comp_exists(c->L, c->l, c->lp, a, b)) continue;
            double dh;
            double h = comp_h(c->d, c->l, c->lp, a, b, c->z, c->zp, &dh);
            int ci = (c->l * 2 + a - 1) * 2 + b - 1;
            double sg = (c->sigma_mode == 1) ? 1.0 : s[ci] - c->s_inf[ci];
            double e = exp(-k * h) * sg;
            F += e;
            Fz += -k * dh * e;
        }
    f[0] = J0 * F;
    f[1] = J0 * Fz;
    f[2] = -k * J1 * F;
}

static double min_h(int L, const double* d, int l, int lp, double z, double zp)
{
    double m = INFINITY, dh;
    for (int a = 1; a <= 2; ++a)
        for (int b = 1; b <= 2; ++b)
            if (comp_exists(L, l, lp, a, b)) m = fmin(m, comp_h(d, l, lp, a, b, z, zp, &dh));
    return m;
}

/* Reaction Green's function sum_ab u^{ab}_{l,lp}(r, r') (times 4 pi) and its
 * target gradient (eqs. generalcomponents, zexponential).
 *
 * Mode 0 (density from the spectral solve).  As k -> inf the interfaces
 * decouple, and sigma(k) tends to sigma_inf, the solve with every
 * e^{-k(d_{j-1}-d_j)} set to 0: the single-interface reflection coefficient
 * when the source's and target's interfaces coincide, 0 otherwise.  The
 * integral is split exactly as
 *   int J0(k rho) e^{-kh} sigma dk = sigma_inf / sqrt(rho^2 + h^2)
 *                                  + int J0(k rho) e^{-kh} (sigma - sigma_inf) dk,
 * the first term by the Lipschitz integral int_0^inf J0(k rho) e^{-kh} dk =
 * 1/sqrt(rho^2 + h^2) (and its h and rho derivatives for the field), the
 * second by adaptive Gauss-Kronrod.  sigma - sigma_inf decays at least like
 * e^{-k Dmin}, Dmin the thinnest inner layer (another interface lies at
 * least Dmin away, and any other path adds 2 Dmin), so the quadrature's
 * interval and oscillation count stay bounded as h -> 0, where the unsplit
 * integrand would need 1/h of the range.  With two layers sigma is constant
 * and the second term vanishes.
 *
 * Mode 1 (sigma == 1, the fake density of the tests): the unsplit integral by
 * quadrature, which exercises the quadrature itself.
 *
 * g[0] = 4 pi u, g[1..3] = 4 pi grad u.  Returns 0, or 1 (and NaN in g) when
 * the quadrature did not converge. */
static int reaction_quad(int L, const double* d, const double* eps, int sigma_mode, int l, int lp, const double* r,
                         const double* rp, double tol, double* g)
{
    double dx = r[0] - rp[0], dy = r[1] - rp[1];
    double rho = sqrt(dx * dx + dy * dy);
    double s_inf[4 * (OR_MAXL + 1)];
    memset(s_inf, 0, sizeof(s_inf));
    double G0 = 0.0, Gz = 0.0, Grho = 0.0; /* closed-form part */
    if (sigma_mode == 0) {
        if (oracle_sigma(L, d, eps, INFINITY, lp, s_inf)) { g[0] = g[1] = g[2] = g[3] = NAN; return 1; }
        for (int a = 1; a <= 2; ++a)
            for (int b = 1; b <= 2; ++b) {
                if (!comp_exists(L, l, lp, a, b)) continue;
                double dh, h = comp_h(d, l, lp, a, b, r[2], rp[2], &dh);
                double si = s_inf[(l * 2 + a - 1) * 2 + b - 1];
                double R2 = rho * rho + h * h, R = sqrt(R2);
                G0 += si / R;
                Gz += -si * dh * h / (R2 * R);
                Grho += -si * rho / (R2 * R);
            }
    }
    pair_ctx c = {L, d, eps, l, lp, rho, r[2], rp[2], sigma_mode, s_inf};
    double hmin = min_h(L, d, l, lp, r[2], rp[2]);
    double kmax;
    if (sigma_mode == 0) {
        if (L < 2) { /* sigma constant in k: nothing left to integrate */
            g[0] = G0; g[3] = Gz;
            g[1] = rho > 0 ? Grho * dx / rho : 0.0;
            g[2] = rho > 0 ? Grho * dy / rho : 0.0;
            return 0;
        }
        double Dmin = INFINITY;
        for (int j = 1; j < L; ++j) Dmin = fmin(Dmin, d[j - 1] - d[j]);
        kmax = 60.0 / (hmin + Dmin);
    } else {
        kmax = 48.0 / hmin;
    }
    int np = 4 + (int)ceil(kmax * rho / OR_PI);
    /* Mode 0: the tolerance is relative to the whole integral, closed-form
     * part included, with a floor of 1e-3 of a unit image at the nearest
     * exponent distance (a remainder that vanishes, as with equal
     * permittivities, is then not chased into rounding noise). */
    double Rh = sqrt(rho * rho + hmin * hmin);
    double fl[3] = {tol * (fabs(G0) + 1e-3 / Rh), tol * (fabs(Gz) + 1e-3 / (Rh * Rh)),
                    tol * (fabs(Grho) + 1e-3 / (Rh * Rh))};
    double I[3];
    int st = gk_adaptive(pair_integrand, &c, 3, 0.0, kmax, np, tol, sigma_mode == 0 ? fl : NULL, I);
    g[0] = G0 + I[0];
    g[3] = Gz + I[1];
    if (rho > 0) { g[1] = (Grho + I[2]) * dx / rho; g[2] = (Grho + I[2]) * dy / rho; }
    else { g[1] = g[2] = 0.0; }
    return st;
}

/* Same quantity by the exact three-layer image series. */
static void reaction_images(const double* d, const double* eps, int l, int lp, const double* r, const double* rp,
                            double* g)
{
    const double D = d[0] - d[1];
    double dx = r[0] - rp[0], dy = r[1] - rp[1];
    double rho2 = dx * dx + dy * dy;
    g[0] = g[1] = g[2] = g[3] = 0.0;
    for (int a = 1; a <= 2; ++a)
        for (int b = 1; b <= 2; ++b) {
            if (!comp_exists(2, l, lp, a, b)) continue;
            double num[3], den0, qq, dh;
            oracle_sigma3_poly(eps, l, lp, a, b, num, &den0, &qq);
            double h = comp_h(d, l, lp, a, b, r[2], rp[2], &dh);
            double nmax = fmax(fabs(num[0]), fmax(fabs(num[1]), fabs(num[2])));
            double gq = 1.0;
            for (int j = 0; j < 200000; ++j) {
                for (int t = 0; t < 3; ++t) {
                    if (num[t] == 0.0) continue;
                    double H = h + (2 * j + t) * D;
                    double R2 = rho2 + H * H, R = sqrt(R2);
                    double c = gq * num[t] / den0;
                    g[0] += c / R;
                    double c3 = c / (R2 * R);
                    g[1] -= c3 * dx;
                    g[2] -= c3 * dy;
                    g[3] -= c3 * H * dh;
                }
                gq *= -qq;
                /* geometric tail below 1e-18 of the largest numerator; a
                 * density that vanishes (equal permittivities) has no terms */
                if (nmax == 0.0 || fabs(gq) / (1.0 - fabs(qq)) < 1e-18) break;
            }
        }
}

/* Potential and field at targets.
 *   n, xyz[n*3], layer[n], q[n]: all charges (sources, and the targets' pool)
 *   nt, targets[nt]: indices of the charges at which Phi, E are wanted
 *   mode: 0 reaction by adaptive quadrature of the spectral-solve density,
 *         1 reaction by the three-layer image series (L == 2 only),
 *         2 reaction by quadrature with the fake density sigma == 1,
 *         3 free-space part only.
 *   phi[nt], field[nt*3] (field may be NULL).
 * Returns 0, -1 on bad input, or -2 when an adaptive quadrature ran out of
 * panels before meeting its tolerance (the affected outputs are NaN). */
int oracle_direct(int L, const double* d, const double* eps, int64_t n, const double* xyz, const int32_t* layer,
                  const double* q, int64_t nt, const int64_t* targets, int mode, double tol, double* phi,
                  double* field, int nthreads)
{
    if (L < 0 || L > OR_MAXL || n < 0 || nt < 0) return -1;
    if (mode == 1 && L != 2) return -1;
    for (int64_t j = 0; j < n; ++j) {
        int l = layer[j];
        double z = xyz[3 * j + 2];
        if (l < 0 || l > L) return -1;
        if (l > 0 && !(z < d[l - 1])) return -1;
        if (l < L && !(z > d[l])) return -1;
    }
    const double inv4pi = 1.0 / (4.0 * OR_PI);
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : failed)
#endif
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t];
        const double* r = &xyz[3 * i];
        int l = layer[i];
        double P = 0.0, Ex = 0.0, Ey = 0.0, Ez = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double* rp = &xyz[3 * j];
            int lp = layer[j];
            if (lp == l && j != i) { /* free-space part, j != i */
                double dx = r[0] - rp[0], dy = r[1] - rp[1], dz = r[2] - rp[2];
                double R2 = dx * dx + dy * dy + dz * dz, R = sqrt(R2);
                P += q[j] / R;
                double c3 = q[j] / (R2 * R);
                Ex += c3 * dx; Ey += c3 * dy; Ez += c3 * dz;
            }
            if (mode == 3 || L == 0) continue;
            double g[4];
            if (mode == 1) reaction_images(d, eps, l, lp, r, rp, g);
            else failed |= reaction_quad(L, d, eps, mode == 2 ? 1 : 0, l, lp, r, rp, tol, g);
            P += q[j] * g[0];
            Ex -= q[j] * g[1]; Ey -= q[j] * g[2]; Ez -= q[j] * g[3];
        }
        phi[t] = P * inv4pi;
        if (field) { field[3 * t] = Ex * inv4pi; field[3 * t + 1] = Ey * inv4pi; field[3 * t + 2] = Ez * inv4pi; }
    }
    return failed ? -2 : 0;
}

/* Reaction Green's function of one pair (4 pi u and 4 pi grad_r u), exposed
 * for the reciprocity / harmonicity / transmission pins. */
int oracle_reaction_pair(int L, const double* d, const double* eps, int l, int lp, const double* r, const double* rp,
                         int mode, double tol, double* g)
{
    if (L == 0) { g[0] = g[1] = g[2] = g[3] = 0; return 0; }
    if (mode == 1) {
        if (L != 2) return -1;
        reaction_images(d, eps, l, lp, r, rp, g);
    } else if (reaction_quad(L, d, eps, mode == 2 ? 1 : 0, l, lp, r, rp, tol, g)) {
        return -2;
    }
    return 0;
}

/* The paper's forward recurrence in m (eq. recurrence) applied to the
 * normalised, scaled integrals S^n I_{n,m}; exposed so that the tests can
 * measure where it is and is not numerically stable.  in: In0[0..2P],
 * In1[0..2P] (In1[0] unused); out: I[(2P+1)*(2P+1)] row-major (n, m). */
void oracle_forward_recurrence(int P, double S, double rho, const double* In0, const double* In1, double* I)
{
    int N2 = 2 * P;
    for (int i = 0; i < (N2 + 1) * (N2 + 1); ++i) I[i] = 0.0;
    for (int n = 0; n <= N2; ++n) I[n * (N2 + 1)] = In0[n];
    for (int n = 1; n <= N2; ++n) I[n * (N2 + 1) + 1] = In1[n];
    for (int m = 1; m < N2; ++m)
        for (int n = m + 1; n <= N2; ++n) {
            double anm = sqrt((double)(n + m) * (n + m + 1.0));
            double anmm = sqrt((double)(n - m) * (n - m + 1.0));
            I[n * (N2 + 1) + m + 1] =
                (2.0 * m / anm) * (S / rho) * I[(n - 1) * (N2 + 1) + m] - (anmm / anm) * I[n * (N2 + 1) + m - 1];
        }
}
