// lfmm_api.cu -- the C ABI of include/lfmm.h: context, medium set-up and the
// build / evaluate entry points.
//
// Medium set-up (Section 3.1 and Appendix A).  For up to three layers the
// reaction densities are rational functions of x = exp(-k D), D = d0 - d1
// the thickness of the middle layer: the spectral interface problem is a
// linear system whose only k-dependence is x.  The host solves it at
// x = 0, 1/2, 1 and fits numerator and denominator (both of degree <= 2) to
// obtain, per component, sigma = num(x)/den(x), its leading behaviour
// C exp(-k zeta) (the lowest power of x) and the remainder
// sigma - C exp(-k zeta) = exp(-k zeta_r) rem(x)/den(x).  Four layers have
// two inner thicknesses and no single x: there the leading term comes from
// the direct path between the source's and the target's interfaces
// (setup_general_density) and the devices solve the interface problem at
// each quadrature node (lf_sigma_solve, lf_sigma_rem in lfmm_internal.cuh).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <cfloat>
#include <new>
#include <thread>
#include <vector>

#include "../../include/lfmm.h"
#include "lfmm_ctx.h"

#define LF_CHECK(call)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return lf_cuda(e_, #call); \
    } while (0)
#define LF_TRY(expr)                \
    do {                            \
        LfErr r_ = (expr);          \
        if (!r_.empty()) return r_; \
    } while (0)

LfErr lf_cuda(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return LfErr();
    return std::string("ECUDA: ") + what + ": " + cudaGetErrorString(e);
}

LfErr lf_reserve(DevBuf& b, size_t bytes)
{
    if (bytes <= b.cap && b.ptr) return LfErr();
    if (b.ptr) {
        cudaFree(b.ptr);
        b.ptr = nullptr;
        b.cap = 0;
    }
    size_t nb = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&b.ptr, nb);
    if (e != cudaSuccess) {
        b.ptr = nullptr;
        cudaGetLastError();
        return std::string("ENOMEM: cudaMalloc of ") + std::to_string(nb) + " bytes failed";
    }
    b.cap = nb;
    return LfErr();
}

static void lf_free(DevBuf& b)
{
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.cap = 0;
}

// ---- profiling ----
int lf_prof_start(lfmm_ctx* ctx, int slot, cudaStream_t st)
{
    if (!ctx->profile) return -1;
    while (ctx->prof_pool.size() < ctx->prof_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        ctx->prof_pool.push_back(e);
    }
    lfmm_ctx::ProfRec r;
    r.slot = slot;
    r.a = ctx->prof_pool[ctx->prof_used++];
    r.b = ctx->prof_pool[ctx->prof_used++];
    cudaEventRecord(r.a, st);
    ctx->prof_recs.push_back(r);
    return (int)ctx->prof_recs.size() - 1;
}

void lf_prof_stop(lfmm_ctx* ctx, int h, cudaStream_t st)
{
    if (h < 0) return;
    cudaEventRecord(ctx->prof_recs[h].b, st);
}

static void prof_reset(lfmm_ctx* ctx)
{
    ctx->prof_recs.clear();
    ctx->prof_used = 0;
}

static void prof_collect(lfmm_ctx* ctx, bool keep_build)
{
    double b = ctx->timings[LFMM_TIME_BUILD];
    for (int i = 0; i < LFMM_TIME_COUNT; ++i) ctx->timings[i] = 0.0;
    if (keep_build) ctx->timings[LFMM_TIME_BUILD] = b;
    for (auto& r : ctx->prof_recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
            ctx->timings[r.slot] += ms;
    }
}

// ---------------------------------------------------------------------------
// Gauss rules by the Golub-Welsch characterisation: the nodes are the
// eigenvalues of the symmetric tridiagonal Jacobi matrix of the weight
// (diagonal a_k, off-diagonal b_k between k-1 and k), found by Sturm-sequence
// bisection; the weights are mu0 / sum_k q_k(t_i)^2 with q_k the orthonormal
// polynomials of the same recurrence (Christoffel numbers).
//   Laguerre (e^{-t} on [0, inf)): a_k = 2k+1, b_k = k,              mu0 = 1
//   Legendre (1 on [-1, 1]):       a_k = 0,    b_k = k/sqrt(4k^2-1), mu0 = 2
// ---------------------------------------------------------------------------
static int sturm_count(int n, const double* a, const double* b, double x)
{
    int cnt = 0;
    double q = a[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < n; ++i) {
        if (q == 0.0) q = 1e-300;
        q = (a[i] - x) - b[i] * b[i] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

static void gauss_from_jacobi(int n, const double* a, const double* b, double mu0, double* t, double* w)
{
    double lo0 = 1e300, hi0 = -1e300;
    for (int i = 0; i < n; ++i) {
        double r = (i > 0 ? fabs(b[i]) : 0.0) + (i + 1 < n ? fabs(b[i + 1]) : 0.0);
        lo0 = std::min(lo0, a[i] - r);
        hi0 = std::max(hi0, a[i] + r);
    }
    for (int i = 0; i < n; ++i) {
        double lo = lo0, up = hi0;
        for (int it = 0; it < 400; ++it) {
            double mid = 0.5 * (lo + up);
            if (mid <= lo || mid >= up) break;
            if (sturm_count(n, a, b, mid) > i) up = mid; else lo = mid;
        }
        double x = 0.5 * (lo + up);
        t[i] = x;
        double q0 = 1.0, q1 = 0.0, ssum = 1.0;
        for (int k = 0; k + 1 < n; ++k) {
            double q2 = ((x - a[k]) * q0 - (k > 0 ? b[k] * q1 : 0.0)) / b[k + 1];
            ssum += q2 * q2;
            q1 = q0;
            q0 = q2;
        }
        w[i] = mu0 / ssum;
    }
}

static int gauss_laguerre(int Q, double* t, double* w)
{
    if (Q < 1 || Q > LFMM_QMAX) return -1;
    std::vector<double> a(Q), b(Q);
    for (int k = 0; k < Q; ++k) {
        a[k] = 2.0 * k + 1.0;
        b[k] = (double)k;
    }
    gauss_from_jacobi(Q, a.data(), b.data(), 1.0, t, w);
    return 0;
}

static int gauss_legendre(int Q, double* t, double* w)
{
    if (Q < 1 || Q > LFMM_QMAX) return -1;
    std::vector<double> a(Q, 0.0), b(Q, 0.0);
    for (int k = 1; k < Q; ++k) b[k] = k / sqrt(4.0 * k * k - 1.0);
    gauss_from_jacobi(Q, a.data(), b.data(), 2.0, t, w);
    return 0;
}

// Quadrature rule for int_0^inf e^{-t} G(t) dt as sum W_i G(T_i).
// Plain: Q-point Gauss-Laguerre.  Composite (a pole of the density just left
// of t = 0): Gauss-Legendre on [0, 1] (W = w e^{-T}) plus Gauss-Laguerre
// shifted to [1, inf) (W = w e^{-1}).
static LfErr make_rule(bool composite, int qleg, int qlag, std::vector<double>& T, std::vector<double>& W)
{
    T.clear();
    W.clear();
    if (composite) {
        std::vector<double> x(qleg), wl(qleg);
        if (gauss_legendre(qleg, x.data(), wl.data())) return "EINVAL: quadrature order out of range";
        for (int i = 0; i < qleg; ++i) {
            double t = 0.5 * (x[i] + 1.0);
            T.push_back(t);
            W.push_back(0.5 * wl[i] * exp(-t));
        }
    }
    std::vector<double> s(qlag), ws(qlag);
    if (gauss_laguerre(qlag, s.data(), ws.data())) return "EINVAL: quadrature order out of range";
    const double t1 = composite ? 1.0 : 0.0;
    for (int i = 0; i < qlag; ++i) {
        T.push_back(t1 + s[i]);
        W.push_back(ws[i] * exp(-t1));
    }
    if ((int)T.size() > LFMM_QMAX) return "EINVAL: quadrature rule too long";
    return LfErr();
}

static LfErr upload_rule(DevBuf& tb, DevBuf& wb, const std::vector<double>& T, const std::vector<double>& W)
{
    LF_TRY(lf_reserve(tb, sizeof(double) * T.size()));
    LF_TRY(lf_reserve(wb, sizeof(double) * W.size()));
    LF_CHECK(cudaMemcpy(tb.ptr, T.data(), sizeof(double) * T.size(), cudaMemcpyHostToDevice));
    LF_CHECK(cudaMemcpy(wb.ptr, W.data(), sizeof(double) * W.size(), cudaMemcpyHostToDevice));
    return LfErr();
}

// Rules of the M2L tables and of the near-field kernel.
static LfErr setup_rules(lfmm_ctx* ctx)
{
    std::vector<double> T, W;
    LF_TRY(make_rule(ctx->near_pole, 32, ctx->near_pole ? 48 : ctx->quad_nodes, T, W));
    LF_TRY(upload_rule(ctx->gl_t_m2l, ctx->gl_w_m2l, T, W));
    ctx->gl_q_m2l = (int)T.size();
    // four or five layers: the remainder mixes more exponential rates, and the field
    // kernels (one more power of k) need 64 nodes for 1e-12 where 32 give 1e-9
    const int qnear = (ctx->L >= 3) ? 64 : (ctx->near_pole ? 48 : 32);
    LF_TRY(make_rule(ctx->near_pole, 32, qnear, T, W));
    LF_TRY(upload_rule(ctx->gl_t_near, ctx->gl_w_near, T, W));
    ctx->gl_q_near = (int)T.size();
    return LfErr();
}

// ---------------------------------------------------------------------------
// Medium: reaction components and their densities.
// ---------------------------------------------------------------------------

// Solve the spectral interface problem (eqs. Laplaceeqlayer, transmissioncond
// in the transformed variable) for L = 2 with x = e^{-k D}; unknowns
// (a0, a1, b1, b2): layer j holds a_j e^{-k(z-d_j)} + b_j e^{-k(d_{j-1}-z)}.
// src_layer / b select the unit source term (b = 1 at the bottom interface
// of the source layer, b = 2 at its top one).  Returns det and solution.
static double solve3(const double* eps, double x, int lp, int b, double sol[4])
{
    double A[4][5];
    memset(A, 0, sizeof(A));
    // interface d0 (layer 0 above, layer 1 below): rows 0 (value) and 1 (eps * slope / k)
    A[0][0] = 1.0;                      // a0 at z = d0
    A[1][0] = -eps[0];
    A[0][1] = -x; A[1][1] = eps[1] * x;  // - a1 e^{-kD} (layer 1 at its top)
    A[0][2] = -1.0; A[1][2] = -eps[1];  // - b1
    // interface d1 (layer 1 above, layer 2 below): rows 2, 3
    A[2][1] = 1.0; A[3][1] = -eps[1];    // a1 at z = d1
    A[2][2] = x; A[3][2] = eps[1] * x;   // b1 e^{-kD}
    A[2][3] = -1.0; A[3][3] = -eps[2];  // - b2
    // source terms: value g and eps * slope: +g below the source, -g above it
    if (b == 1) {  // bottom interface of layer lp
        int j = lp;  // interface index d_lp, the source layer is above it
        A[2 * j][4] -= 1.0;
        A[2 * j + 1][4] -= eps[lp];
    } else {  // top interface d_{lp-1}, the source layer is below it
        int j = lp - 1;
        A[2 * j][4] -= -1.0;
        A[2 * j + 1][4] -= eps[lp];
    }
    // Gaussian elimination with partial pivoting, tracking the determinant
    double det = 1.0;
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c) {
            for (int j = 0; j < 5; ++j) std::swap(A[c][j], A[piv][j]);
            det = -det;
        }
        det *= A[c][c];
        for (int r = c + 1; r < 4; ++r) {
            double f = A[r][c] / A[c][c];
            for (int j = c; j < 5; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int r = 3; r >= 0; --r) {
        double s = A[r][4];
        for (int j = r + 1; j < 4; ++j) s -= A[r][j] * sol[j];
        sol[r] = s / A[r][r];
    }
    return det;
}

// sigma^{ab}_{l lp} for L = 1 (constant): solve the 2x2 problem.
static double sigma_two_layer(const double* eps, int l, int lp, int a, int b)
{
    // unknowns a0 (layer 0), b1 (layer 1); interface d0
    double e0 = eps[0], e1 = eps[1];
    (void)a;
    (void)b;
    if (lp == 0) {  // source above: b = 1
        double a0 = (e0 - e1) / (e0 + e1);
        double b1 = 2.0 * e0 / (e0 + e1);
        return l == 0 ? a0 : b1;
    } else {  // source below: b = 2
        double b1 = (e1 - e0) / (e0 + e1);
        double a0 = 2.0 * e1 / (e0 + e1);
        return l == 1 ? b1 : a0;
    }
}

static void poly_fit3(const double* xs, const double* ys, double* c)
{
    // quadratic through three points (Newton form -> monomial)
    double d1 = (ys[1] - ys[0]) / (xs[1] - xs[0]);
    double d2 = ((ys[2] - ys[1]) / (xs[2] - xs[1]) - d1) / (xs[2] - xs[0]);
    c[2] = d2;
    c[1] = d1 - d2 * (xs[0] + xs[1]);
    c[0] = ys[0] - d1 * xs[0] + d2 * xs[0] * xs[1];
}

// Reflection or transmission coefficient of interface i (layer i above,
// i + 1 below) for a wave arriving from layer u and leaving into layer v: the
// two-layer problem of that interface alone.
static double iface_coef(const double* eps, int i, int u, int v)
{
    const int o = (u == i) ? i + 1 : i;
    if (v == u) return (eps[u] - eps[o]) / (eps[u] + eps[o]);
    return 2.0 * eps[u] / (eps[u] + eps[v]);
}

// Density of a reaction component for three or more interfaces.  The free part
// of the source leaves interface i_s (d_lp for b = 1, d_{lp-1} for b = 2) and
// the reaction term of the target leaves interface i_t (d_l for a = 1,
// d_{l-1} for a = 2).  Every contribution follows a path of reflections and
// transmissions between interfaces, each full crossing of layer j adding
// e^{-k D_j}.  The direct path gives the leading term C e^{-k zeta} with
// zeta = |d_{i_s} - d_{i_t}| and C the product of the single-interface
// coefficients along it; any other path with the same ends crosses some layer
// twice more, so the remainder decays at least like e^{-k (zeta + 2 D_min)}.
// The leading term is checked against the interface problem at large k, and
// the remainder series (lf_sigma_rem) against the solve at moderate k.
static LfErr setup_general_density(const lfmm_ctx* ctx, LfmmComp& c)
{
    const int L = ctx->L;
    const double* d = ctx->d;
    const double* eps = ctx->eps;
    const int is = (c.b == 1) ? c.lp : c.lp - 1;
    const int it = (c.a == 1) ? c.l : c.l - 1;
    double C;
    if (is == it) {
        C = iface_coef(eps, is, c.lp, c.l);
    } else if (it > is) {  // downward
        C = iface_coef(eps, is, c.lp, is + 1);
        for (int i = is + 1; i < it; ++i) C *= iface_coef(eps, i, i, i + 1);
        C *= iface_coef(eps, it, it, c.l);
    } else {  // upward
        C = iface_coef(eps, is, c.lp, is);
        for (int i = is - 1; i > it; --i) C *= iface_coef(eps, i, i + 1, i);
        C *= iface_coef(eps, it, it + 1, c.l);
    }
    double dmin = INFINITY;
    for (int j = 1; j < L; ++j) dmin = std::min(dmin, d[j - 1] - d[j]);
    c.C = C;
    c.zeta = fabs(d[is] - d[it]);
    c.zeta_r = c.zeta + 2.0 * dmin;
    c.has_rem = 1;
    c.D = dmin;
    // coupling steps of the remainder series: D_min (N + 1) >= zeta_r, plus
    // one.  Fewer would let the tail's rounding grow like e^{k zeta_r} at the
    // large nodes, so a medium needing more than the limit is refused.
    const double nsteps = std::ceil(c.zeta_r / dmin) + 1.0;
    if (!(nsteps <= 1024.0)) return "EINVAL: an inner layer is too thin against the layers it sits between";
    c.nterm = (int)nsteps;
    const double k1 = std::min(30.0 / dmin, 600.0 / std::max(c.zeta, 1e-300));
    const double lead = lf_sigma_solve(c, k1) * exp(k1 * c.zeta);
    if (!(fabs(lead - C) <= 1e-8 * (1.0 + fabs(C)))) return "EINVAL: interface problem of the medium is singular";
    // where the subtraction is still harmless the series must reproduce it
    for (double kk : {0.05 / dmin, 0.5 / dmin, 2.0 / dmin}) {
        const double direct = (lf_sigma_solve(c, kk) * exp(kk * c.zeta) - C) * exp(kk * (c.zeta_r - c.zeta));
        const double series = lf_sigma_rem<true>(c, kk);
        if (!(fabs(series - direct) <= 1e-9 * (1.0 + fabs(direct))))
            return "EINVAL: remainder series of the interface problem does not converge";
    }
    return LfErr();
}

// Whether the determinant of the interface problem changes sign for
// k in [-ln(1.5) / D_max, 0]: a pole just left of the integration range, which
// the composite quadrature rule resolves (the same criterion as x <= 1.5 for
// one inner layer).
static bool general_near_pole(const lfmm_ctx* ctx, const LfmmComp& c)
{
    double dmax = 0.0;
    for (int j = 1; j < ctx->L; ++j) dmax = std::max(dmax, ctx->d[j - 1] - ctx->d[j]);
    const double klo = -log(1.5) / dmax;
    double prev = 0.0;
    for (int k = 0; k <= 300; ++k) {
        double det = 0.0;
        lf_sigma_solve(c, klo * (1.0 - k / 300.0), &det);
        if (k > 0 && det * prev <= 0.0) return true;
        prev = det;
    }
    return false;
}

static LfErr setup_components(lfmm_ctx* ctx)
{
    const int L = ctx->L;
    const double* d = ctx->d;
    int nc = 0;
    for (int l = 0; l <= L; ++l) {
        LfmmComp c;
        memset(&c, 0, sizeof(c));
        c.l = l;
        c.lp = l;
        c.is_free = 1;
        c.s = 1.0;
        c.C = 1.0;
        ctx->comp[nc++] = c;
    }
    for (int l = 0; l <= L && L > 0; ++l)
        for (int lp = 0; lp <= L; ++lp)
            for (int a = 1; a <= 2; ++a)
                for (int b = 1; b <= 2; ++b) {
                    if ((a == 1 && l == L) || (a == 2 && l == 0) || (b == 1 && lp == L) || (b == 2 && lp == 0))
                        continue;
                    LfmmComp c;
                    memset(&c, 0, sizeof(c));
                    c.l = l;
                    c.lp = lp;
                    c.a = a;
                    c.b = b;
                    // polarization source (eq. eqpolarizedsource): z'' = s z' + o
                    if (a == 1 && b == 1) { c.s = -1.0; c.o = d[l] + d[lp]; }
                    if (a == 1 && b == 2) { c.s = 1.0; c.o = d[l] - d[lp - 1]; }
                    if (a == 2 && b == 1) { c.s = 1.0; c.o = d[l - 1] - d[lp]; }
                    if (a == 2 && b == 2) { c.s = -1.0; c.o = d[l - 1] + d[lp - 1]; }
                    c.refl = c.s < 0;
                    c.iface = (a == 1) ? d[l] : d[l - 1];
                    c.nif = L;
                    for (int j = 0; j < L; ++j) c.md[j] = d[j];
                    for (int j = 0; j <= L; ++j) c.me[j] = ctx->eps[j];
                    if (L >= 3) {
                        LF_TRY(setup_general_density(ctx, c));
                        if (general_near_pole(ctx, c)) ctx->near_pole = 1;
                    } else if (L == 1) {
                        c.D = 0.0;
                        c.C = sigma_two_layer(ctx->eps, l, lp, a, b);
                        c.zeta = 0.0;
                        c.has_rem = 0;
                        c.den[0] = 1.0;
                    } else {
                        const double D = d[0] - d[1];
                        c.D = D;
                        double xs[3] = {0.0, 0.5, 1.0}, dv[3], nv[3];
                        for (int k = 0; k < 3; ++k) {
                            double sol[4];
                            double det = solve3(ctx->eps, xs[k], lp, b, sol);
                            // a_l -> index l (l = 0, 1), b_l -> index l + 1 (l = 1, 2)
                            double sig = (a == 1) ? sol[l] : sol[l + 1];
                            dv[k] = det;
                            nv[k] = sig * det;
                        }
                        double den[3], num[3];
                        poly_fit3(xs, dv, den);
                        poly_fit3(xs, nv, num);
                        double d0 = den[0];
                        if (fabs(d0) < 1e-300) return "EINVAL: singular interface problem";
                        for (int k = 0; k < 3; ++k) {
                            den[k] /= d0;
                            num[k] /= d0;
                        }
                        double nmax = std::max(fabs(num[0]), std::max(fabs(num[1]), fabs(num[2])));
                        for (int k = 0; k < 3; ++k) {
                            if (fabs(num[k]) < 1e-13 * nmax) num[k] = 0.0;
                            if (fabs(den[k]) < 1e-13) den[k] = 0.0;
                        }
                        int j = 0;
                        while (j < 3 && num[j] == 0.0) ++j;
                        if (j == 3) {  // no coupling at all (cannot happen for eps > 0)
                            c.C = 0.0;
                            c.has_rem = 0;
                        } else {
                            c.C = num[j];
                            c.zeta = j * D;
                            double r[5] = {0, 0, 0, 0, 0};
                            for (int k = 0; k < 3; ++k) r[k] += num[k];
                            for (int k = 0; k < 3; ++k) r[j + k] -= c.C * den[k];
                            double rmax = 0.0;
                            for (int k = 0; k < 5; ++k) rmax = std::max(rmax, fabs(r[k]));
                            for (int k = 0; k < 5; ++k)
                                if (fabs(r[k]) < 1e-13 * std::max(nmax, fabs(c.C)) || k <= j) r[k] = 0.0;
                            int jr = 0;
                            while (jr < 5 && r[jr] == 0.0) ++jr;
                            if (jr == 5) {
                                c.has_rem = 0;
                            } else {
                                c.has_rem = 1;
                                c.zeta_r = jr * D;
                                for (int k = jr; k < 5; ++k) c.rem[k - jr] = r[k];
                            }
                        }
                        for (int k = 0; k < 3; ++k) c.den[k] = den[k];
                        // the remainder's series in x: rem(x)/den(x) = sum a_n x^n, by
                        // exact division (den[0] = 1)
                        {
                            double t[5];
                            for (int k = 0; k < 5; ++k) t[k] = c.has_rem ? c.rem[k] : 0.0;
                            for (int n = 0; n < LFMM_IMG_N; ++n) {
                                const double a = t[0];
                                c.img[n] = a;
                                t[0] = t[1] - a * den[1];
                                t[1] = t[2] - a * den[2];
                                t[2] = t[3];
                                t[3] = t[4];
                                t[4] = 0.0;
                            }
                        }
                        // a real zero of den(x) close to x = 1 (k slightly negative) makes the
                        // remainder nearly singular at k = 0: use the composite rule
                        for (int k = 0; k <= 300; ++k) {
                            double x0 = k * 0.005, x1 = x0 + 0.005;
                            double f0 = den[0] + den[1] * x0 + den[2] * x0 * x0;
                            double f1 = den[0] + den[1] * x1 + den[2] * x1 * x1;
                            if (f0 * f1 <= 0.0) ctx->near_pole = 1;
                        }
                    }
                    ctx->comp[nc++] = c;
                }
    ctx->ncomp = nc;
    return LfErr();
}

// Free-space M2L tables: T_N^mu of the offset (t - s)/h in the rotated half
// plane (rho = |offset_xy|, z = offset_z), for |offset|_inf in [2, TR]: TR = 3
// (classic separation) or 5 (wider separation of high orders, whose finer-level
// pairs reach offsets of 5).
static LfErr setup_tables(lfmm_ctx* ctx)
{
    const int p = ctx->p, TS = 2 * p + 1, TT = TS * TS, nre = lf_nre(p);
    const int TR = ctx->sep_ext ? 5 : 3, TW = 2 * TR + 1;
    std::vector<double> T((size_t)TW * TW * TW * TT, 0.0);
    for (int ox = -TR; ox <= TR; ++ox)
        for (int oy = -TR; oy <= TR; ++oy)
            for (int oz = -TR; oz <= TR; ++oz) {
                int mx = std::max(abs(ox), std::max(abs(oy), abs(oz)));
                if (mx < 2) continue;
                double* t = &T[(size_t)(((ox + TR) * TW + (oy + TR)) * TW + (oz + TR)) * TT];
                double rho = sqrt((double)(ox * ox + oy * oy));
                for (int mu = 0; mu <= 2 * p; ++mu) lf_theta_column(rho, (double)oz, mu, 2 * p, 1.0, t, TS);
            }
    std::vector<float> Tf(T.size());
    for (size_t i = 0; i < T.size(); ++i) Tf[i] = (float)T[i];
    LF_TRY(lf_reserve(ctx->free_T64, T.size() * 8));
    LF_TRY(lf_reserve(ctx->free_T32, T.size() * 4));
    LF_CHECK(cudaMemcpy(ctx->free_T64.ptr, T.data(), T.size() * 8, cudaMemcpyHostToDevice));
    LF_CHECK(cudaMemcpy(ctx->free_T32.ptr, Tf.data(), Tf.size() * 4, cudaMemcpyHostToDevice));
    // child offsets (+-1/4)^3 in parent box units
    std::vector<double> U((size_t)8 * 2 * nre);
    for (int o = 0; o < 8; ++o) {
        double x = (o & 1) ? 0.25 : -0.25, y = (o & 2) ? 0.25 : -0.25, z = (o & 4) ? 0.25 : -0.25;
        lf_regular<double>(p, x, y, z, &U[(size_t)o * 2 * nre], &U[(size_t)o * 2 * nre + nre]);
    }
    std::vector<float> Uf(U.size());
    for (size_t i = 0; i < U.size(); ++i) Uf[i] = (float)U[i];
    LF_TRY(lf_reserve(ctx->oct_U64, U.size() * 8));
    LF_TRY(lf_reserve(ctx->oct_U32, U.size() * 4));
    LF_CHECK(cudaMemcpy(ctx->oct_U64.ptr, U.data(), U.size() * 8, cudaMemcpyHostToDevice));
    LF_CHECK(cudaMemcpy(ctx->oct_U32.ptr, Uf.data(), Uf.size() * 4, cudaMemcpyHostToDevice));
    return LfErr();
}

static lfmm_status status_of(const LfErr& e)
{
    if (e.empty()) return LFMM_OK;
    if (e.compare(0, 6, "EINVAL") == 0) return LFMM_EINVAL;
    if (e.compare(0, 6, "ENOMEM") == 0) return LFMM_ENOMEM;
    if (e.compare(0, 8, "ENUMERIC") == 0) return LFMM_ENUMERIC;
    if (e.compare(0, 5, "ECUDA") == 0) return LFMM_ECUDA;
    return LFMM_ECUDA;
}

static lfmm_status fail(lfmm_ctx* ctx, const LfErr& e)
{
    if (ctx) ctx->err = e;
    return status_of(e);
}

// ---- host-side input checks (no device work for invalid inputs) ----
// Branch-free passes over [0, n) split between a few threads for large n;
// the first offending index is located only when a pass reports one.
template <typename F>
static bool any_bad(int64_t n, F bad_range)
{
    const int64_t chunk = 1 << 18;
    const unsigned hw = std::thread::hardware_concurrency();
    const int nt = (int)std::min<int64_t>(std::min<unsigned>(hw ? hw : 1, 8u), (n + chunk - 1) / chunk);
    if (nt <= 1) return bad_range(0, n);
    std::vector<std::thread> th;
    std::vector<char> res(nt, 0);
    for (int k = 0; k < nt; ++k)
        th.emplace_back([&, k] { res[k] = bad_range(n * k / nt, n * (k + 1) / nt); });
    for (auto& t : th) t.join();
    for (char r : res)
        if (r) return true;
    return false;
}

// layer l spans dd[l + 1] < z < dd[l] with dd[0] = +inf, dd[L + 1] = -inf
static bool points_bad(const lfmm_ctx* ctx, const double* xyz, const int32_t* layer, int64_t b, int64_t e)
{
    double dd[LFMM_MAXL + 2];
    const int L = ctx->L;
    dd[0] = INFINITY;
    for (int k = 0; k < L; ++k) dd[k + 1] = ctx->d[k];
    dd[L + 1] = -INFINITY;
    int bad = 0;
    for (int64_t i = b; i < e; ++i) {
        const int l = layer[i];
        const int lc = l < 0 ? 0 : (l > L ? L : l);
        const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        bad |= (l != lc) | !(z < dd[lc]) | !(z > dd[lc + 1]) | !(fabs(x) <= DBL_MAX) | !(fabs(y) <= DBL_MAX);
    }
    return bad != 0;
}

static bool charges_bad(const double* q, int64_t b, int64_t e)
{
    int bad = 0;
    for (int64_t i = b; i < e; ++i) bad |= !(fabs(q[i]) <= DBL_MAX);
    return bad != 0;
}

int lf_find_comp(const lfmm_ctx* ctx, int l, int lp, int a, int b)
{
    for (int c = 0; c < ctx->ncomp; ++c) {
        const LfmmComp& cp = ctx->comp[c];
        if (!cp.is_free && cp.l == l && cp.lp == lp && cp.a == a && cp.b == b) return c;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
static LfErr auto_near_tables(lfmm_ctx* ctx);  // below, beside the build

extern "C" {

lfmm_status lfmm_gauss_laguerre(int Q, double* nodes, double* weights)
{
    if (!nodes || !weights) return LFMM_EINVAL;
    return gauss_laguerre(Q, nodes, weights) ? LFMM_EINVAL : LFMM_OK;
}

// interfaces finite and strictly decreasing, permittivities finite and positive
static bool medium_ok(const double* d, int L, const double* eps)
{
    if (L < 0 || L > LFMM_MAXL || !eps || (L > 0 && !d)) return false;
    for (int l = 0; l <= L; ++l)
        if (!(eps[l] > 0.0) || !std::isfinite(eps[l])) return false;
    for (int l = 0; l < L; ++l)
        if (!std::isfinite(d[l])) return false;
    for (int l = 1; l < L; ++l)
        if (!(d[l - 1] > d[l])) return false;
    return true;
}

lfmm_status lfmm_medium_components(const double* d, int L, const double* eps, double* out, int max_rows, int* nrows)
{
    if (nrows) *nrows = 0;
    if (!medium_ok(d, L, eps) || (out && max_rows < 0)) return LFMM_EINVAL;
    lfmm_ctx* ctx = new (std::nothrow) lfmm_ctx();
    if (!ctx) return LFMM_ENOMEM;
    ctx->L = L;
    for (int l = 0; l < L; ++l) ctx->d[l] = d[l];
    for (int l = 0; l <= L; ++l) ctx->eps[l] = eps[l];
    const lfmm_status st = status_of(setup_components(ctx));  // host only
    lfmm_status ret = st;
    if (st == LFMM_OK) {
        const int nc = ctx->ncomp;
        if (nrows) *nrows = nc;  // always the full count
        const int w = (out && max_rows >= nc) ? nc : 0;
        if (out && max_rows < nc) ret = LFMM_EINVAL;  // too small: nothing written
        for (int c = 0; c < w; ++c) {
            const LfmmComp& cp = ctx->comp[c];
            const double row[LFMM_MEDIUM_COLS] = {(double)cp.l, (double)cp.lp, (double)cp.a, (double)cp.b,
                                                  (double)cp.is_free, cp.s, cp.o, cp.iface, cp.C, cp.zeta,
                                                  cp.has_rem ? cp.zeta_r : -1.0};
            std::copy(row, row + LFMM_MEDIUM_COLS, out + (size_t)c * LFMM_MEDIUM_COLS);
        }
    }
    delete ctx;
    return ret;
}

lfmm_status lfmm_create(const double* d, int L, const double* eps, int p, lfmm_ctx** out)
{
    if (!out) return LFMM_EINVAL;
    *out = nullptr;
    if (!medium_ok(d, L, eps) || p < 1 || p > LFMM_PMAX) return LFMM_EINVAL;
    lfmm_ctx* ctx = new (std::nothrow) lfmm_ctx();
    if (!ctx) return LFMM_ENOMEM;
    ctx->L = L;
    for (int l = 0; l < L; ++l) ctx->d[l] = d[l];
    for (int l = 0; l <= L; ++l) ctx->eps[l] = eps[l];
    ctx->p = p;
    ctx->sep_ext = (p >= LFMM_SEP_EXT_P) ? 1 : 0;
    LfErr e = setup_components(ctx);
    if (e.empty()) e = lf_cuda(cudaGetDevice(&ctx->device), "cudaGetDevice");
    if (e.empty()) e = lf_cuda(cudaFree(0), "context init");
    // the far field (a chain of dependent per-level launches) is the critical
    // path; the near field runs beside it at lower priority and fills the gaps
    int prio_lo = 0, prio_hi = 0;
    if (e.empty()) e = lf_cuda(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi), "stream priorities");
    if (e.empty())
        e = lf_cuda(cudaStreamCreateWithPriority(&ctx->s_main, cudaStreamNonBlocking, prio_hi), "stream");
    if (e.empty())
        e = lf_cuda(cudaStreamCreateWithPriority(&ctx->s_near, cudaStreamNonBlocking, prio_lo), "stream");
    if (e.empty()) e = lf_cuda(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming), "event");
    if (e.empty()) e = lf_cuda(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming), "event");
    if (e.empty()) e = lf_cuda(cudaEventCreateWithFlags(&ctx->ev_m2r, cudaEventDisableTiming), "event");
    // per-context component array: kernels read it by pointer, so contexts with
    // different media can run side by side (no module-global state)
    if (e.empty()) e = lf_reserve(ctx->comp_dev, sizeof(LfmmComp) * LFMM_MAXCOMP);
    if (e.empty())
        e = lf_cuda(cudaMemcpy(ctx->comp_dev.ptr, ctx->comp, sizeof(LfmmComp) * ctx->ncomp, cudaMemcpyHostToDevice),
                    "components");
    if (e.empty()) e = setup_rules(ctx);
    if (e.empty()) e = setup_tables(ctx);
    if (e.empty()) e = lf_setup_m2l_ops(ctx);
    // the setup tables travel by pageable copies on the legacy stream, which
    // the context's non-blocking streams do not wait for
    if (e.empty()) e = lf_cuda(cudaMallocHost(&ctx->host_pin, LFMM_PIN_BYTES), "pinned host buffer");
    if (e.empty()) e = lf_cuda(cudaDeviceSynchronize(), "setup copies");
    if (!e.empty()) {
        lfmm_status s = status_of(e);
        lfmm_destroy(ctx);
        return s;
    }
    *out = ctx;
    return LFMM_OK;
}

static lfmm_status set_option(lfmm_ctx* ctx, int opt, double v);

lfmm_status lfmm_set_option(lfmm_ctx* ctx, int opt, double v)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    const lfmm_status s = set_option(ctx, opt, v);
    if (s == LFMM_OK) ++ctx->serial;
    return s;
}

static lfmm_status set_option(lfmm_ctx* ctx, int opt, double v)
{
    switch (opt) {
    case LFMM_OPT_PRECISION: {
        if (v != 0.0 && v != 1.0) return fail(ctx, "EINVAL: precision must be 0 or 1");
        if (v == 1.0 && ctx->p > 14) return fail(ctx, "EINVAL: the FP32 form supports p <= 14");
        ctx->precision = (int)v;
        const LfErr e = auto_near_tables(ctx);
        return e.empty() ? LFMM_OK : fail(ctx, e);
    }
    case LFMM_OPT_LEAF_CAP:
        if (!(v >= 1.0 && v <= 100000.0)) return fail(ctx, "EINVAL: leaf capacity out of range");
        ctx->leaf_cap = (int)v;
        return LFMM_OK;
    case LFMM_OPT_PROFILE:
        ctx->profile = (v != 0.0);
        return LFMM_OK;
    case LFMM_OPT_QUAD_NODES: {
        int Q = (int)v;
        if (Q < 16 || Q > LFMM_QMAX || (double)Q != v) return fail(ctx, "EINVAL: quadrature nodes out of range");
        ctx->quad_nodes = Q;
        return fail(ctx, setup_rules(ctx));
    }
    case LFMM_OPT_SURROGATE:
        if (v != 0.0 && !ctx->surr_ready) return fail(ctx, "ESTATE: train the surrogate first"), LFMM_ESTATE;
        ctx->use_surr = (v != 0.0);
        return LFMM_OK;
    case LFMM_OPT_TENSOR_CORES:
        if (v != 0.0 && v != 1.0 && v != 2.0) return fail(ctx, "EINVAL: tensor-core option must be 0, 1 or 2");
        ctx->use_tc = (int)v;
        return LFMM_OK;
    case LFMM_OPT_SERIAL_NEAR:
        if (v != 0.0 && v != 1.0) return fail(ctx, "EINVAL: serial near-field option must be 0 or 1");
        ctx->serial_near = (v != 0.0);
        return LFMM_OK;
    case LFMM_OPT_P2P_STAGED:
        if (v != 0.0 && v != 1.0) return fail(ctx, "EINVAL: staged near-field option must be 0 or 1");
        ctx->p2p_staged = (v != 0.0);
        return LFMM_OK;
    case LFMM_OPT_TC_PERSISTENT:
        if (v != 0.0 && v != 1.0) return fail(ctx, "EINVAL: persistent tensor-core option must be 0 or 1");
        ctx->tc_persistent = (v != 0.0);
        return LFMM_OK;
    case LFMM_OPT_NEAR_TABLES: {
        if (v != 0.0 && v != 1.0 && v != 2.0) return fail(ctx, "EINVAL: near tables option must be 0, 1 or 2");
        if (v == 1.0 && !ctx->near_tab_ready) {
            const LfErr e = lf_near_tables(ctx, nullptr);
            if (!e.empty()) return fail(ctx, e);
        }
        ctx->use_near_tab = (int)v;
        const LfErr e = auto_near_tables(ctx);
        return e.empty() ? LFMM_OK : fail(ctx, e);
    }
    case LFMM_OPT_TC_GROUPS: {
        const int k = (int)v;
        if ((double)k != v || k < 0 || (k > 0 && 189 % k != 0))
            return fail(ctx, "EINVAL: tensor-core groups must divide 189 (or be 0: automatic)");
        ctx->tc_groups = k;
        return LFMM_OK;
    }
    case LFMM_OPT_P2P_SPLIT: {
        const int k = (int)v;
        if ((double)k != v || k < 0 || k > LFMM_P2P_SPLIT_MAX || (k & (k - 1)))
            return fail(ctx, "EINVAL: near-list split must be 0 (automatic) or a power of two <= 16");
        ctx->p2p_split = k;
        return LFMM_OK;
    }
    case LFMM_OPT_SURROGATE_TOL:
        if (!(v > 0.0)) return fail(ctx, "EINVAL: tolerance must be positive");
        ctx->surr_tol = v;
        return LFMM_OK;
    default:
        return fail(ctx, "EINVAL: unknown option");
    }
}

}  // extern "C"

// Automatic near tables (the default): the float32 form takes the pre-computed
// remainder tables once a built tree's near lists hold reaction pairs (their
// deviation from the quadrature, ~2e-8, is far below float32 rounding); the
// tables are built here once per context, outside any evaluation.
static LfErr auto_near_tables(lfmm_ctx* ctx)
{
    if (ctx->use_near_tab != 2 || ctx->precision != 1 || !ctx->built || ctx->near_reaction_entries == 0 ||
        ctx->near_tab_ready)
        return LfErr();
    return lf_near_tables(ctx, nullptr);
}

lfmm_status lf_build_dev(lfmm_ctx* ctx, int64_t n, const double* xyz_dev, const int32_t* layer_dev)
{
    ctx->built = false;
    prof_reset(ctx);
    int ph = lf_prof_start(ctx, LFMM_TIME_BUILD, ctx->s_main);
    LfErr e = lf_build_tree(ctx, xyz_dev, layer_dev, n, ctx->s_main);  // (and the near field's positions)
    lf_prof_stop(ctx, ph, ctx->s_main);
    if (!e.empty()) {
        cudaStreamSynchronize(ctx->s_near);
        cudaStreamSynchronize(ctx->s_main);
        return fail(ctx, e);
    }
    cudaError_t ce = cudaStreamSynchronize(ctx->s_main);
    if (ce != cudaSuccess) return fail(ctx, lf_cuda(ce, "build"));
    if (ctx->profile) prof_collect(ctx, false);
    prof_reset(ctx);
    ctx->built = true;
    ++ctx->serial;
    e = auto_near_tables(ctx);
    if (!e.empty()) return fail(ctx, e);
    return LFMM_OK;
}

extern "C" {

lfmm_status lfmm_build(lfmm_ctx* ctx, int64_t n, const double* xyz, const int32_t* layer)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    if (n < 1 || !xyz || !layer) return fail(ctx, "EINVAL: need n >= 1 and non-null arrays");
    if (any_bad(n, [&](int64_t b, int64_t e) { return points_bad(ctx, xyz, layer, b, e); })) {
        for (int64_t i = 0; i < n; ++i) {
            const int l = layer[i];
            const double z = xyz[3 * i + 2];
            if (l < 0 || l > ctx->L || (l > 0 && !(z < ctx->d[l - 1])) || (l < ctx->L && !(z > ctx->d[l]))) {
                char buf[128];
                snprintf(buf, sizeof buf, "EINVAL: charge %lld has an invalid layer id or lies outside its layer",
                         (long long)i);
                return fail(ctx, buf);
            }
            if (!std::isfinite(xyz[3 * i]) || !std::isfinite(xyz[3 * i + 1]) || !std::isfinite(z))
                return fail(ctx, "EINVAL: non-finite coordinate");
        }
    }
    LfErr e = lf_reserve(ctx->xyz_in, (size_t)n * 24);
    if (e.empty()) e = lf_reserve(ctx->layer_in, (size_t)n * 4);
    if (!e.empty()) return fail(ctx, e);
    cudaError_t ce = cudaMemcpyAsync(ctx->xyz_in.ptr, xyz, (size_t)n * 24, cudaMemcpyHostToDevice, ctx->s_main);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(ctx->layer_in.ptr, layer, (size_t)n * 4, cudaMemcpyHostToDevice, ctx->s_main);
    if (ce != cudaSuccess) return fail(ctx, lf_cuda(ce, "copy inputs"));
    return lf_build_dev(ctx, n, ctx->xyz_in.as<double>(), ctx->layer_in.as<int32_t>());
}

lfmm_status lfmm_build_device(lfmm_ctx* ctx, int64_t n, const double* xyz_dev, const int32_t* layer_dev,
                              void* cuda_stream)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    if (n < 1 || !xyz_dev || !layer_dev) return fail(ctx, "EINVAL: need n >= 1 and non-null arrays");
    cudaStream_t us = (cudaStream_t)cuda_stream;
    cudaError_t ce = cudaEventRecord(ctx->ev_fork, us);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ctx->s_main, ctx->ev_fork, 0);
    if (ce != cudaSuccess) return fail(ctx, lf_cuda(ce, "stream order"));
    return lf_build_dev(ctx, n, xyz_dev, layer_dev);
}

}  // extern "C"

lfmm_status lf_eval_enqueue(lfmm_ctx* ctx, int nrhs, const double* q_dev, double* phi_dev, double* fld_dev)
{
    const int64_t n = ctx->n;
    prof_reset(ctx);
    cudaError_t ce = cudaMemsetAsync(ctx->counts.as<char>() + LFMM_TIMEOUT_OFF, 0, 4, ctx->s_main);
    if (ce != cudaSuccess) return fail(ctx, lf_cuda(ce, "timeout flag"));
    for (int r = 0; r < nrhs; r += LFMM_RHS_BATCH) {
        const int nb = nrhs - r < LFMM_RHS_BATCH ? nrhs - r : LFMM_RHS_BATCH;
        LfErr e = lf_evaluate_sorted(ctx, nb, q_dev + (size_t)r * n, phi_dev + (size_t)r * n,
                                     fld_dev ? fld_dev + (size_t)r * n * 3 : nullptr, ctx->s_main);
        if (!e.empty()) return fail(ctx, e);
    }
    return LFMM_OK;
}

extern "C" {

lfmm_status lfmm_evaluate(lfmm_ctx* ctx, int nrhs, const double* q, double* phi, double* field)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    if (!ctx->built) return fail(ctx, "ESTATE: evaluate before a successful build"), LFMM_ESTATE;
    if (nrhs < 1 || !q || !phi) return fail(ctx, "EINVAL: need nrhs >= 1, q and phi");
    const int64_t n = ctx->n;
    if (any_bad(n * nrhs, [&](int64_t b, int64_t e) { return charges_bad(q, b, e); }))
        return fail(ctx, "ENUMERIC: non-finite charge"), LFMM_ENUMERIC;
    LfErr e = lf_reserve(ctx->q_stage, (size_t)n * nrhs * 8);
    if (e.empty()) e = lf_reserve(ctx->phi_stage, (size_t)n * nrhs * 8);
    if (e.empty() && field) e = lf_reserve(ctx->fld_stage, (size_t)n * nrhs * 24);
    if (!e.empty()) return fail(ctx, e);
    cudaError_t ce = cudaMemcpyAsync(ctx->q_stage.ptr, q, (size_t)n * nrhs * 8, cudaMemcpyHostToDevice, ctx->s_main);
    if (ce != cudaSuccess) return fail(ctx, lf_cuda(ce, "copy charges"));
    lfmm_status s = lf_eval_enqueue(ctx, nrhs, ctx->q_stage.as<double>(), ctx->phi_stage.as<double>(),
                                field ? ctx->fld_stage.as<double>() : nullptr);
    if (s != LFMM_OK) {
        cudaStreamSynchronize(ctx->s_main);
        return s;
    }
    ce = cudaMemcpyAsync(phi, ctx->phi_stage.ptr, (size_t)n * nrhs * 8, cudaMemcpyDeviceToHost, ctx->s_main);
    if (ce == cudaSuccess && field)
        ce = cudaMemcpyAsync(field, ctx->fld_stage.ptr, (size_t)n * nrhs * 24, cudaMemcpyDeviceToHost, ctx->s_main);
    int timeouts = 0;
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(&timeouts, ctx->counts.as<char>() + LFMM_TIMEOUT_OFF, 4, cudaMemcpyDeviceToHost,
                             ctx->s_main);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->s_main);
    if (ce != cudaSuccess) return fail(ctx, lf_cuda(ce, "evaluate"));
    if (timeouts) return fail(ctx, "ETIMEOUT: a device wait of the tensor-core M2L ran out"), LFMM_ETIMEOUT;
    if (ctx->profile) prof_collect(ctx, true);
    return LFMM_OK;
}

lfmm_status lfmm_evaluate_device(lfmm_ctx* ctx, int nrhs, const double* q_dev, double* phi_dev, double* field_dev,
                                 void* cuda_stream)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    if (!ctx->built) return fail(ctx, "ESTATE: evaluate before a successful build"), LFMM_ESTATE;
    if (nrhs < 1 || !q_dev || !phi_dev) return fail(ctx, "EINVAL: need nrhs >= 1, q and phi");
    cudaStream_t us = (cudaStream_t)cuda_stream;
    cudaError_t ce = cudaEventRecord(ctx->ev_fork, us);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ctx->s_main, ctx->ev_fork, 0);
    if (ce != cudaSuccess) return fail(ctx, lf_cuda(ce, "stream order"));
    lfmm_status s = lf_eval_enqueue(ctx, nrhs, q_dev, phi_dev, field_dev);
    if (s != LFMM_OK) return s;
    ce = cudaEventRecord(ctx->ev_join, ctx->s_main);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(us, ctx->ev_join, 0);
    if (ce != cudaSuccess) return fail(ctx, lf_cuda(ce, "stream order"));
    if (ctx->profile) {
        cudaStreamSynchronize(ctx->s_main);
        prof_collect(ctx, true);
    }
    return LFMM_OK;
}

lfmm_status lfmm_near_tables(lfmm_ctx* ctx, double* max_rel_err)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    const LfErr e = lf_near_tables(ctx, max_rel_err);
    return e.empty() ? LFMM_OK : fail(ctx, e);
}

lfmm_status lfmm_check_bounded_wait(lfmm_ctx* ctx, double limit_ms)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    if (!(limit_ms > 0.0 && limit_ms <= 2000.0)) return fail(ctx, "EINVAL: limit_ms must be in (0, 2000]");
    LfErr e = lf_reserve(ctx->counts, 65536);
    int timed_out = 0;
    if (e.empty()) e = lf_wait_probe(ctx, limit_ms, &timed_out);
    if (!e.empty()) return fail(ctx, e);
    if (timed_out) return fail(ctx, "ETIMEOUT: the probe's wait ran out, as designed"), LFMM_ETIMEOUT;
    return LFMM_OK;
}

const char* lfmm_last_error(const lfmm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void lfmm_destroy(lfmm_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->s_main) cudaStreamSynchronize(ctx->s_main);
    if (ctx->s_near) cudaStreamSynchronize(ctx->s_near);
    DevBuf* bufs[] = {&ctx->gl_t_m2l, &ctx->gl_w_m2l, &ctx->gl_t_near, &ctx->gl_w_near, &ctx->free_T64, &ctx->free_T32,
                      &ctx->oct_U64, &ctx->oct_U32, &ctx->comp_dev, &ctx->perm, &ctx->xs, &ctx->ys, &ctx->zs,
                      &ctx->keys, &ctx->keys_tmp, &ctx->vals_tmp, &ctx->scan_tmp, &ctx->hist, &ctx->keys_tmp2, &ctx->vals_tmp2, &ctx->scan_tmp2, &ctx->hist2, &ctx->xyz_in,
                      &ctx->layer_in, &ctx->err_flag, &ctx->counts, &ctx->box_key, &ctx->box_pbeg, &ctx->box_pend,
                      &ctx->box_parent, &ctx->box_cbeg, &ctx->box_cend, &ctx->box_center, &ctx->box_grid, &ctx->pos_rel, &ctx->leaf_of, &ctx->near_tab, &ctx->near_tab4, &ctx->level_consts, &ctx->flags, &ctx->idx,
                      &ctx->near_off, &ctx->near_ent, &ctx->m2l_off, &ctx->m2l_ent, &ctx->m2r_off, &ctx->m2r_ent,
                      &ctx->q_sorted, &ctx->Mexp, &ctx->Lexp, &ctx->phi_far, &ctx->phi_near, &ctx->fld_far,
                      &ctx->fld_near, &ctx->q_stage, &ctx->phi_stage, &ctx->fld_stage, &ctx->m2l_A64, &ctx->m2l_A32,
                      &ctx->m2l_cls, &ctx->m2l_inv, &ctx->m2l_slots, &ctx->m2l_keys, &ctx->m2l_sorted,
                      &ctx->m2l_tiles, &ctx->m2l_levelh, &ctx->m2r_keys, &ctx->m2r_order,
                      &ctx->m2r_tgt, &ctx->m2r_ops, &ctx->m2r_phase, &ctx->m2r_pairs, &ctx->m2r_kstart, &ctx->m2r_kval, &ctx->m2r_tables, &ctx->m2r_levelh, &ctx->m2r_zfrac, &ctx->m2r_zbase,
                      &ctx->m2r_batches, &ctx->m2r_tdesc, &ctx->m2r_ktab, &ctx->surr_theta, &ctx->surr_grad, &ctx->surr_m1,
                      &ctx->surr_m2, &ctx->surr_w, &ctx->surr_b, &ctx->surr_meta, &ctx->surr_err, &ctx->surr_comps,
                      &ctx->surr_xoff, &ctx->surr_counters, &ctx->m2l_Atc, &ctx->m2m_Atc, &ctx->l2l_Atc, &ctx->tc_shift_tiles, &ctx->m2l_tc_tiles, &ctx->tc_mseg, &ctx->m2l_Ms, &ctx->m2m_A64, &ctx->m2m_A32,
                      &ctx->l2l_A64, &ctx->l2l_A32, &ctx->shift_cls, &ctx->m2m_slots, &ctx->shift_tiles};
    for (DevBuf* b : bufs) lf_free(*b);
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_m2r) cudaEventDestroy(ctx->ev_m2r);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->s_main) cudaStreamDestroy(ctx->s_main);
    if (ctx->s_near) cudaStreamDestroy(ctx->s_near);
    if (ctx->host_pin) cudaFreeHost(ctx->host_pin);
    delete ctx;
}

lfmm_status lfmm_get_stats(const lfmm_ctx* ctx, int64_t* out, int nout)
{
    if (!ctx || !out || nout < 1) return LFMM_EINVAL;
    if (ctx->p2p_stats_stale && nout > LFMM_STAT_P2P_FREE) {
        // the pair counts are a statistic, computed from the near lists on request
        lfmm_ctx* mc = const_cast<lfmm_ctx*>(ctx);
        cudaStreamSynchronize(ctx->s_near);
        const LfErr e = lf_p2p_pair_stats(mc);
        if (!e.empty()) return fail(mc, e);
    }
    for (int i = 0; i < nout && i < LFMM_STAT_COUNT; ++i) out[i] = ctx->stats[i];
    if (nout > LFMM_STAT_LAUNCHES) out[LFMM_STAT_LAUNCHES] = ctx->launches;
    if (nout > LFMM_STAT_TIMEOUTS && ctx->counts.ptr) {
        int tmo = 0;
        cudaStreamSynchronize(ctx->s_near);
        if (lf_d2h(&tmo, ctx->counts.as<char>() + LFMM_TIMEOUT_OFF, 4, ctx->s_main) == cudaSuccess)
            out[LFMM_STAT_TIMEOUTS] = tmo;
    }
    if (nout > LFMM_STAT_SURR_QUAD && ctx->surr_counters.ptr) {
        unsigned long long c[2] = {0, 0};
        cudaStreamSynchronize(ctx->s_near);
        if (lf_d2h(c, ctx->surr_counters.ptr, sizeof(c), ctx->s_main) == cudaSuccess) {
            out[LFMM_STAT_SURR_NET] = (int64_t)c[0];
            out[LFMM_STAT_SURR_QUAD] = (int64_t)c[1];
        }
    }
    return ctx->built ? LFMM_OK : LFMM_ESTATE;
}

lfmm_status lfmm_get_timings(const lfmm_ctx* ctx, double* out, int nout)
{
    if (!ctx || !out || nout < 1) return LFMM_EINVAL;
    for (int i = 0; i < nout && i < LFMM_TIME_COUNT; ++i) out[i] = ctx->timings[i];
    return LFMM_OK;
}

lfmm_status lfmm_sommerfeld_tables(lfmm_ctx* ctx, int l, int lp, int a, int b, int npts, const double* rho,
                                   const double* z, double S, int P, double* out)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    int c = lf_find_comp(ctx, l, lp, a, b);
    if (c < 0) return fail(ctx, "EINVAL: no such reaction component");
    if (npts < 1 || !rho || !z || !out || P < 0 || P > LFMM_PMAX || !(S > 0.0))
        return fail(ctx, "EINVAL: bad table request");
    for (int i = 0; i < npts; ++i)
        if (!(z[i] > 0.0) || !(rho[i] >= 0.0)) return fail(ctx, "EINVAL: need z > 0 and rho >= 0");
    const int TS = 2 * P + 1;
    DevBuf drho, dz, dout;
    LfErr e = lf_reserve(drho, (size_t)npts * 8);
    if (e.empty()) e = lf_reserve(dz, (size_t)npts * 8);
    if (e.empty()) e = lf_reserve(dout, (size_t)npts * TS * TS * 8);
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(drho.ptr, rho, (size_t)npts * 8, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dz.ptr, z, (size_t)npts * 8, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_sommerfeld_tables_dev(ctx, c, npts, drho.as<double>(), dz.as<double>(), S, P, dout.as<double>());
    if (e.empty()) e = lf_cuda(cudaStreamSynchronize(ctx->s_main), "tables");
    if (e.empty())
        e = lf_cuda(lf_d2h(out, dout.ptr, (size_t)npts * TS * TS * 8, ctx->s_main), "copy back");
    lf_free(drho);
    lf_free(dz);
    lf_free(dout);
    return fail(ctx, e);
}

lfmm_status lfmm_reaction_kernel(lfmm_ctx* ctx, int l, int lp, int a, int b, int npts, const double* rho,
                                 const double* h, double* out)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    int c = lf_find_comp(ctx, l, lp, a, b);
    if (c < 0) return fail(ctx, "EINVAL: no such reaction component");
    if (npts < 1 || !rho || !h || !out) return fail(ctx, "EINVAL: bad kernel request");
    for (int i = 0; i < npts; ++i)
        if (!(h[i] > 0.0) || !(rho[i] >= 0.0)) return fail(ctx, "EINVAL: need h > 0 and rho >= 0");
    DevBuf drho, dh, dout;
    LfErr e = lf_reserve(drho, (size_t)npts * 8);
    if (e.empty()) e = lf_reserve(dh, (size_t)npts * 8);
    if (e.empty()) e = lf_reserve(dout, (size_t)npts * 24);
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(drho.ptr, rho, (size_t)npts * 8, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dh.ptr, h, (size_t)npts * 8, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_reaction_kernel_dev(ctx, c, npts, drho.as<double>(), dh.as<double>(), dout.as<double>());
    if (e.empty()) e = lf_cuda(cudaStreamSynchronize(ctx->s_main), "kernel");
    if (e.empty()) e = lf_cuda(lf_d2h(out, dout.ptr, (size_t)npts * 24, ctx->s_main), "copy back");
    lf_free(drho);
    lf_free(dh);
    lf_free(dout);
    return fail(ctx, e);
}

lfmm_status lfmm_surrogate_train(lfmm_ctx* ctx, int64_t nsamples, int epochs, uint64_t seed)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    prof_reset(ctx);
    LfErr e = lf_surrogate_train(ctx, nsamples, epochs, seed);
    ++ctx->serial;
    if (!e.empty()) {
        cudaStreamSynchronize(ctx->s_main);
        return fail(ctx, e);
    }
    return LFMM_OK;
}

lfmm_status lfmm_surrogate_info(const lfmm_ctx* ctx, int l, int lp, int a, int b, double* out)
{
    if (!ctx || !out) return LFMM_EINVAL;
    int c = lf_find_comp(ctx, l, lp, a, b);
    if (c < 0) return LFMM_EINVAL;
    for (int q = 0; q < 8; ++q) out[q] = ctx->surr_info[c][q];
    return LFMM_OK;
}

lfmm_status lfmm_surrogate_eval(lfmm_ctx* ctx, int l, int lp, int a, int b, int npts, const double* rho,
                                const double* ht, const double* hs, double* out)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    int c = lf_find_comp(ctx, l, lp, a, b);
    if (c < 0) return fail(ctx, "EINVAL: no such reaction component");
    if (npts < 1 || !rho || !ht || !hs || !out) return fail(ctx, "EINVAL: bad request");
    if (!ctx->surr_ready || !ctx->surr_meta_h[c].trained) return fail(ctx, "ESTATE: surrogate not trained"), LFMM_ESTATE;
    DevBuf dr, dt, ds, dout;
    LfErr e = lf_reserve(dr, (size_t)npts * 8);
    if (e.empty()) e = lf_reserve(dt, (size_t)npts * 8);
    if (e.empty()) e = lf_reserve(ds, (size_t)npts * 8);
    if (e.empty()) e = lf_reserve(dout, (size_t)npts * 32);
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dr.ptr, rho, (size_t)npts * 8, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dt.ptr, ht, (size_t)npts * 8, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(ds.ptr, hs, (size_t)npts * 8, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_surrogate_eval_dev(ctx, c, npts, dr.as<double>(), dt.as<double>(), ds.as<double>(), dout.as<double>());
    if (e.empty()) e = lf_cuda(cudaStreamSynchronize(ctx->s_main), "eval");
    if (e.empty()) e = lf_cuda(lf_d2h(out, dout.ptr, (size_t)npts * 32, ctx->s_main), "copy back");
    lf_free(dr);
    lf_free(dt);
    lf_free(ds);
    lf_free(dout);
    return fail(ctx, e);
}

lfmm_status lfmm_surrogate_get_params(const lfmm_ctx* ctx, int l, int lp, int a, int b, float* theta)
{
    if (!ctx || !theta) return LFMM_EINVAL;
    int c = lf_find_comp(ctx, l, lp, a, b);
    if (c < 0 || !ctx->surr_theta.ptr) return LFMM_EINVAL;
    cudaError_t e = lf_d2h(theta, ctx->surr_theta.as<float>() + (size_t)c * LFMM_SURR_NP, LFMM_SURR_NP * 4, ctx->s_main);
    return e == cudaSuccess ? LFMM_OK : LFMM_ECUDA;
}

lfmm_status lfmm_surrogate_set_params(lfmm_ctx* ctx, int l, int lp, int a, int b, const float* theta)
{
    if (!ctx || !theta) return LFMM_EINVAL;
    ctx->err.clear();
    int c = lf_find_comp(ctx, l, lp, a, b);
    if (c < 0) return fail(ctx, "EINVAL: no such reaction component");
    LfErr e = lf_surrogate_alloc(ctx);
    if (e.empty())
        e = lf_cuda(cudaMemcpyAsync(ctx->surr_theta.as<float>() + (size_t)c * LFMM_SURR_NP, theta, LFMM_SURR_NP * 4, cudaMemcpyHostToDevice, ctx->s_main), "copy params");
    if (e.empty()) e = lf_surrogate_pack(ctx, c);
    if (e.empty()) e = lf_cuda(cudaStreamSynchronize(ctx->s_main), "pack");
    ++ctx->serial;
    return fail(ctx, e);
}

lfmm_status lfmm_surrogate_forward(lfmm_ctx* ctx, int l, int lp, int a, int b, int n, const float* x, float* y)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    int c = lf_find_comp(ctx, l, lp, a, b);
    if (c < 0) return fail(ctx, "EINVAL: no such reaction component");
    if (n < 1 || !x || !y) return fail(ctx, "EINVAL: bad request");
    DevBuf dx, dy;
    LfErr e = lf_reserve(dx, (size_t)n * 16);
    if (e.empty()) e = lf_reserve(dy, (size_t)n * 12);
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dx.ptr, x, (size_t)n * 16, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_surrogate_forward_dev(ctx, c, n, dx.as<float>(), dy.as<float>());
    if (e.empty()) e = lf_cuda(cudaStreamSynchronize(ctx->s_main), "forward");
    if (e.empty()) e = lf_cuda(lf_d2h(y, dy.ptr, (size_t)n * 12, ctx->s_main), "copy back");
    lf_free(dx);
    lf_free(dy);
    return fail(ctx, e);
}

lfmm_status lfmm_surrogate_loss_grad(lfmm_ctx* ctx, int l, int lp, int a, int b, int n, const float* x,
                                     const float* y, double* loss, float* grad)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    int c = lf_find_comp(ctx, l, lp, a, b);
    if (c < 0) return fail(ctx, "EINVAL: no such reaction component");
    if (n < 64 || (n % 64) || !x || !y || !loss || !grad) return fail(ctx, "EINVAL: need n a multiple of 64");
    DevBuf dx, dy;
    LfErr e = lf_surrogate_alloc(ctx);
    if (e.empty()) e = lf_reserve(dx, (size_t)n * 16);
    if (e.empty()) e = lf_reserve(dy, (size_t)n * 12);
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dx.ptr, x, (size_t)n * 16, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dy.ptr, y, (size_t)n * 12, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_surrogate_grad_dev(ctx, c, n, dx.as<float>(), dy.as<float>(), loss, grad);
    lf_free(dx);
    lf_free(dy);
    return fail(ctx, e);
}

}  // extern "C"
