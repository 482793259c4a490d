// lfmm_internal.cuh -- shared definitions of the layered-media FMM library.
//
// Expansion normalisation used on the device (differs from the paper's by a
// diagonal factor; every operator below is the paper's operator conjugated by
// that diagonal):
//   regular solid harmonic    U_n^m(v) = r^n Pbar_n^m(cos t) e^{i m f} / (n+m)!
//   irregular solid harmonic  T_n^m(v) = (n-m)! Pbar_n^m(cos t) e^{i m f} / r^{n+1}
// with Pbar_n^m the associated Legendre function WITHOUT the Condon-Shortley
// phase, and U_n^{-m} = (-1)^m conj(U_n^m) (same for T).  With these,
//   1/|x - y| = sum conj(U_n^m(y)) T_n^m(x)                        (|y| < |x|)
// multipole  M_n^m = sum_j q_j conj(U_n^m(x_j - s))                  (P2M)
// local      Phi(x) = sum L_n^m conj(U_n^m(x - t))                   (L2P)
// M2M        M'_n^m = sum M_k^l conj(U_{n-k}^{m-l}(s - s'))
// M2L        L_k^l  = (-1)^k sum M_n^m T_{n+k}^{m+l}(t - s)
// L2L        L'_j^i = sum L_k^l conj(U_{k-j}^{l-i}(t' - t)).
// The paper's coefficients relate by M^paper_nm = sqrt(4pi/(2n+1))
// sqrt((n-m)!(n+m)!) M_n^m (eq. freespaceexpcoef), likewise for L.
//
// Reaction components (Section 3.3): with the polarization source
// z'' = s z' + o (eq. eqpolarizedsource) the reaction kernel is a function of
// x - x'' that is harmonic on the target side, and the same M2L holds with
//   T_N^mu -> e^{i mu f} K_{N,mu}(rho, dz)                 (a = 1, dz > 0)
//   T_N^mu -> (-1)^{N+mu} e^{i mu f} K_{N,mu}(rho, -dz)    (a = 2, dz < 0)
//   K_{N,mu}(rho, z) = int_0^inf J_mu(k rho) k^N e^{-k z} sigma(k) dk,
// the unnormalised form of eq. uniformintegral; for sigma == 1 it equals T.
// A reflected map (s = -1) multiplies M_n^m by (-1)^{n+m}.
//
// Storage: every expansion is a vector of (p+1)^2 reals, Re(n,m) for
// 0 <= m <= n at n(n+1)/2 + m, then Im(n,m) for 1 <= m <= n at
// NRE + n(n-1)/2 + m - 1, NRE = (p+1)(p+2)/2.  Expansions are scaled by the
// box size S of their level (M/S^n, L S^n, eq. scaledsommerfeldint), so all
// operators act on box-unit vectors.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define LFMM_PMAX 20
#define LFMM_MAXL 4      // interfaces (five layers)
#define LFMM_MAXCOMP 69  // (L + 1) free + (2L)^2 reaction components
#define LFMM_QMAX 128
// A box key holds the layer id above the Morton code of the fine grid: a
// fine level of 10 (30 bits) leaves two bits, four layers; five layers take
// three bits over a fine level of 9 (lf_fine_level).
#define LFMM_FINE_LEVEL 10
__host__ __device__ __forceinline__ int lf_fine_level(int L) { return L >= 4 ? 9 : LFMM_FINE_LEVEL; }
// interaction-list entry: component << LFMM_ENT_SHIFT | box (7 bits of
// component, up to 2^25 boxes)
#define LFMM_ENT_SHIFT 25
#define LFMM_ENT_MASK ((1u << LFMM_ENT_SHIFT) - 1u)
#define LFMM_MAX_DEVICES 64

// Box centre (x, y, z) and layer id (w), 32-byte aligned.
struct __align__(32) LfD4 {
    double x, y, z, w;
};

// Surrogate network of one reaction component: sizes and per-component data.
#define LFMM_SURR_NP 8835   // 4-64-64-64-3 parameters
#define LFMM_SURR_CELLS 32  // error table: cells in log10(rho) and in h
struct LfmmSurrMeta {
    float mu[3], sd[3];  // output standardisation
    float Tt, Ts;        // trained target / source depth ranges
    int trained;
};
struct LfmmSurrView {  // what the near-field kernel needs
    int ready;
    const void* W;       // bf16 weights [ncomp][9728]
    const float* B;      // biases [ncomp][200]
    const float* err;    // [ncomp][CELLS*CELLS]
    const LfmmSurrMeta* meta;
    float tol;
    unsigned long long* counters;  // [2]: pairs by network, pairs by quadrature
};

// One FMM component: free space (a = b = 0) or a reaction component
// (l, lp, a, b).  Plain data, copied to constant memory.
// terms of the remainder's image series a near-field pair may take (far pairs)
#define LFMM_IMG_N 32
// a pair takes images when rho exceeds this many times its remainder depth
#define LFMM_IMG_RATIO 4

struct LfmmComp {
    int l, lp, a, b;
    int is_free;
    int refl;        // 1: the polarization map reflects z
    double s, o;     // z'' = s z' + o
    double iface;    // interface between targets and polarization sources
    // density sigma(k) = num(x) / den(x), x = exp(-D k)
    double D;
    double C, zeta;  // leading behaviour C exp(-k zeta)
    int has_rem;     // remainder sigma - C e^{-k zeta} non-zero
    double zeta_r;   // remainder ~ exp(-k zeta_r)
    double rem[5];   // remainder numerator / x^{zeta_r / D}
    double den[3];   // den[0] = 1
    double img[LFMM_IMG_N];  // series of rem(x) / den(x) in powers of x (the remainder's images)
    // more than two interfaces: sigma(k) has no single x; it is evaluated by
    // solving the interface problem of the medium at each k
    int nif;                         // interfaces of the medium
    int nterm;                       // coupling steps summed for the remainder (nif >= 3)
    double md[LFMM_MAXL];            // interface heights
    double me[LFMM_MAXL + 1];        // permittivities
};

__host__ __device__ __forceinline__ int lf_nre(int p) { return (p + 1) * (p + 2) / 2; }
__host__ __device__ __forceinline__ int lf_nc(int p) { return (p + 1) * (p + 1); }
__host__ __device__ __forceinline__ int lf_re(int n, int m) { return n * (n + 1) / 2 + m; }
__host__ __device__ __forceinline__ int lf_im(int p, int n, int m) { return lf_nre(p) + n * (n - 1) / 2 + m - 1; }
__host__ __device__ __forceinline__ double lf_sgn(int k) { return (k & 1) ? -1.0 : 1.0; }

// Decode packed output index j into (n, m, is_imag).
__host__ __device__ __forceinline__ void lf_decode(int p, int j, int& n, int& m, int& im)
{
    int nre = lf_nre(p);
    if (j < nre) {
        im = 0;
        n = 0;
        while ((n + 1) * (n + 2) / 2 <= j) ++n;
        m = j - n * (n + 1) / 2;
    } else {
        im = 1;
        int r = j - nre;
        n = 1;
        while ((n + 1) * n / 2 <= r) ++n;
        m = r - n * (n - 1) / 2 + 1;
    }
}

// Morton interleave of three 10-bit integers (x in bit 0).
__host__ __device__ __forceinline__ uint32_t lf_spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t lf_compact3(uint32_t v)
{
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030C30C3u;
    v = (v | (v >> 4)) & 0x0300F00Fu;
    v = (v | (v >> 8)) & 0x030000FFu;
    v = (v | (v >> 16)) & 0x000003FFu;
    return v;
}

// Irregular solid harmonics in the x-z half plane (azimuth 0), real:
// out[N*ld + mu] = T_N^mu(rho, 0, z) for 0 <= mu <= N <= nmax, scaled by
// `scale`.  Column recurrence in N (stable upward Legendre recurrence):
//   T_mu^mu   = (2mu-1)!! rho^mu / r^{2mu+1}
//   T_{mu+1}^mu = (2mu+1) z T_mu^mu / r^2
//   T_n^mu    = [(2n-1) z T_{n-1}^mu - (n+mu-1)(n-mu-1) T_{n-2}^mu] / r^2.
// Computes the column mu only (so threads can split columns).
__host__ __device__ __forceinline__ void lf_theta_column(double rho, double z, int mu, int nmax, double scale,
                                                         double* out, int ld)
{
    double r2 = rho * rho + z * z;
    double ir2 = 1.0 / r2;
    double ir = sqrt(ir2);
    double t = scale * ir;  // T_0^0 = 1/r
    for (int m = 1; m <= mu; ++m) t *= (2.0 * m - 1.0) * rho * ir2;
    if (mu > nmax) return;
    out[mu * ld + mu] = t;
    if (mu + 1 > nmax) return;
    double tm1 = t;
    double tn = (2.0 * mu + 1.0) * z * ir2 * t;
    out[(mu + 1) * ld + mu] = tn;
    for (int n = mu + 2; n <= nmax; ++n) {
        double tnew = ((2.0 * n - 1.0) * z * tn - (double)(n + mu - 1) * (double)(n - mu - 1) * tm1) * ir2;
        out[n * ld + mu] = tnew;
        tm1 = tn;
        tn = tnew;
    }
}

// Regular solid harmonics U_n^m(v) for 0 <= m <= n <= p (complex, packed as
// re/im arrays of length NRE).  Recurrences:
//   U_m^m = U_{m-1}^{m-1} (x + i y) / (2m)
//   U_{m+1}^m = z U_m^m
//   U_n^m = [(2n-1) z U_{n-1}^m - r^2 U_{n-2}^m] / (n^2 - m^2).
template <typename R>
__host__ __device__ __forceinline__ void lf_regular(int p, R x, R y, R z, R* ure, R* uim)
{
    R r2 = x * x + y * y + z * z;
    R dre = 1, dim = 0;  // U_m^m
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            R inv = R(1) / R(2 * m);
            R nre = (dre * x - dim * y) * inv;
            R nim = (dre * y + dim * x) * inv;
            dre = nre;
            dim = nim;
        }
        ure[lf_re(m, m)] = dre;
        uim[lf_re(m, m)] = dim;
        if (m + 1 <= p) {
            ure[lf_re(m + 1, m)] = z * dre;
            uim[lf_re(m + 1, m)] = z * dim;
        }
        for (int n = m + 2; n <= p; ++n) {
            R inv = R(1) / R(n * n - m * m);
            R a = R(2 * n - 1) * z;
            ure[lf_re(n, m)] = (a * ure[lf_re(n - 1, m)] - r2 * ure[lf_re(n - 2, m)]) * inv;
            uim[lf_re(n, m)] = (a * uim[lf_re(n - 1, m)] - r2 * uim[lf_re(n - 2, m)]) * inv;
        }
    }
}

// Bessel functions J_0..J_nmax at x >= 0 into out[0..nmax].  For x > nmax
// the upward recurrence from J_0, J_1 is stable; otherwise Miller's
// downward recurrence normalised by J_0 + 2 sum J_{2k} = 1.
__device__ __forceinline__ void lf_bessel_j_set(double x, int nmax, double* out)
{
    if (x == 0.0) {
        out[0] = 1.0;
        for (int m = 1; m <= nmax; ++m) out[m] = 0.0;
        return;
    }
    if (x > (double)nmax) {
        double jm1 = j0(x), jc = j1(x);
        out[0] = jm1;
        if (nmax >= 1) out[1] = jc;
        for (int m = 1; m < nmax; ++m) {
            double jn = (2.0 * m / x) * jc - jm1;
            out[m + 1] = jn;
            jm1 = jc;
            jc = jn;
        }
        return;
    }
    int start = nmax + 24 + (int)x;
    start += (start & 1);
    double jp1 = 0.0, jc = 1e-300, sum = 0.0;
    double ix2 = 2.0 / x;
    for (int m = start; m >= 1; --m) {
        // jc = J_m (unnormalised); J_{m-1} = (2m/x) J_m - J_{m+1}
        double jm1 = m * ix2 * jc - jp1;
        jp1 = jc;
        jc = jm1;  // now J_{m-1}
        if (m - 1 <= nmax) out[m - 1] = jc;
        if (((m - 1) & 1) == 0 && m - 1 > 0) sum += 2.0 * jc;
        if (fabs(jc) > 1e250) {
            const double sc = 1e-250;
            jc *= sc;
            jp1 *= sc;
            sum *= sc;
            for (int k = m - 1; k <= nmax; ++k) out[k] *= sc;
        }
    }
    sum += jc;  // + J_0
    double inv = 1.0 / sum;
    for (int m = 0; m <= nmax; ++m) out[m] *= inv;
}

__host__ __device__ __forceinline__ double lf_poly(const double* c, int n, double x)
{
    double v = 0.0;
    for (int i = n - 1; i >= 0; --i) v = v * x + c[i];
    return v;
}

// The spectral interface problem (Section 3.1, Appendix A) of a medium with
// 3 <= nif <= LFMM_MAXL interfaces at one k.  In layer j the reaction part is
// A_j e^{-k(z - d_j)} (j < L) + B_j e^{-k(d_{j-1} - z)} (j > 0); the free part
// of the source in layer lp is split at its interfaces: b = 1 keeps the part
// that reaches d_lp (value 1 there, slope +k), b = 2 the part that reaches
// d_{lp-1} (value 1, slope -k).  Each interface d_i gives two rows
// (continuity of u and of eps du/dz, divided by k) in the unknowns ordered
// A_0, B_1, A_1, B_2, ..., B_L: A_i (column 2i) and B_{i+1} (column 2i + 1)
// belong to interface i, whose rows couple them with the constant block
//   A0_i = [[1, -1], [-eps_i, -eps_{i+1}]]
// and reach the neighbouring interfaces' unknowns B_i and A_{i+1} through
// x_i = e^{-k D_i} and x_{i+1} (the coupling X).  sigma^{1b} = A_l,
// sigma^{2b} = B_l.
struct LfIfaceProblem {
    int L;
    double x[LFMM_MAXL + 1];  // x[j] = e^{-k D_j} of the inner layers 1 .. L-1
    const double* eps;
};

__host__ __device__ __forceinline__ void lf_iface_setup(const LfmmComp& c, double k, LfIfaceProblem& P)
{
    P.L = c.nif;
    P.eps = c.me;
    for (int j = 0; j <= LFMM_MAXL; ++j) P.x[j] = 0.0;
    for (int j = 1; j < c.nif; ++j) P.x[j] = exp(-k * (c.md[j - 1] - c.md[j]));
}

// v <- T v with T = -A0^{-1} X (one more coupling step between interfaces)
__host__ __device__ __forceinline__ void lf_iface_step(const LfIfaceProblem& P, double* v)
{
    double w[2 * LFMM_MAXL];
    const int L = P.L;
    for (int i = 0; i < L; ++i) {
        const double ea = P.eps[i], eb = P.eps[i + 1];
        double cu = 0.0, fl = 0.0;
        if (i > 0) {  // B_i of interface i - 1
            cu += P.x[i] * v[2 * i - 1];
            fl += ea * P.x[i] * v[2 * i - 1];
        }
        if (i + 1 < L) {  // A_{i+1} of interface i + 1
            cu -= P.x[i + 1] * v[2 * i + 2];
            fl += eb * P.x[i + 1] * v[2 * i + 2];
        }
        // -A0_i^{-1} (cu, fl), A0_i^{-1} = [[eb, -1], [-ea, -1]] / (ea + eb)
        const double s = 1.0 / (ea + eb);
        w[2 * i] = -(eb * cu - fl) * s;
        w[2 * i + 1] = (ea * cu + fl) * s;
    }
    for (int r = 0; r < 2 * L; ++r) v[r] = w[r];
}

// the uncoupled response u0 = A0^{-1} b to the component's source term
__host__ __device__ __forceinline__ void lf_iface_u0(const LfmmComp& c, const LfIfaceProblem& P, double* u0)
{
    for (int r = 0; r < 2 * P.L; ++r) u0[r] = 0.0;
    const int i = (c.b == 1) ? c.lp : c.lp - 1;
    const double ea = P.eps[i], eb = P.eps[i + 1];
    // right-hand side of interface i: b = 1 (source above): (-1, -ea); b = 2 (below): (+1, -eb)
    const double cu = (c.b == 1) ? -1.0 : 1.0, fl = (c.b == 1) ? -ea : -eb;
    const double s = 1.0 / (ea + eb);
    u0[2 * i] = (eb * cu - fl) * s;
    u0[2 * i + 1] = (-ea * cu - fl) * s;
}

// Full solve (dense elimination with partial pivoting, n = 2L <= 6) of the
// interface problem; returns the component's density sigma^{ab}_{l lp}(k)
// and, if asked, the whole solution u and the determinant (whose sign
// locates poles).
__host__ __device__ __forceinline__ double lf_sigma_solve(const LfmmComp& c, double k, double* det = nullptr,
                                                          double* u = nullptr)
{
    const int L = c.nif, n = 2 * L;
    double M[2 * LFMM_MAXL][2 * LFMM_MAXL + 1];
    for (int r = 0; r < n; ++r)
        for (int j = 0; j <= n; ++j) M[r][j] = 0.0;
    for (int i = 0; i < L; ++i) {
        double* cu = M[2 * i];
        double* fl = M[2 * i + 1];
        const double ea = c.me[i], eb = c.me[i + 1];
        // layer i (above) at z = d_i
        cu[2 * i] += 1.0;
        fl[2 * i] -= ea;
        if (i > 0) {
            const double x = exp(-k * (c.md[i - 1] - c.md[i]));
            cu[2 * i - 1] += x;
            fl[2 * i - 1] += ea * x;
        }
        // layer i + 1 (below) at z = d_i, subtracted
        cu[2 * i + 1] -= 1.0;
        fl[2 * i + 1] -= eb;
        if (i + 1 < L) {
            const double x = exp(-k * (c.md[i] - c.md[i + 1]));
            cu[2 * i + 2] -= x;
            fl[2 * i + 2] += eb * x;
        }
        // the source's free part, on the right-hand side
        if (c.b == 1 && i == c.lp) {  // source above d_i
            cu[n] -= 1.0;
            fl[n] -= ea;
        }
        if (c.b == 2 && i + 1 == c.lp) {  // source below d_i
            cu[n] += 1.0;
            fl[n] -= eb;
        }
    }
    double dt = 1.0;
    for (int col = 0; col < n; ++col) {
        int pr = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(M[r][col]) > fabs(M[pr][col])) pr = r;
        if (pr != col) {
            for (int j = 0; j <= n; ++j) {
                const double t = M[col][j];
                M[col][j] = M[pr][j];
                M[pr][j] = t;
            }
            dt = -dt;
        }
        const double pv = M[col][col];
        dt *= pv;
        if (pv == 0.0) {
            if (det) *det = 0.0;
            return 0.0;
        }
        for (int r = col + 1; r < n; ++r) {
            const double f = M[r][col] / pv;
            for (int j = col; j <= n; ++j) M[r][j] -= f * M[col][j];
        }
    }
    if (det) *det = dt;
    double xs[2 * LFMM_MAXL];
    for (int r = n - 1; r >= 0; --r) {
        double v = M[r][n];
        for (int j = r + 1; j < n; ++j) v -= M[r][j] * xs[j];
        xs[r] = v / M[r][r];
    }
    if (u)
        for (int r = 0; r < n; ++r) u[r] = xs[r];
    return (c.a == 1) ? xs[2 * c.l] : xs[2 * c.l - 1];
}

// The remainder of a reaction density in the form every quadrature uses:
//   (sigma(k) - C e^{-k zeta}) e^{k zeta_r},
// bounded for k >= 0.  Up to two interfaces it is rem(x) / den(x) with
// x = e^{-k D}.  Beyond, the solution of (A0 + X) u = b satisfies
// u = u0 + T u (T = -A0^{-1} X, u0 = A0^{-1} b), hence for any N
//   u = sum_{n <= N} T^n u0 + T^{N+1} u.
// T moves a response one interface on and multiplies it by the crossed
// layer's x, so the target entry of T^n u0 vanishes for n < m (m = layers
// between the source's and the target's interface) and equals the direct
// path C e^{-k zeta} for n = m.  The remainder is therefore the sum of the
// terms n = m+1 .. N plus the tail T^{N+1} u: products of small factors, with
// no cancellation against C.  With D_min (N+1) >= zeta_r the tail's rounding
// error stays below e^{-k zeta_r} times machine precision, so the scaled
// remainder keeps full relative accuracy at every k.  The solve and the
// series are compiled only into kernels instantiated with GEN (launched for
// media of four layers), so the kernels of thinner media keep their registers.
template <bool GEN>
__host__ __device__ __forceinline__ double lf_sigma_rem(const LfmmComp& c, double k)
{
    if (!GEN || c.nif <= 2) {
        const double x = exp(-c.D * k);
        return lf_poly(c.rem, 5, x) / lf_poly(c.den, 3, x);
    }
    LfIfaceProblem P;
    lf_iface_setup(c, k, P);
    double u[2 * LFMM_MAXL], v[2 * LFMM_MAXL];
    lf_sigma_solve(c, k, nullptr, u);
    lf_iface_u0(c, P, v);
    const int it = (c.a == 1) ? 2 * c.l : 2 * c.l - 1;  // target entry
    const int is = (c.b == 1) ? c.lp : c.lp - 1, ib = (c.a == 1) ? c.l : c.l - 1;
    const int m = is > ib ? is - ib : ib - is;
    const int N = c.nterm;
    double rem = 0.0;
    for (int n = 1; n <= N; ++n) {
        lf_iface_step(P, v);
        if (n > m) rem += v[it];
    }
    for (int n = 0; n <= N; ++n) lf_iface_step(P, u);
    rem += u[it];
    return rem * exp(k * c.zeta_r);
}

template <bool GEN = false>
__device__ __forceinline__ void lf_sommerfeld_table_block(const LfmmComp& c, double rho_h, double z_h, double S,
                                                          int nmax, double* T, int ld, int Q, const double* gl_t,
                                                          const double* gl_w, double* sJ, double* sA)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int w = nmax + 1;
    for (int mu = tid; mu <= nmax; mu += nt)
        lf_theta_column(rho_h, z_h + c.zeta / S, mu, nmax, c.C, T, ld);
    if (c.has_rem) {
        const double Zh = z_h + c.zeta_r / S;
        const double iZ = 1.0 / Zh;
        for (int q = tid; q < Q; q += nt) {
            double kap = gl_t[q] * iZ;
            // kap is in box units: the density's k is kap / S
            double rt = lf_sigma_rem<GEN>(c, kap / S);
            double a = gl_w[q] * iZ * rt;
            double* Arow = sA + q * w;
            for (int N = 0; N <= nmax; ++N) {
                Arow[N] = a;
                a *= kap;
            }
            lf_bessel_j_set(kap * rho_h, nmax, sJ + q * w);
        }
        __syncthreads();
        const int nent = w * w;
        for (int e = tid; e < nent; e += nt) {
            int N = e / w, mu = e - N * w;
            if (mu > N) continue;
            double s = 0.0;
            for (int q = 0; q < Q; ++q) s += sA[q * w + N] * sJ[q * w + mu];
            T[N * ld + mu] += s;
        }
    }
    __syncthreads();
}

// Near-field reaction kernel of one component (Algorithm 1, local direct
// interactions): (I_00, I_10, I_11') = int (J0, k J0, k J1)(k rho) e^{-kh} sigma dk
// as the closed-form leading image plus the remainder by the quadrature rule
// (gl_t, gl_w) in t = k (h + zeta_r).
template <typename R>
struct LfMath;
template <>
struct LfMath<double> {
    static __device__ __forceinline__ double J0(double x) { return j0(x); }
    static __device__ __forceinline__ double J1(double x) { return j1(x); }
    static __device__ __forceinline__ double Exp(double x) { return exp(x); }
    static __device__ __forceinline__ double Sqrt(double x) { return sqrt(x); }
    static __device__ __forceinline__ double Rsqrt(double x) { return rsqrt(x); }
};
template <>
struct LfMath<float> {
    static __device__ __forceinline__ float J0(float x) { return j0f(x); }
    static __device__ __forceinline__ float J1(float x) { return j1f(x); }
    static __device__ __forceinline__ float Exp(float x) { return expf(x); }
    static __device__ __forceinline__ float Sqrt(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float Rsqrt(float x) { return rsqrtf(x); }
};

template <typename R>
struct LfSum {
    R s = 0, c = 0;
    __device__ __forceinline__ void add(R x)
    {
        R y = x - c;
        R t = s + y;
        c = (t - s) - y;
        s = t;
    }
};
template <>
struct LfSum<double> {
    double s = 0, c = 0;
    __device__ __forceinline__ void add(double x) { s += x; }
};

// Reaction pair kernel: (I_00, I_10, I_11') of one component at (rho, h).
// ---------------------------------------------------------------------------
// Pre-computed remainder tables of the near-field reaction kernels (the
// paper's "pre-computed tables" variant of Section 4, here for the three
// near-field kernels of each reaction component).  With Z = h + zeta_r,
// s = rho / Z and w = zeta_r / Z (in (0, 1]), the scaled remainders
// T00 = Z r00, T10 = Z^2 r10, T11 = Z^2 r11 are smooth functions of (s, w):
// in t = k Z they are integrals of e^{-t} f(x) t^N J_mu(t s) with
// x = exp(-D t w / zeta_r).  They are tabulated on a uniform grid of
// LF_NT_NS x LF_NT_NW points over [0, LF_NT_SMAX] x [0, 1] and read back by
// 4 x 4-point Lagrange interpolation (fourth order); pairs with s beyond the
// table keep the quadrature.
#define LF_NT_NS 257
#define LF_NT_NW 129
#define LF_NT_SMAX 4.0
#define LF_NT_PER (3 * LF_NT_NS * LF_NT_NW)  // doubles per component: [kernel][w][s]

// the three scaled remainders at (s, w) by the quadrature rule in t
template <bool GEN = false>
__device__ __forceinline__ void lf_nt_point(const LfmmComp& c, double s, double w, int Q, const double* gl_t,
                                            const double* gl_w, double out[3])
{
    double a00 = 0.0, a10 = 0.0, a11 = 0.0;
    // t = k Z and w = zeta_r / Z: k = t w / zeta_r
    const double kw = w / c.zeta_r;
    for (int q = 0; q < Q; ++q) {
        const double t = gl_t[q];
        const double f = gl_w[q] * lf_sigma_rem<GEN>(c, t * kw);
        const double j0v = j0(t * s), j1v = j1(t * s);
        a00 += f * j0v;
        a10 += f * t * j0v;
        a11 += f * t * j1v;
    }
    out[0] = a00;
    out[1] = a10;
    out[2] = a11;
}

// weights of the 4-point Lagrange stencil at position x in [0, 3]
template <typename R>
__device__ __forceinline__ void lf_lagrange4(R x, R wgt[4])
{
    const R x1 = x - R(1), x2 = x - R(2), x3 = x - R(3);
    wgt[0] = -x1 * x2 * x3 * R(1.0 / 6.0);
    wgt[1] = x * x2 * x3 * R(0.5);
    wgt[2] = -x * x1 * x3 * R(0.5);
    wgt[3] = x * x1 * x2 * R(1.0 / 6.0);
}

// remainders from the component's table ctab; false where the table does not reach
template <typename R>
__device__ __forceinline__ bool lf_nt_remainder(const double* __restrict__ ctab, const LfmmComp& c, R rho, R h,
                                                R& r00, R& r10, R& r11)
{
    const R Z = h + (R)c.zeta_r;
    const R iZ = R(1) / Z;
    const R fs = rho * iZ * R((LF_NT_NS - 1) / LF_NT_SMAX);
    if (!(fs <= R(LF_NT_NS - 1))) return false;
    const R fw = (R)c.zeta_r * iZ * R(LF_NT_NW - 1);
    int is = (int)fs - 1, iw = (int)fw - 1;
    is = is < 0 ? 0 : (is > LF_NT_NS - 4 ? LF_NT_NS - 4 : is);
    iw = iw < 0 ? 0 : (iw > LF_NT_NW - 4 ? LF_NT_NW - 4 : iw);
    R ws[4], ww[4];
    lf_lagrange4<R>(fs - (R)is, ws);
    lf_lagrange4<R>(fw - (R)iw, ww);
    R acc[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double* tk = ctab + (size_t)k * LF_NT_NS * LF_NT_NW + (size_t)iw * LF_NT_NS + is;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            R row = R(0);
#pragma unroll
            for (int a = 0; a < 4; ++a) row += ws[a] * (R)__ldg(tk + (size_t)b * LF_NT_NS + a);
            acc[k] += ww[b] * row;
        }
    }
    r00 = acc[0] * iZ;
    r10 = acc[1] * iZ * iZ;
    r11 = acc[2] * iZ * iZ;
    return true;
}

// the same from the float32 copy of the table, one float4 {T00, T10, T11, 0}
// per grid point ([w][s]): 16 loads of 16 bytes per pair instead of 48 of 8
template <typename R>
__device__ __forceinline__ bool lf_nt_remainder4(const float4* __restrict__ ctab, const LfmmComp& c, R rho, R h,
                                                 R& r00, R& r10, R& r11)
{
    const R Z = h + (R)c.zeta_r;
    const R iZ = R(1) / Z;
    const R fs = rho * iZ * R((LF_NT_NS - 1) / LF_NT_SMAX);
    if (!(fs <= R(LF_NT_NS - 1))) return false;
    const R fw = (R)c.zeta_r * iZ * R(LF_NT_NW - 1);
    int is = (int)fs - 1, iw = (int)fw - 1;
    is = is < 0 ? 0 : (is > LF_NT_NS - 4 ? LF_NT_NS - 4 : is);
    iw = iw < 0 ? 0 : (iw > LF_NT_NW - 4 ? LF_NT_NW - 4 : iw);
    R ws[4], ww[4];
    lf_lagrange4<R>(fs - (R)is, ws);
    lf_lagrange4<R>(fw - (R)iw, ww);
    R a0 = R(0), a1 = R(0), a2 = R(0);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const float4* row = ctab + (size_t)(iw + b) * LF_NT_NS + is;
        R s0 = R(0), s1 = R(0), s2 = R(0);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const float4 v = __ldg(row + a);
            s0 += ws[a] * (R)v.x;
            s1 += ws[a] * (R)v.y;
            s2 += ws[a] * (R)v.z;
        }
        a0 += ww[b] * s0;
        a1 += ww[b] * s1;
        a2 += ww[b] * s2;
    }
    r00 = a0 * iZ;
    r10 = a1 * iZ * iZ;
    r11 = a2 * iZ * iZ;
    return true;
}

template <typename R, bool GEN = false>
__device__ __forceinline__ void lf_reaction_pair(const LfmmComp& c, R rho, R h, int Q, const double* gl_t,
                                                 const double* gl_w, R& k00, R& k10, R& k11,
                                                 const double* ctab = nullptr, const float4* ctab4 = nullptr)
{
    typedef LfMath<R> F;
    R H = h + (R)c.zeta;
    R r2 = rho * rho + H * H;
    R ir = F::Rsqrt(r2);
    R ir3 = ir * ir * ir;
    R C = (R)c.C;
    k00 = C * ir;
    k10 = C * H * ir3;
    k11 = C * rho * ir3;
    if (!c.has_rem) return;
    if (ctab4) {
        R r00, r10, r11;
        if (lf_nt_remainder4<R>(ctab4, c, rho, h, r00, r10, r11)) {
            k00 += r00;
            k10 += r10;
            k11 += r11;
            return;
        }
    } else if (ctab) {
        R r00, r10, r11;
        if (lf_nt_remainder<R>(ctab, c, rho, h, r00, r10, r11)) {
            k00 += r00;
            k10 += r10;
            k11 += r11;
            return;
        }
    }
    R Z = h + (R)c.zeta_r;
    R D = (R)c.D;
    // Far pairs (rho > LFMM_IMG_RATIO Z) of a rational remainder rem(x)/den(x),
    // x = e^{-k D}: its series sum a_n x^n splits off M + 1 terms, each an
    // image at depth Z + n D integrated in closed form, and leaves
    // x^{M+1} t(x)/den(x) (t by exact division, t <- (t - a_n den)/x), whose
    // quadrature sees the depth Z + (M + 1) D: the Gauss-Laguerre rule in k Z
    // cannot follow J0(k rho) once rho is many times Z.
    R t[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) t[i] = (R)c.rem[i];
    if ((!GEN || c.nif <= 2) && D > R(0) && rho > (R)LFMM_IMG_RATIO * Z) {
        int M = (int)ceil((double)((rho * (R)(1.0 / LFMM_IMG_RATIO) - Z) / D)) - 1;
        M = M < 0 ? 0 : (M > LFMM_IMG_N - 1 ? LFMM_IMG_N - 1 : M);
        for (int n = 0; n <= M; ++n) {
            const R a = (R)c.img[n];
            const R Hn = Z + (R)n * D;
            const R rr = F::Rsqrt(rho * rho + Hn * Hn);
            const R rr3 = rr * rr * rr;
            k00 += a * rr;
            k10 += a * Hn * rr3;
            k11 += a * rho * rr3;
            // t <- (t - a den) / x (t[0] - a den[0] = 0 by the choice of a)
            t[0] = t[1] - a * (R)c.den[1];
            t[1] = t[2] - a * (R)c.den[2];
            t[2] = t[3];
            t[3] = t[4];
            t[4] = R(0);
        }
        Z += (R)(M + 1) * D;
    }
    R iZ = R(1) / Z;
    for (int q = 0; q < Q; ++q) {
        R kap = (R)gl_t[q] * iZ;
        R w;
        if (!GEN || c.nif <= 2) {
            R x = F::Exp(-D * kap);
            R num = t[4];
            for (int i = 3; i >= 0; --i) num = num * x + t[i];
            R den = ((R)c.den[2] * x + (R)c.den[1]) * x + (R)c.den[0];
            R rt = num / den;
            w = (R)gl_w[q] * iZ * rt;
        } else {
            // the solved remainder carries rounding noise times e^{k (zeta_r - zeta)},
            // which only the node weight (~e^{-t}) brings back to size: form the
            // product in double before narrowing
            w = (R)(gl_w[q] * (double)iZ * lf_sigma_rem<true>(c, (double)kap));
        }
        R a = kap * rho;
        R j0v = F::J0(a), j1v = F::J1(a);
        k00 += w * j0v;
        k10 += w * kap * j0v;
        k11 += w * kap * j1v;
    }
}

// ---------------------------------------------------------------------------
// Host-side declarations shared between translation units.
// ---------------------------------------------------------------------------
struct LfmmDeviceLevel {
    int nbox;     // boxes of this level (all layers)
    int off;      // first global box id
    double h;     // box size
};
