// lfmm_fmm.cu -- far-field kernels of the layered-media FMM (Algorithm 1:
// upward pass, downward pass, evaluation of the local expansions) and the
// driver of one evaluation.
//
// Every component targeting layer l adds into ONE local-expansion tree of
// that layer: the free-space M2L of eq. metole and the reaction M2L of eqs.
// metoleimage1 / coefintable (built from the Sommerfeld tables of
// lfmm_sommerfeld_table_block) both land in the same L; L2L (eq. letole) and
// L2P are then done once per layer instead of once per component.  This is
// the sum of Algorithm 2 moved before the (linear) downward pass.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

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

static inline int lf_blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }


template <typename R>
struct LfAcc {  // compensated (Kahan) sum in single precision, plain sum in double
    R s = 0, c = 0;
    __device__ __forceinline__ void add(R x)
    {
        R y = x - c;
        R t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ R get() const { return s; }
};
template <>
struct LfAcc<double> {
    double s = 0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double get() const { return s; }
};

// ---------------------------------------------------------------------------
// Regular solid harmonics U_k^j(x, y, z), column by column (j = 0..p, then
// k = j..p), by the recurrences of the diagonal U_j^j = (x + iy) U_{j-1}^{j-1} / (2j),
// U_{j+1}^j = z U_j^j and (k^2 - j^2) U_k^j = (2k - 1) z U_{k-1}^j - r^2 U_{k-2}^j,
// handing each value to f(k, j, re, im) as it is formed: no array is needed.
// ---------------------------------------------------------------------------
template <typename R, typename F>
__device__ __forceinline__ void lf_regular_walk(int p, R x, R y, R z, F&& f)
{
    const R r2 = x * x + y * y + z * z;
    R dre = 1, dim = 0;
    for (int j = 0; j <= p; ++j) {
        if (j > 0) {
            const R inv = R(1) / R(2 * j);
            const R nre = (dre * x - dim * y) * inv;
            const R nim = (dre * y + dim * x) * inv;
            dre = nre;
            dim = nim;
        }
        f(j, j, dre, dim);
        R p1re = dre, p1im = dim, p2re = 0, p2im = 0;
        for (int k = j + 1; k <= p; ++k) {
            R ure, uim;
            if (k == j + 1) {
                ure = z * p1re;
                uim = z * p1im;
            } else {
                const R inv = R(1) / R(k * k - j * j);
                const R a = R(2 * k - 1) * z;
                ure = (a * p1re - r2 * p2re) * inv;
                uim = (a * p1im - r2 * p2im) * inv;
            }
            p2re = p1re;
            p2im = p1im;
            p1re = ure;
            p1im = uim;
            f(k, j, ure, uim);
        }
    }
}

// ---------------------------------------------------------------------------
// P2M (eq. mefreespace / melayerupgoingimage): M_n^m = sum_j q_j conj(U_n^m((x_j - s)/h)).
// One thread per charge (sorted order, so the charges of a leaf are
// consecutive): each coefficient is summed over the lanes of one leaf by a
// segmented shuffle reduction and added by the leaf's first lane of the warp
// into the (zeroed) multipoles.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(128) k_p2m(int64_t n, int p, const int* __restrict__ leaf_of,
                                             const LfD4* __restrict__ cen, const double* __restrict__ xs,
                                             const double* __restrict__ ys, const double* __restrict__ zs,
                                             const R* __restrict__ q, double ih, R* __restrict__ M, int nrhs,
                                             int64_t qstride, size_t mstride)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < n;
    const int b = valid ? leaf_of[i] : -1 - lane;  // a lane past the end is a segment of its own
    // same[k]: lane + 2^k holds a charge of the same leaf (segments are contiguous)
    unsigned same = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int d = 1 << k;
        const int bd = __shfl_down_sync(0xffffffffu, b, d);
        if (lane + d < 32 && bd == b) same |= 1u << k;
    }
    const int bprev = __shfl_up_sync(0xffffffffu, b, 1);  // every lane takes part
    const bool head = valid && (lane == 0 || bprev != b);
    R x = 0, y = 0, z = 0;
    if (valid) {
        const LfD4 c = cen[b];  // ih = 1 / h of the leaf level, divided once on the host
        x = (R)((xs[i] - c.x) * ih);
        y = (R)((ys[i] - c.y) * ih);
        z = (R)((zs[i] - c.z) * ih);
    }
    const int nc = lf_nc(p);
    for (int r = 0; r < nrhs; ++r) {
        const R qv = valid ? q[(size_t)r * qstride + i] : R(0);
        R* Mb = M + (size_t)r * mstride + (size_t)(valid ? b : 0) * nc;
        lf_regular_walk<R>(p, x, y, z, [&](int k, int j, R ure, R uim) {
            R vre = qv * ure, vim = -qv * uim;  // q conj(U)
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const R wre = __shfl_down_sync(0xffffffffu, vre, 1 << s);
                const R wim = __shfl_down_sync(0xffffffffu, vim, 1 << s);
                if (same & (1u << s)) {
                    vre += wre;
                    vim += wim;
                }
            }
            if (head) {
                atomicAdd(Mb + lf_re(k, j), vre);
                if (j > 0) atomicAdd(Mb + lf_im(p, k, j), vim);
            }
        });
    }
}

// Complex helpers for packed coefficient arrays (m may be negative).
template <typename R>
__device__ __forceinline__ void lf_get(const R* v, int p, int n, int m, R& re, R& im)
{
    if (m >= 0) {
        re = v[lf_re(n, m)];
        im = (m > 0) ? v[lf_im(p, n, m)] : R(0);
    } else {
        int a = -m;
        R s = (a & 1) ? R(-1) : R(1);
        re = s * v[lf_re(n, a)];
        im = -s * v[lf_im(p, n, a)];
    }
}
// regular harmonics stored as separate re/im arrays of length NRE
template <typename R>
__device__ __forceinline__ void lf_getU(const R* ure, const R* uim, int n, int m, R& re, R& im)
{
    if (m >= 0) {
        re = ure[lf_re(n, m)];
        im = uim[lf_re(n, m)];
    } else {
        int a = -m;
        R s = (a & 1) ? R(-1) : R(1);
        re = s * ure[lf_re(n, a)];
        im = -s * uim[lf_re(n, a)];
    }
}

__device__ __forceinline__ int lf_octant(LfD4 child, LfD4 parent)
{
    return (child.x > parent.x ? 1 : 0) | (child.y > parent.y ? 2 : 0) | (child.z > parent.z ? 4 : 0);
}

// ---------------------------------------------------------------------------
// M2M (eq. metome): M_p(n,m) = sum_{k,l} 2^{-k} M_c(k,l) conj(U_{n-k}^{m-l}(d)),
// d = (child - parent)/h_parent in {+-1/4}^3.  One block per parent box.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_m2m(int off, int p, const LfD4* __restrict__ cen, const int* __restrict__ cbeg,
                      const int* __restrict__ cend, const R* __restrict__ octU, R* __restrict__ M)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nre = lf_nre(p), nc = lf_nc(p);
    R* sM = reinterpret_cast<R*>(smem_raw);
    R* sUr = sM + nc;
    R* sUi = sUr + nre;
    const int b = off + blockIdx.x;
    const int tid = threadIdx.x;
    int n = 0, m = 0, im = 0;
    const bool act = tid < nre;
    if (act) lf_decode(p, tid, n, m, im);
    R ar = 0, ai = 0;
    const LfD4 pc = cen[b];
    for (int ch = cbeg[b]; ch < cend[b]; ++ch) {
        int o = lf_octant(cen[ch], pc);
        for (int j = tid; j < nc; j += blockDim.x) sM[j] = M[(size_t)ch * nc + j];
        for (int j = tid; j < nre; j += blockDim.x) {
            sUr[j] = octU[(size_t)o * 2 * nre + j];
            sUi[j] = octU[(size_t)o * 2 * nre + nre + j];
        }
        __syncthreads();
        if (act) {
            R sc = 1;
            for (int k = 0; k <= n; ++k) {
                for (int l = -k; l <= k; ++l) {
                    int dm = m - l;
                    if (dm > n - k || dm < -(n - k)) continue;
                    R mr, mi, ur, ui;
                    lf_get(sM, p, k, l, mr, mi);
                    lf_getU(sUr, sUi, n - k, dm, ur, ui);
                    // M * conj(U)
                    ar += sc * (mr * ur + mi * ui);
                    ai += sc * (mi * ur - mr * ui);
                }
                sc *= R(0.5);
            }
        }
        __syncthreads();
    }
    if (act) {
        M[(size_t)b * nc + lf_re(n, m)] = ar;
        if (m > 0) M[(size_t)b * nc + lf_im(p, n, m)] = ai;
    }
}

// ---------------------------------------------------------------------------
// L2L (eq. letole): L_c(j,i) = sum_{k>=j,l} 2^{-j} L_p(k,l) conj(U_{k-j}^{l-i}(d)).
// One block per child box; adds into L of the child (which holds its M2L).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_l2l(int off, int p, const LfD4* __restrict__ cen, const int* __restrict__ parent,
                      const R* __restrict__ octU, R* __restrict__ L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nre = lf_nre(p), nc = lf_nc(p);
    R* sL = reinterpret_cast<R*>(smem_raw);
    R* sUr = sL + nc;
    R* sUi = sUr + nre;
    const int b = off + blockIdx.x;
    const int tid = threadIdx.x;
    const int pb = parent[b];
    const int o = lf_octant(cen[b], cen[pb]);
    for (int j = tid; j < nc; j += blockDim.x) sL[j] = L[(size_t)pb * nc + j];
    for (int j = tid; j < nre; j += blockDim.x) {
        sUr[j] = octU[(size_t)o * 2 * nre + j];
        sUi[j] = octU[(size_t)o * 2 * nre + nre + j];
    }
    __syncthreads();
    if (tid >= nre) return;
    int jn, im_, mm;
    lf_decode(p, tid, jn, mm, im_);
    R ar = 0, ai = 0;
    for (int k = jn; k <= p; ++k) {
        for (int l = -k; l <= k; ++l) {
            int dm = l - mm;
            if (dm > k - jn || dm < -(k - jn)) continue;
            R lr, li, ur, ui;
            lf_get(sL, p, k, l, lr, li);
            lf_getU(sUr, sUi, k - jn, dm, ur, ui);
            ar += lr * ur + li * ui;
            ai += li * ur - lr * ui;
        }
    }
    R sc = 1;
    for (int q = 0; q < jn; ++q) sc *= R(0.5);
    L[(size_t)b * nc + lf_re(jn, mm)] += sc * ar;
    if (mm > 0) L[(size_t)b * nc + lf_im(p, jn, mm)] += sc * ai;
}

// ---------------------------------------------------------------------------
// M2L for one level, all components, one block per target box.
// Output j of the packed layout is owned by thread j.  Per entry (c, s):
//   v = (t - P_c(s)) / h, (rho, phi) its horizontal polar coordinates;
//   M' = M_s e^{i m phi} (times (-1)^{n+m} for a reflecting map);
//   T  = real table in the phi = 0 half plane: free space T_N^mu(v) from the
//        per-offset table, reaction components from the Sommerfeld routine;
//   L'_k^l = sum_{n,m} M'_n^m T_{n+k}^{m+l},  L_k^l += (-1)^k e^{i l phi} L'_k^l / h.
// ---------------------------------------------------------------------------
struct M2LArgs {
    int p;
    int level_off;
    double h;
    const LfD4* cen;
    const int* mbeg;
    const int* mend;
    const uint32_t* ment;
    const void* M;
    void* L;
    const LfmmComp* comps;  // the context's components
    const void* freeT;  // [(2 tr + 1)^3][TS*TS] in R, offsets in [-tr, tr]^3
    int tr;
    const double* gl_t;
    const double* gl_w;
    int Q;
};

// GEN: reaction components of media of four or five layers
template <typename R, bool REACT, bool GEN = false>
__global__ void k_m2l(M2LArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = a.p, nre = lf_nre(p), nc = lf_nc(p), TS = 2 * p + 1, TT = TS * TS;
    const int nq = REACT ? a.Q : 0;
    double* sTd = reinterpret_cast<double*>(smem_raw);  // TT (reaction only)
    double* sJ = sTd + (REACT ? TT : 0);                 // Q*TS
    double* sA = sJ + nq * TS;                           // Q*TS
    R* sT = reinterpret_cast<R*>(sA + nq * TS);          // TT
    R* sM = sT + TT;                                     // nc
    R* sOut = sM + nc;                                   // nc
    R* sC = sOut + nc;                                   // p+1 (cos m phi)
    R* sS = sC + (p + 1);                                // p+1 (sin m phi)

    const R* M = reinterpret_cast<const R*>(a.M);
    R* L = reinterpret_cast<R*>(a.L);
    const R* freeT = reinterpret_cast<const R*>(a.freeT);

    const int t = a.level_off + blockIdx.x;
    const int tid = threadIdx.x;
    const bool act = tid < nc;
    int k = 0, l = 0, isim = 0;
    if (act) lf_decode(p, tid, k, l, isim);
    const LfD4 ct = a.cen[t];
    LfAcc<R> acc;
    const double ih = 1.0 / a.h;

    for (int e = a.mbeg[t]; e < a.mend[t]; ++e) {
        const uint32_t ent = a.ment[e];
        const int c = (int)(ent >> LFMM_ENT_SHIFT);
        const int s = (int)(ent & LFMM_ENT_MASK);
        const LfmmComp cp = a.comps[c];
        const LfD4 cs = a.cen[s];
        const double psz = cp.is_free ? cs.z : cp.s * cs.z + cp.o;
        const double vx = (ct.x - cs.x) * ih, vy = (ct.y - cs.y) * ih, vz = (ct.z - psz) * ih;
        const double rho = sqrt(vx * vx + vy * vy);
        const double phi = (rho > 0.0) ? atan2(vy, vx) : 0.0;
        if (tid <= p) {
            double sn, cs_;
            sincos(tid * phi, &sn, &cs_);
            sC[tid] = (R)cs_;
            sS[tid] = (R)sn;
        }
        if (!REACT) {
            int ox = (int)lrint(vx), oy = (int)lrint(vy), oz = (int)lrint(vz);
            const int tw = 2 * a.tr + 1;
            const R* src = freeT + (size_t)(((ox + a.tr) * tw + (oy + a.tr)) * tw + (oz + a.tr)) * TT;
            for (int j = tid; j < TT; j += blockDim.x) sT[j] = src[j];
        } else {
            const double zz = (cp.a == 1) ? vz : -vz;  // > 0 for valid entries
            lf_sommerfeld_table_block<GEN>(cp, rho, zz, a.h, 2 * p, sTd, TS, a.Q, a.gl_t, a.gl_w, sJ, sA);
            for (int j = tid; j < TT; j += blockDim.x) {
                int N = j / TS, mu = j - N * TS;
                double v = (mu <= N) ? sTd[j] : 0.0;
                if (cp.a == 2 && ((N + mu) & 1)) v = -v;
                sT[j] = (R)v;
            }
        }
        __syncthreads();
        // rotated (and for reflections sign-flipped) multipole of the source
        const R* Ms = M + (size_t)s * nc;
        for (int j = tid; j < nre; j += blockDim.x) {
            int n, m, dummy;
            lf_decode(p, j, n, m, dummy);
            R mr = Ms[j];
            R mi = (m > 0) ? Ms[lf_im(p, n, m)] : R(0);
            R cr = sC[m], sr = sS[m];
            R rr = mr * cr - mi * sr, ri = mr * sr + mi * cr;
            if (cp.refl && ((n + m) & 1)) {
                rr = -rr;
                ri = -ri;
            }
            sM[j] = rr;
            if (m > 0) sM[lf_im(p, n, m)] = ri;
        }
        __syncthreads();
        if (act) {
            R sum = 0;
            for (int n = 0; n <= p; ++n) {
                const R* Trow = sT + (n + k) * TS;
                const int b0 = lf_re(n, 0);
                const int bi = lf_im(p, n, 1) - 1;  // Im(n,m) at bi + m
                if (!isim) sum += sM[b0] * Trow[l];
                for (int m = 1; m <= n; ++m) {
                    R mv = isim ? sM[bi + m] : sM[b0 + m];
                    sum += mv * Trow[m + l];
                    int mu = l - m;
                    R tv = Trow[mu >= 0 ? mu : -mu];
                    // (-1)^m from M_n^{-m}, (-1)^mu from T_N^{-mu}, -1 for the imaginary part
                    int par = m + ((mu < 0) ? -mu : 0) + isim;
                    sum += (par & 1) ? -mv * tv : mv * tv;
                }
            }
            sOut[tid] = sum;
        }
        __syncthreads();
        if (act) {
            R re = sOut[lf_re(k, l)];
            R im = (l > 0) ? sOut[lf_im(p, k, l)] : R(0);
            R cr = sC[l], sr = sS[l];
            R v = isim ? (sr * re + cr * im) : (cr * re - sr * im);
            acc.add((k & 1) ? -v : v);
        }
        __syncthreads();
    }
    if (act) L[(size_t)t * nc + tid] += acc.get() * (R)ih;
}

// ---------------------------------------------------------------------------
// L2P with gradient: Phi = sum L_k^l conj(U_k^l((x - t)/h)),
// dz Phi = sum L_k^l conj(U_{k-1}^l), (dx + i dy) Phi = sum L_k^l conj(U_{k-1}^{l-1}).
// One thread per charge.  Every harmonic U_k^j is paired, as the recurrence
// forms it, with the coefficients it multiplies: L_k^j (potential), L_{k+1}^j
// (dz), L_{k+1}^{j+1} and L_{k+1}^{j-1} (dx, dy); the local expansion of the
// charge's leaf is read through the cache (the lanes of a warp share a few
// leaves).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(128) k_l2p(int64_t n, int p, const int* __restrict__ leaf_of,
                                             const LfD4* __restrict__ cen, const double* __restrict__ xs,
                                             const double* __restrict__ ys, const double* __restrict__ zs, double ih,
                                             const R* __restrict__ L, double* __restrict__ phi,
                                             double* __restrict__ fld, int nrhs, size_t lstride, int64_t ostride)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = leaf_of[i];
    const LfD4 c = cen[b];  // ih = 1 / h of the leaf level, divided once on the host
    const R x = (R)((xs[i] - c.x) * ih), y = (R)((ys[i] - c.y) * ih), z = (R)((zs[i] - c.z) * ih);
    const int nc = lf_nc(p);
    for (int r = 0; r < nrhs; ++r) {
        const R* Lb = L + (size_t)r * lstride + (size_t)b * nc;
        LfAcc<R> P, Gz, Gx, Gy;
        lf_regular_walk<R>(p, x, y, z, [&](int k, int j, R ur, R ui) {
            if (j == 0)
                P.add(__ldg(Lb + lf_re(k, 0)) * ur);
            else
                P.add(R(2) * (__ldg(Lb + lf_re(k, j)) * ur + __ldg(Lb + lf_im(p, k, j)) * ui));
            if (k + 1 > p) return;
            if (j == 0)
                Gz.add(__ldg(Lb + lf_re(k + 1, 0)) * ur);
            else
                Gz.add(R(2) * (__ldg(Lb + lf_re(k + 1, j)) * ur + __ldg(Lb + lf_im(p, k + 1, j)) * ui));
            // L_{k+1}^{j+1} conj(U_k^j)
            R lr = __ldg(Lb + lf_re(k + 1, j + 1)), li = __ldg(Lb + lf_im(p, k + 1, j + 1));
            Gx.add(lr * ur + li * ui);
            Gy.add(li * ur - lr * ui);
            if (j >= 1) {
                // -conj(L_{k+1}^{j-1}) U_k^j (L_{k+1}^0 is real)
                lr = __ldg(Lb + lf_re(k + 1, j - 1));
                li = (j > 1) ? __ldg(Lb + lf_im(p, k + 1, j - 1)) : R(0);
                Gx.add(-(lr * ur + li * ui));
                Gy.add(-(lr * ui - li * ur));
            }
        });
        const size_t o = (size_t)r * ostride + i;
        phi[o] = (double)P.get();
        fld[3 * o + 0] = -(double)Gx.get() * ih;
        fld[3 * o + 1] = -(double)Gy.get() * ih;
        fld[3 * o + 2] = -(double)Gz.get() * ih;
    }
}

// ---------------------------------------------------------------------------
// Charges in sorted order, and the final combination in caller order.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_gather_q(const double* __restrict__ q, const int32_t* __restrict__ perm, int64_t n,
                           R* __restrict__ qs)
{
    // blockIdx.y: right-hand side (vectors of n, caller order in, sorted order out)
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t r = blockIdx.y;
    if (i < n) qs[r * n + i] = (R)q[r * n + perm[i]];
}

__global__ void k_combine(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ pf,
                          const double* __restrict__ pn, const double* __restrict__ ff,
                          const double* __restrict__ fn, double* __restrict__ phi, double* __restrict__ fld)
{
    // blockIdx.y: right-hand side; all arrays are vectors of n per right-hand side
    int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 >= n) return;
    const int64_t r = blockIdx.y;
    const double s = 0.079577471545947667884;  // 1 / (4 pi)
    const int64_t i = r * n + i0, j = r * n + perm[i0];
    phi[j] = (pf[i] + pn[i]) * s;
    if (fld) {
        fld[3 * j + 0] = (ff[3 * i + 0] + fn[3 * i + 0]) * s;
        fld[3 * j + 1] = (ff[3 * i + 1] + fn[3 * i + 1]) * s;
        fld[3 * j + 2] = (ff[3 * i + 2] + fn[3 * i + 2]) * s;
    }
}

// ---------------------------------------------------------------------------
// Driver.
// ---------------------------------------------------------------------------
template <typename R>
static size_t m2l_smem(int p, int Q, bool react)
{
    int TS = 2 * p + 1, TT = TS * TS, nc = lf_nc(p);
    size_t d = react ? (size_t)TT + 2 * (size_t)Q * TS : 0;
    return sizeof(double) * d + sizeof(R) * (TT + 2 * nc + 2 * (p + 1)) + 64;
}

template <typename R>
static LfErr far_field(lfmm_ctx* ctx, cudaStream_t st)
{
    const int p = ctx->p, nc = lf_nc(p), nre = lf_nre(p);
    const int depth = ctx->depth;
    const LfmmLevel& leaf = ctx->levels[depth];
    R* M = ctx->Mexp.as<R>();
    R* L = ctx->Lexp.as<R>();
    const int nr = ctx->nrhs_b;  // right-hand sides of this pass: expansions [nr][boxes][nc]
    const size_t ms = (size_t)ctx->nbox_total * nc;
    const LfD4* cen = ctx->box_center.as<LfD4>();
    const int* pbeg = ctx->box_pbeg.as<int>();
    const int* pend = ctx->box_pend.as<int>();
    const int* cbeg = ctx->box_cbeg.as<int>();
    const int* cend = ctx->box_cend.as<int>();
    const int* par = ctx->box_parent.as<int>();
    const R* octU = reinterpret_cast<const R*>(sizeof(R) == 8 ? ctx->oct_U64.ptr : ctx->oct_U32.ptr);
    const R* freeT = reinterpret_cast<const R*>(sizeof(R) == 8 ? ctx->free_T64.ptr : ctx->free_T32.ptr);

    // levels below lmin take part in no M2L: no multipoles are needed there and
    // their locals stay zero, so M2M stops and L2L starts at lmin
    int lmin = depth;
    for (int l = 0; l <= depth; ++l)
        if (ctx->levels[l].m2l_count + ctx->levels[l].m2r_count > 0) {
            lmin = l;
            break;
        }
    // upward pass
    int ph = lf_prof_start(ctx, LFMM_TIME_P2M, st);
    {
        // the leaf multipoles are sums of atomic contributions: zero them first
        LF_CHECK(cudaMemset2DAsync(M + (size_t)leaf.off * nc, ms * sizeof(R), 0, sizeof(R) * (size_t)leaf.nbox * nc,
                                   nr, st));
        ++ctx->launches, k_p2m<R><<<lf_blocks(ctx->n, 128), 128, 0, st>>>(
            ctx->n, p, ctx->leaf_of.as<int>(), cen, ctx->xs.as<double>(), ctx->ys.as<double>(),
            ctx->zs.as<double>(), ctx->q_sorted.as<R>(), 1.0 / leaf.h, M, nr, ctx->n, ms);
        LF_TRY(lf_cuda(cudaGetLastError(), "p2m"));
    }
    lf_prof_stop(ctx, ph, st);
    {
        size_t sm = sizeof(R) * (nc + 2 * (size_t)nre);
        int th = ((nre + 31) / 32) * 32;
        for (int l = depth - 1; l >= lmin; --l) {
            const LfmmLevel& lv = ctx->levels[l];
            if (lv.nbox == 0) continue;
            ph = lf_prof_start(ctx, LFMM_TIME_M2M, st);
            if (ctx->shift_ready)
                LF_TRY(lf_shift_gemm(ctx, l, false, st));
            else
                for (int r = 0; r < nr; ++r)
                    ++ctx->launches, k_m2m<R><<<lv.nbox, th, sm, st>>>(lv.off, p, cen, cbeg, cend, octU, M + r * ms);
            lf_prof_stop(ctx, ph, st);
        }
        LF_TRY(lf_cuda(cudaGetLastError(), "m2m"));
    }
    // downward pass: all M2L into zeroed L, then L2L top-down (child += shifted parent)
    const int Q = ctx->gl_q_m2l;
    const size_t msm_f = m2l_smem<R>(p, Q, false), msm_r = m2l_smem<R>(p, Q, true);
    LF_CHECK(cudaFuncSetAttribute(k_m2l<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm_f));
    LF_CHECK(cudaFuncSetAttribute(k_m2l<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm_r));
    const bool general = ctx->L >= 3;
    if (general)
        LF_CHECK(cudaFuncSetAttribute(k_m2l<R, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm_r));
    const int mth = ((nc + 31) / 32) * 32;
    const size_t lsm = sizeof(R) * (nc + 2 * (size_t)nre);
    const int lth = ((nre + 31) / 32) * 32;
    LF_CHECK(cudaMemsetAsync(L, 0, sizeof(R) * ms * nr, st));
    const bool gemm = ctx->m2l_ntiles > 0;
    if (gemm) {
        ph = lf_prof_start(ctx, LFMM_TIME_M2L_FREE, st);
        if (sizeof(R) == 4 && lf_tc_on(ctx) && ctx->m2l_tc_ntiles > 0)
            LF_TRY(lf_m2l_tc(ctx, st));
        else
            LF_TRY(lf_m2l_gemm(ctx, st));
        lf_prof_stop(ctx, ph, st);
    }
    if (ctx->m2r_wait) {
        LF_CHECK(cudaStreamWaitEvent(st, ctx->ev_m2r, 0));
        ctx->m2r_wait = 0;
    }
    if (ctx->m2r_nbatch > 0) {
        ph = lf_prof_start(ctx, LFMM_TIME_M2L_REACTION, st);
        LF_TRY(lf_m2r_apply(ctx, st));
        lf_prof_stop(ctx, ph, st);
    }
    for (int l = 0; l <= depth; ++l) {
        const LfmmLevel& lv = ctx->levels[l];
        if (lv.nbox == 0) continue;
        M2LArgs a;
        a.p = p;
        a.level_off = lv.off;
        a.h = lv.h;
        a.cen = cen;
        a.M = M;
        a.L = L;
        a.freeT = freeT;
        a.comps = ctx->comp_dev.as<LfmmComp>();
        a.tr = ctx->sep_ext ? 5 : 3;
        a.gl_t = ctx->gl_t_m2l.as<double>();
        a.gl_w = ctx->gl_w_m2l.as<double>();
        a.Q = Q;
        if (!gemm && lv.m2l_count > 0) {
            a.mbeg = ctx->m2l_off.as<int>();
            a.mend = ctx->m2l_off.as<int>() + ctx->nbox_total;
            a.ment = ctx->m2l_ent.as<uint32_t>();
            ph = lf_prof_start(ctx, LFMM_TIME_M2L_FREE, st);
            for (int r = 0; r < nr; ++r) {
                a.M = M + r * ms;
                a.L = L + r * ms;
                ++ctx->launches, k_m2l<R, false><<<lv.nbox, mth, msm_f, st>>>(a);
            }
            lf_prof_stop(ctx, ph, st);
        }
        if (lv.m2r_count > 0 && l < ctx->m2r_keyed_from) {
            a.mbeg = ctx->m2r_off.as<int>();
            a.mend = ctx->m2r_off.as<int>() + ctx->nbox_total;
            a.ment = ctx->m2r_ent.as<uint32_t>();
            ph = lf_prof_start(ctx, LFMM_TIME_M2L_REACTION, st);
            for (int r = 0; r < nr; ++r) {
                a.M = M + r * ms;
                a.L = L + r * ms;
                if (general)
                    ++ctx->launches, k_m2l<R, true, true><<<lv.nbox, mth, msm_r, st>>>(a);
                else
                    ++ctx->launches, k_m2l<R, true><<<lv.nbox, mth, msm_r, st>>>(a);
            }
            lf_prof_stop(ctx, ph, st);
        }
        LF_TRY(lf_cuda(cudaGetLastError(), "m2l"));
    }
    for (int l = lmin + 1; l <= depth; ++l) {
        const LfmmLevel& lv = ctx->levels[l];
        if (lv.nbox == 0) continue;
        ph = lf_prof_start(ctx, LFMM_TIME_L2L, st);
        if (ctx->shift_ready)
            LF_TRY(lf_shift_gemm(ctx, l, true, st));
        else
            for (int r = 0; r < nr; ++r)
                ++ctx->launches, k_l2l<R><<<lv.nbox, lth, lsm, st>>>(lv.off, p, cen, par, octU, L + r * ms);
        lf_prof_stop(ctx, ph, st);
        LF_TRY(lf_cuda(cudaGetLastError(), "l2l"));
    }
    ph = lf_prof_start(ctx, LFMM_TIME_L2P, st);
    {
        ++ctx->launches, k_l2p<R><<<lf_blocks(ctx->n, 128), 128, 0, st>>>(
            ctx->n, p, ctx->leaf_of.as<int>(), cen, ctx->xs.as<double>(), ctx->ys.as<double>(),
            ctx->zs.as<double>(), 1.0 / leaf.h, L, ctx->phi_far.as<double>(), ctx->fld_far.as<double>(), nr, ms,
            ctx->n);
        LF_TRY(lf_cuda(cudaGetLastError(), "l2p"));
    }
    lf_prof_stop(ctx, ph, st);
    return LfErr();
}

LfErr lf_evaluate_sorted(lfmm_ctx* ctx, int nrhs, const double* q_dev, double* phi_dev, double* field_dev,
                         cudaStream_t st)
{
    // one pass over nrhs charge vectors on the same tree: [nrhs][n] in, [nrhs][n] (and [nrhs][n][3]) out
    const int64_t n = ctx->n;
    const int nc = lf_nc(ctx->p);
    const size_t rs = ctx->precision ? sizeof(float) : sizeof(double);
    const size_t nr = (size_t)nrhs;
    ctx->nrhs_b = nrhs;
    LF_TRY(lf_reserve(ctx->q_sorted, (size_t)n * rs * nr));
    LF_TRY(lf_reserve(ctx->Mexp, (size_t)ctx->nbox_total * nc * rs * nr));
    LF_TRY(lf_reserve(ctx->Lexp, (size_t)ctx->nbox_total * nc * rs * nr));
    LF_TRY(lf_reserve(ctx->phi_far, (size_t)n * 8 * nr));
    LF_TRY(lf_reserve(ctx->phi_near, (size_t)n * 8 * nr));
    LF_TRY(lf_reserve(ctx->fld_far, (size_t)n * 24 * nr));
    LF_TRY(lf_reserve(ctx->fld_near, (size_t)n * 24 * nr));
    const int ptot = lf_prof_start(ctx, LFMM_TIME_TOTAL, st);
    const dim3 g1(lf_blocks(n, 256), (unsigned)nrhs);
    if (ctx->precision)
        ++ctx->launches, k_gather_q<float><<<g1, 256, 0, st>>>(q_dev, ctx->perm.as<int32_t>(), n, ctx->q_sorted.as<float>());
    else
        ++ctx->launches, k_gather_q<double><<<g1, 256, 0, st>>>(q_dev, ctx->perm.as<int32_t>(), n,
                                                               ctx->q_sorted.as<double>());
    LF_TRY(lf_cuda(cudaGetLastError(), "gather q"));
    // the reaction M2L's tables and operators of a fresh build: on the
    // near-field stream ahead of the near field, beside the far field's
    // upward pass; the far field waits for them before the reaction M2L
    const bool m2r_dev = ctx->m2r_dev_pending != 0;
    if (ctx->serial_near) {
        if (m2r_dev) LF_TRY(lf_m2r_device(ctx, st));
        // near field alone on the calling stream, before the far field (its
        // stage time is then the near-field kernels' own duration)
        LF_TRY(lf_near_field(ctx, st));
        if (ctx->precision)
            LF_TRY(far_field<float>(ctx, st));
        else
            LF_TRY(far_field<double>(ctx, st));
    } else {
        // near field on its own stream, concurrent with the far field
        LF_CHECK(cudaEventRecord(ctx->ev_fork, st));
        LF_CHECK(cudaStreamWaitEvent(ctx->s_near, ctx->ev_fork, 0));
        if (m2r_dev) {
            LF_TRY(lf_m2r_device(ctx, ctx->s_near));
            LF_CHECK(cudaEventRecord(ctx->ev_m2r, ctx->s_near));
            ctx->m2r_wait = 1;
        }
        LF_TRY(lf_near_field(ctx, ctx->s_near));
        LF_CHECK(cudaEventRecord(ctx->ev_join, ctx->s_near));
        if (ctx->precision)
            LF_TRY(far_field<float>(ctx, st));
        else
            LF_TRY(far_field<double>(ctx, st));
        LF_CHECK(cudaStreamWaitEvent(st, ctx->ev_join, 0));
    }
    ++ctx->launches, k_combine<<<g1, 256, 0, st>>>(n, ctx->perm.as<int32_t>(), ctx->phi_far.as<double>(),
                                                    ctx->phi_near.as<double>(), ctx->fld_far.as<double>(),
                                                    ctx->fld_near.as<double>(), phi_dev, field_dev);
    LF_TRY(lf_cuda(cudaGetLastError(), "combine"));
    lf_prof_stop(ctx, ptot, st);
    return LfErr();
}
