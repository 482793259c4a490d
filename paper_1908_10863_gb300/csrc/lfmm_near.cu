// lfmm_near.cu -- near-field interactions of the layered-media FMM.
//
// Free space (eq. freereactioncomponents): Phi += q / |r_i - r_j|, j != i.
// Reaction components (Algorithm 1, "Local Direct Interactions"): with the
// polarization source z'' = s z_j + o and h = |z_i - z''| the pair kernel is
//   I_00 = int J0(k rho) e^{-k h} sigma(k) dk,
// and the field needs I_10 = int k J0 e^{-kh} sigma, I_11' = int k J1 e^{-kh} sigma.
// Each is the closed form of the leading exponential C e^{-k zeta} of sigma
// (C/R, C H/R^3, C rho/R^3 with H = h + zeta) plus the remainder by
// Gauss-Laguerre quadrature in t = k (h + zeta_r).
// One block per leaf target box; sources of each near box are staged in
// shared memory relative to the target box centre.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

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

__constant__ LfmmComp c_ncomp[LFMM_MAXCOMP];
__constant__ double c_gl_t[LFMM_QMAX];
__constant__ double c_gl_w[LFMM_QMAX];

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
template <typename R>
__device__ __forceinline__ void lf_reaction_pair(const LfmmComp& c, R rho, R h, int Q, R& k00, R& k10, R& k11)
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
    R Z = h + (R)c.zeta_r;
    R iZ = R(1) / Z;
    R D = (R)c.D;
    for (int q = 0; q < Q; ++q) {
        R kap = (R)c_gl_t[q] * iZ;
        R x = F::Exp(-D * kap);
        R num = (R)c.rem[4];
        for (int i = 3; i >= 0; --i) num = num * x + (R)c.rem[i];
        R den = ((R)c.den[2] * x + (R)c.den[1]) * x + (R)c.den[0];
        R w = (R)c_gl_w[q] * iZ * num / den;
        R a = kap * rho;
        R j0v = F::J0(a), j1v = F::J1(a);
        k00 += w * j0v;
        k10 += w * kap * j0v;
        k11 += w * kap * j1v;
    }
}

struct P2PArgs {
    int leaf_off;
    const LfD4* cen;
    const int* pbeg;
    const int* pend;
    const int* nbeg;
    const int* nend;
    const uint32_t* nent;
    const double* xs;
    const double* ys;
    const double* zs;
    const void* q;
    double* phi;
    double* fld;
    int Qn;
};

#define P2P_T 128

template <typename R>
__global__ void __launch_bounds__(P2P_T) k_p2p(P2PArgs a)
{
    typedef LfMath<R> F;
    __shared__ R sx[P2P_T], sy[P2P_T], sz[P2P_T], sq[P2P_T];
    const R* q = reinterpret_cast<const R*>(a.q);
    const int t = a.leaf_off + blockIdx.x;
    const int tid = threadIdx.x;
    const LfD4 ct = a.cen[t];
    const int tb = a.pbeg[t], te = a.pend[t];
    for (int base = tb; base < te; base += P2P_T) {
        const int i = base + tid;
        const bool valid = i < te;
        R xi = 0, yi = 0, zi = 0;
        if (valid) {
            xi = (R)(a.xs[i] - ct.x);
            yi = (R)(a.ys[i] - ct.y);
            zi = (R)(a.zs[i] - ct.z);
        }
        LfSum<R> P, Ex, Ey, Ez;
        for (int e = a.nbeg[t]; e < a.nend[t]; ++e) {
            const uint32_t ent = a.nent[e];
            const int c = (int)(ent >> LFMM_ENT_SHIFT);
            const int s = (int)(ent & LFMM_ENT_MASK);
            const LfmmComp& cp = c_ncomp[c];
            const int sb = a.pbeg[s], se = a.pend[s];
            for (int cb = sb; cb < se; cb += P2P_T) {
                const int j = cb + tid;
                __syncthreads();
                if (j < se) {
                    sx[tid] = (R)(a.xs[j] - ct.x);
                    sy[tid] = (R)(a.ys[j] - ct.y);
                    double zj = cp.is_free ? a.zs[j] : cp.s * a.zs[j] + cp.o;
                    sz[tid] = (R)(zj - ct.z);
                    sq[tid] = q[j];
                }
                __syncthreads();
                if (!valid) continue;
                const int cnt = min(P2P_T, se - cb);
                if (cp.is_free) {
                    for (int u = 0; u < cnt; ++u) {
                        R dx = xi - sx[u], dy = yi - sy[u], dz = zi - sz[u];
                        R r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 > R(0)) {
                            R ir = F::Rsqrt(r2);
                            R qi = sq[u] * ir;
                            R q3 = qi * ir * ir;
                            P.add(qi);
                            Ex.add(q3 * dx);
                            Ey.add(q3 * dy);
                            Ez.add(q3 * dz);
                        }
                    }
                } else {
                    for (int u = 0; u < cnt; ++u) {
                        R dx = xi - sx[u], dy = yi - sy[u];
                        R dz = zi - sz[u];
                        R h = (cp.a == 1) ? dz : -dz;
                        R rho = F::Sqrt(dx * dx + dy * dy);
                        R k00, k10, k11;
                        lf_reaction_pair<R>(cp, rho, h, a.Qn, k00, k10, k11);
                        R qs = sq[u];
                        P.add(qs * k00);
                        Ez.add((cp.a == 1) ? qs * k10 : -qs * k10);
                        if (rho > R(0)) {
                            R g = qs * k11 / rho;
                            Ex.add(g * dx);
                            Ey.add(g * dy);
                        }
                    }
                }
            }
        }
        if (valid) {
            a.phi[i] = (double)P.s;
            a.fld[3 * (size_t)i + 0] = (double)Ex.s;
            a.fld[3 * (size_t)i + 1] = (double)Ey.s;
            a.fld[3 * (size_t)i + 2] = (double)Ez.s;
        }
    }
}

static LfErr upload_consts(lfmm_ctx* ctx, cudaStream_t st)
{
    LF_CHECK(cudaMemcpyToSymbolAsync(c_ncomp, ctx->comp, sizeof(LfmmComp) * ctx->ncomp, 0, cudaMemcpyHostToDevice, st));
    LF_CHECK(cudaMemcpyToSymbolAsync(c_gl_t, ctx->gl_t_near.ptr, sizeof(double) * ctx->gl_q_near, 0,
                                     cudaMemcpyDeviceToDevice, st));
    LF_CHECK(cudaMemcpyToSymbolAsync(c_gl_w, ctx->gl_w_near.ptr, sizeof(double) * ctx->gl_q_near, 0,
                                     cudaMemcpyDeviceToDevice, st));
    return LfErr();
}

LfErr lf_near_field(lfmm_ctx* ctx, cudaStream_t st)
{
    LF_TRY(upload_consts(ctx, st));
    const LfmmLevel& leaf = ctx->levels[ctx->depth];
    P2PArgs a;
    a.leaf_off = leaf.off;
    a.cen = ctx->box_center.as<LfD4>();
    a.pbeg = ctx->box_pbeg.as<int>();
    a.pend = ctx->box_pend.as<int>();
    a.nbeg = ctx->near_off.as<int>();
    a.nend = ctx->near_off.as<int>() + ctx->nbox_total;
    a.nent = ctx->near_ent.as<uint32_t>();
    a.xs = ctx->xs.as<double>();
    a.ys = ctx->ys.as<double>();
    a.zs = ctx->zs.as<double>();
    a.q = ctx->q_sorted.ptr;
    a.phi = ctx->phi_near.as<double>();
    a.fld = ctx->fld_near.as<double>();
    a.Qn = ctx->gl_q_near;
    const int ph = lf_prof_start(ctx, LFMM_TIME_P2P, st);
    if (ctx->precision)
        ++ctx->launches, k_p2p<float><<<leaf.nbox, P2P_T, 0, st>>>(a);
    else
        ++ctx->launches, k_p2p<double><<<leaf.nbox, P2P_T, 0, st>>>(a);
    LF_TRY(lf_cuda(cudaGetLastError(), "p2p"));
    lf_prof_stop(ctx, ph, st);
    return LfErr();
}

// ---------------------------------------------------------------------------
// Parity entry points: the same device routines on caller-given geometries.
// ---------------------------------------------------------------------------
__global__ void k_som_tables(LfmmComp c, int npts, const double* __restrict__ rho, const double* __restrict__ z,
                             double S, int P, const double* __restrict__ gt, const double* __restrict__ gw, int Q,
                             double* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TS = 2 * P + 1, TT = TS * TS;
    double* sT = reinterpret_cast<double*>(smem_raw);
    double* sJ = sT + TT;
    double* sA = sJ + Q * TS;
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < TT; j += blockDim.x) sT[j] = 0.0;
    __syncthreads();
    lf_sommerfeld_table_block(c, rho[i] / S, z[i] / S, S, 2 * P, sT, TS, Q, gt, gw, sJ, sA);
    for (int j = threadIdx.x; j < TT; j += blockDim.x) out[(size_t)i * TT + j] = sT[j];
}

LfErr lf_sommerfeld_tables_dev(lfmm_ctx* ctx, int comp, int npts, const double* rho, const double* z, double S,
                               int P, double* out)
{
    const int TS = 2 * P + 1;
    const int Q = ctx->gl_q_m2l;
    size_t sm = sizeof(double) * ((size_t)TS * TS + 2 * (size_t)Q * TS);
    LF_CHECK(cudaFuncSetAttribute(k_som_tables, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    ++ctx->launches, k_som_tables<<<npts, 128, sm, ctx->s_main>>>(ctx->comp[comp], npts, rho, z, S, P, ctx->gl_t_m2l.as<double>(),
                                                  ctx->gl_w_m2l.as<double>(), Q, out);
    return lf_cuda(cudaGetLastError(), "sommerfeld tables");
}

__global__ void k_reaction_kernel(int comp, int npts, const double* __restrict__ rho, const double* __restrict__ h,
                                  int Q, double* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    double k00, k10, k11;
    lf_reaction_pair<double>(c_ncomp[comp], rho[i], h[i], Q, k00, k10, k11);
    out[3 * (size_t)i] = k00;
    out[3 * (size_t)i + 1] = k10;
    out[3 * (size_t)i + 2] = k11;
}

LfErr lf_reaction_kernel_dev(lfmm_ctx* ctx, int comp, int npts, const double* rho, const double* h, double* out)
{
    LF_TRY(upload_consts(ctx, ctx->s_main));
    ++ctx->launches, k_reaction_kernel<<<lf_blocks(npts, 128), 128, 0, ctx->s_main>>>(comp, npts, rho, h, ctx->gl_q_near, out);
    return lf_cuda(cudaGetLastError(), "reaction kernel");
}

// ---------------------------------------------------------------------------
// Allocation-free variant of lfmm_reaction_kernel.
//
// Some callers cannot allocate device memory at the point where they need the
// layered reaction kernel: code running inside a stream capture, real-time or
// embedded loops that forbid allocator calls, or hosts that manage a fixed
// device-memory budget themselves.  lfmm_reaction_kernel stages its inputs and
// outputs through buffers it allocates on every call; this variant stages them
// through one file-scope device array instead, so the call itself makes no
// cudaMalloc / cudaFree (or any other allocating call).
//
// The array holds LFMM_NOALLOC_MAX_POINTS points (rho, h and three outputs per
// point: 5 doubles, 2.6 MB).  It is defined once per process and every GPU
// that loads this library keeps its copy until the process exits.  All calls
// share it and it keeps the last call's contents; nothing in it needs to start
// at zero because every entry a call reads is written by that call first.
// Calls that overlap on the GPU (several host threads, several contexts on one
// device) race on the array and must be serialised by the caller.
//
// The device address of the array is resolved with cudaGetSymbolAddress the
// first time the entry point runs on a device (with that device current) and
// cached per device; that first call therefore must not happen inside a stream
// capture.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_scratch[5 * LFMM_NOALLOC_MAX_POINTS];

static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[LFMM_MAX_DEVICES] = {nullptr};

static LfErr noalloc_scratch(int device, double** out)
{
    if (device < 0 || device >= LFMM_MAX_DEVICES) return "EINVAL: device index out of range";
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return lf_cuda(e, "cudaGetDevice");
        if (cur != device) {
            e = cudaSetDevice(device);
            if (e != cudaSuccess) return lf_cuda(e, "cudaSetDevice");
        }
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (cur != device) cudaSetDevice(cur);
        if (e != cudaSuccess) return lf_cuda(e, "cudaGetSymbolAddress");
        g_noalloc_ptr[device] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[device];
    return LfErr();
}

extern "C" lfmm_status lfmm_reaction_kernel_noalloc(lfmm_ctx* ctx, int l, int lp, int a, int b, int npts,
                                                     const double* rho, const double* h, double* out)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    int c = lf_find_comp(ctx, l, lp, a, b);
    if (c < 0) {
        ctx->err = "EINVAL: no such reaction component";
        return LFMM_EINVAL;
    }
    if (npts < 1 || !rho || !h || !out) {
        ctx->err = "EINVAL: bad kernel request";
        return LFMM_EINVAL;
    }
    if (npts > LFMM_NOALLOC_MAX_POINTS) {
        ctx->err = "EINVAL: npts exceeds LFMM_NOALLOC_MAX_POINTS (" + std::to_string(LFMM_NOALLOC_MAX_POINTS) +
                   ") of the allocation-free entry point";
        return LFMM_EINVAL;
    }
    for (int i = 0; i < npts; ++i)
        if (!(h[i] > 0.0) || !(rho[i] >= 0.0)) {
            ctx->err = "EINVAL: need h > 0 and rho >= 0";
            return LFMM_EINVAL;
        }
    double* base = nullptr;
    LfErr e = noalloc_scratch(ctx->device, &base);
    double* drho = base;
    double* dh = base + LFMM_NOALLOC_MAX_POINTS;
    double* dout = base + 2 * LFMM_NOALLOC_MAX_POINTS;
    cudaStream_t st = ctx->s_main;
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(drho, rho, sizeof(double) * npts, cudaMemcpyHostToDevice, st), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dh, h, sizeof(double) * npts, cudaMemcpyHostToDevice, st), "copy");
    if (e.empty()) e = upload_consts(ctx, st);
    if (e.empty()) {
        ++ctx->launches, k_reaction_kernel<<<lf_blocks(npts, 128), 128, 0, st>>>(c, npts, drho, dh, ctx->gl_q_near, dout);
        e = lf_cuda(cudaGetLastError(), "reaction kernel");
    }
    if (e.empty())
        e = lf_cuda(cudaMemcpyAsync(out, dout, sizeof(double) * 3 * npts, cudaMemcpyDeviceToHost, st), "copy back");
    if (e.empty()) e = lf_cuda(cudaStreamSynchronize(st), "reaction kernel");
    if (!e.empty()) {
        ctx->err = e;
        return e.compare(0, 6, "EINVAL") == 0 ? LFMM_EINVAL : LFMM_ECUDA;
    }
    return LFMM_OK;
}
