// lfmm_surrogate.cu -- learned surrogate for the near-field reaction kernels.
//
// Not in the paper: for each reaction component a small network replaces the
// Sommerfeld quadrature of the local direct interactions of Algorithm 1 (the
// integrals I_00, I_10, I_11 of a pair).  The closed-form leading image of
// the density stays exact; the network predicts the remainder
//   y_k = (K_k - lead_k) / s_k,  s_0 = |C_r| / R_r,  s_1 = s_2 = |C_r| / R_r^2,
// R_r = sqrt(rho^2 + (h + zeta_r)^2), with C_r e^{-k zeta_r} the remainder's
// leading term, standardised per output.  Inputs (4): log10 rho, the target
// and source depths below/above their interfaces (h_t, h_s) and
// log10(rho / h), h = h_t + h_s, each mapped to about [-1, 1].
// Network: 4 -> 64 -> 64 -> 64 -> 3, SiLU, one network per component,
// weights stored as bfloat16, biases and all accumulation in float32.
//
// Training (on the device, by the kernels below): labels from the FP64
// quadrature (lf_reaction_pair), mean-squared loss, Adam on float32 master
// weights; the forward pass uses the bfloat16-rounded weights and their
// gradient updates the master weights (straight-through).
// Inference: one warp evaluates 32 pairs with mma.sync m16n8k16 (bfloat16
// operands, float32 accumulate).  Activations and inputs are split into a
// bfloat16 high part and a bfloat16 remainder (two MMAs), so they carry ~16
// significant bits.  A per-component table of the validation error on a
// 32 x 32 grid of (log10 rho, log10 h) is the error estimate: a pair whose cell
// error exceeds the tolerance, or that lies outside the trained range, falls
// back to the quadrature.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <random>
#include <vector>

#include "lfmm_ctx.h"
#include "lfmm_surrogate.cuh"

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

// ---------------------------------------------------------------------------
// Labels: FP64 quadrature of the three kernels for every sample.
// in: rho, ht, hs (double); out: x [n][4] float, y [n][3] float (raw), and for
// validation the exact kernels and the lead scales (double [n][3] each).
// ---------------------------------------------------------------------------
__global__ void k_surr_labels(LfmmComp c, LfmmSurrMeta m, int n, const double* __restrict__ rho,
                              const double* __restrict__ ht, const double* __restrict__ hs, int Q,
                              const double* __restrict__ gt, const double* __restrict__ gw, float* __restrict__ x,
                              float* __restrict__ y, double* __restrict__ kex)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double h = ht[i] + hs[i];
    double k00, k10, k11;
    lf_reaction_pair<double>(c, rho[i], h, Q, gt, gw, k00, k10, k11);
    double lead[3], sc[3];
    surr_lead(c, rho[i], h, lead, sc);
    float f[4];
    surr_features(m, (float)rho[i], (float)ht[i], (float)hs[i], f);
    for (int k = 0; k < 4; ++k) x[4 * (size_t)i + k] = f[k];
    y[3 * (size_t)i + 0] = (float)((k00 - lead[0]) / sc[0]);
    y[3 * (size_t)i + 1] = (float)((k10 - lead[1]) / sc[1]);
    y[3 * (size_t)i + 2] = (float)((k11 - lead[2]) / sc[2]);
    if (kex) {
        kex[3 * (size_t)i + 0] = k00;
        kex[3 * (size_t)i + 1] = k10;
        kex[3 * (size_t)i + 2] = k11;
    }
}

// ---------------------------------------------------------------------------
// Training: forward + backward of TRAIN_B samples per block, gradients summed
// into grad (float32, atomics).  Loss = (1/ntot) sum (out - ystd)^2.
// ---------------------------------------------------------------------------
struct TrainArgs {
    const float* theta;  // [ncomp][NP]
    float* grad;         // [ncomp][NP]
    const float* x;      // per component: [n][4]
    const float* y;      // per component: [n][3]
    const int64_t* xoff; // per component: sample offset into x/y
    const int* nsamp;    // per component: number of samples
    const int* comps;    // trained component ids (grid.y index -> component)
    const LfmmSurrMeta* meta;
    int start;           // first sample of this step (wraps)
    int ntot;            // samples per component in this step (for the mean)
    double* loss;        // [ncomp] accumulated loss
};

__global__ void __launch_bounds__(TRAIN_B) k_surr_train(TrainArgs a)
{
    extern __shared__ __align__(16) float sm[];
    float* P = sm;                          // parameters (weights rounded to bf16), LFMM_SURR_NP
    float* Z1 = P + LFMM_SURR_NP;           // [64][S] pre-activations / deltas
    float* A1 = Z1 + 64 * TRAIN_S;          // activations
    float* Z2 = A1 + 64 * TRAIN_S;
    float* A2 = Z2 + 64 * TRAIN_S;
    float* Z3 = A2 + 64 * TRAIN_S;
    float* A3 = Z3 + 64 * TRAIN_S;
    float* X = A3 + 64 * TRAIN_S;           // [4][S]
    float* DO = X + 4 * TRAIN_S;            // [3][S]
    __shared__ float s_loss[TRAIN_B];
    const int c = a.comps[blockIdx.y];
    const int b = threadIdx.x;
    const LfmmSurrMeta m = a.meta[c];
    const float* th = a.theta + (size_t)c * LFMM_SURR_NP;
    for (int i = b; i < LFMM_SURR_NP; i += TRAIN_B) {
        float v = th[i];
        bool isw = (i < SO_B1) || (i >= SO_W2 && i < SO_B2) || (i >= SO_W3 && i < SO_B3) || (i >= SO_W4 && i < SO_B4);
        P[i] = isw ? bf16r(v) : v;
    }
    const int ns = a.nsamp[c];
    int si = (a.start + blockIdx.x * TRAIN_B + b) % ns;
    const float* xs = a.x + (size_t)a.xoff[c] * 4 + (size_t)si * 4;
    const float* ys = a.y + (size_t)a.xoff[c] * 3 + (size_t)si * 3;
    float xv[4], yv[3];
    for (int k = 0; k < 4; ++k) {
        xv[k] = xs[k];
        X[k * TRAIN_S + b] = xv[k];
    }
    for (int k = 0; k < 3; ++k) yv[k] = (ys[k] - m.mu[k]) / m.sd[k];
    __syncthreads();
    // forward
    for (int j = 0; j < 64; ++j) {
        float z = P[SO_B1 + j];
        for (int i = 0; i < 4; ++i) z += P[SO_W1 + j * 4 + i] * xv[i];
        Z1[j * TRAIN_S + b] = z;
        A1[j * TRAIN_S + b] = silu_f(z);
    }
    for (int j = 0; j < 64; ++j) {
        float z = P[SO_B2 + j];
        for (int i = 0; i < 64; ++i) z += P[SO_W2 + j * 64 + i] * A1[i * TRAIN_S + b];
        Z2[j * TRAIN_S + b] = z;
        A2[j * TRAIN_S + b] = silu_f(z);
    }
    for (int j = 0; j < 64; ++j) {
        float z = P[SO_B3 + j];
        for (int i = 0; i < 64; ++i) z += P[SO_W3 + j * 64 + i] * A2[i * TRAIN_S + b];
        Z3[j * TRAIN_S + b] = z;
        A3[j * TRAIN_S + b] = silu_f(z);
    }
    float lsum = 0.f;
    const float inv = 1.0f / (float)a.ntot;
    for (int k = 0; k < 3; ++k) {
        float o = P[SO_B4 + k];
        for (int i = 0; i < 64; ++i) o += P[SO_W4 + k * 64 + i] * A3[i * TRAIN_S + b];
        float r = o - yv[k];
        lsum += r * r;
        DO[k * TRAIN_S + b] = 2.0f * r * inv;
    }
    s_loss[b] = lsum;
    // backward: delta3 into Z3 (own column)
    for (int i = 0; i < 64; ++i) {
        float s = 0.f;
        for (int k = 0; k < 3; ++k) s += P[SO_W4 + k * 64 + i] * DO[k * TRAIN_S + b];
        Z3[i * TRAIN_S + b] = s * dsilu_f(Z3[i * TRAIN_S + b]);
    }
    // delta2 into Z2
    for (int i = 0; i < 64; ++i) {
        float s = 0.f;
        for (int j = 0; j < 64; ++j) s += P[SO_W3 + j * 64 + i] * Z3[j * TRAIN_S + b];
        Z2[i * TRAIN_S + b] = s * dsilu_f(Z2[i * TRAIN_S + b]);
    }
    // delta1 into Z1
    for (int i = 0; i < 64; ++i) {
        float s = 0.f;
        for (int j = 0; j < 64; ++j) s += P[SO_W2 + j * 64 + i] * Z2[j * TRAIN_S + b];
        Z1[i * TRAIN_S + b] = s * dsilu_f(Z1[i * TRAIN_S + b]);
    }
    __syncthreads();
    // weight gradients summed over the block's samples
    float* g = a.grad + (size_t)c * LFMM_SURR_NP;
    for (int e = b; e < 3 * 64; e += TRAIN_B) {
        int k = e / 64, i = e % 64;
        float s = 0.f;
        for (int q = 0; q < TRAIN_B; ++q) s += DO[k * TRAIN_S + q] * A3[i * TRAIN_S + q];
        atomicAdd(&g[SO_W4 + e], s);
    }
    if (b < 3) {
        float s = 0.f;
        for (int q = 0; q < TRAIN_B; ++q) s += DO[b * TRAIN_S + q];
        atomicAdd(&g[SO_B4 + b], s);
    }
    const float* D[3] = {Z1, Z2, Z3};
    const float* Ain[3] = {X, A1, A2};
    const int wo[3] = {SO_W1, SO_W2, SO_W3}, bo[3] = {SO_B1, SO_B2, SO_B3}, nin[3] = {4, 64, 64};
    for (int L = 0; L < 3; ++L) {
        const int ni = nin[L];
        for (int e = b; e < 64 * ni; e += TRAIN_B) {
            int j = e / ni, i = e % ni;
            float s = 0.f;
            for (int q = 0; q < TRAIN_B; ++q) s += D[L][j * TRAIN_S + q] * Ain[L][i * TRAIN_S + q];
            atomicAdd(&g[wo[L] + e], s);
        }
        {
            int j = b;  // 64 threads, 64 biases
            float s = 0.f;
            for (int q = 0; q < TRAIN_B; ++q) s += D[L][j * TRAIN_S + q];
            atomicAdd(&g[bo[L] + j], s);
        }
    }
    if (b == 0 && a.loss) {
        float t = 0.f;
        for (int q = 0; q < TRAIN_B; ++q) t += s_loss[q];
        atomicAdd(&a.loss[c], (double)t * inv);
    }
}

__global__ void k_adam(float* __restrict__ theta, float* __restrict__ grad, float* __restrict__ m1,
                       float* __restrict__ m2, int n, float lr, float b1, float b2, float bc1, float bc2, float eps)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float g = grad[i];
    float a = b1 * m1[i] + (1.0f - b1) * g;
    float v = b2 * m2[i] + (1.0f - b2) * g * g;
    m1[i] = a;
    m2[i] = v;
    theta[i] -= lr * (a / bc1) / (sqrtf(v / bc2) + eps);
    grad[i] = 0.f;
}

// bfloat16 inference weights and float32 biases from the master parameters
__global__ void k_surr_pack(const float* __restrict__ theta, const int* __restrict__ comps, int c0,
                            __nv_bfloat16* __restrict__ w, float* __restrict__ bias)
{
    const int c = comps ? comps[blockIdx.x] : c0;
    const float* th = theta + (size_t)c * LFMM_SURR_NP;
    __nv_bfloat16* wc = w + (size_t)c * SW_N;
    float* bc = bias + (size_t)c * SB_N;
    for (int e = threadIdx.x; e < SW_N; e += blockDim.x) {
        const int frag = e >> 7, lane = (e >> 2) & 31, j = e & 3;
        const int g = lane >> 2, t = lane & 3;
        const int kk = 2 * t + (j & 1) + ((j & 2) ? 8 : 0);
        int wo, nin, nout, nt, ks;
        if (frag < SW_F2) {
            wo = SO_W1, nin = 4, nout = 64, nt = frag - SW_F1, ks = 0;
        } else if (frag < SW_F3) {
            wo = SO_W2, nin = 64, nout = 64, nt = (frag - SW_F2) >> 2, ks = (frag - SW_F2) & 3;
        } else if (frag < SW_F4) {
            wo = SO_W3, nin = 64, nout = 64, nt = (frag - SW_F3) >> 2, ks = (frag - SW_F3) & 3;
        } else {
            wo = SO_W4, nin = 64, nout = 3, nt = 0, ks = frag - SW_F4;
        }
        const int n = 8 * nt + g, k = 16 * ks + kk;
        const float v = (n < nout && k < nin) ? th[wo + n * nin + k] : 0.f;
        wc[e] = __float2bfloat16_rn(v);
    }
    for (int e = threadIdx.x; e < SB_N; e += blockDim.x) {
        float v = 0.f;
        if (e < 64) v = th[SO_B1 + e];
        else if (e < 128) v = th[SO_B2 + e - 64];
        else if (e < 192) v = th[SO_B3 + e - 128];
        else if (e < 195) v = th[SO_B4 + e - 192];
        bc[e] = v;
    }
}

// Validation: one warp per 32 samples; per-cell maximum error relative to the
// kernel scale (surr_err_scale), as float bits (non-negative floats order as
// integers), and per-cell sample counts (cells without samples are rejected).
__global__ void k_surr_validate(LfmmComp c, LfmmSurrMeta m, int n, const double* __restrict__ rho,
                                const double* __restrict__ ht, const double* __restrict__ hs,
                                const double* __restrict__ kex, const __nv_bfloat16* __restrict__ W,
                                const float* __restrict__ B, unsigned int* __restrict__ cellerr,
                                unsigned int* __restrict__ cellcnt, unsigned int* __restrict__ gmax)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const int ii = valid ? i : 0;
    float f[4];
    surr_features(m, (float)rho[ii], (float)ht[ii], (float)hs[ii], f);
    float y[3];
    lf_surr_warp(W, B, f, y);
    if (!valid) return;
    double h = fmax(ht[i] + hs[i], 1e-4);
    double K[3];
    lf_surr_kernels(c, m, rho[i], h, y, K);
    double s0, s1;
    surr_err_scale(c, rho[i], h, s0, s1);
    double e = fabs(K[0] - kex[3 * (size_t)i]) / s0;
    e = fmax(e, fabs(K[1] - kex[3 * (size_t)i + 1]) / s1);
    e = fmax(e, fabs(K[2] - kex[3 * (size_t)i + 2]) / s1);
    float ef = (float)e;
    if (!(ef <= 1e30f)) ef = 1e30f;
    const int cell = surr_cell(m, (float)rho[i], (float)(ht[i] + hs[i]));
    atomicMax(&cellerr[cell], __float_as_uint(ef));
    atomicAdd(&cellcnt[cell], 1u);
    atomicMax(gmax, __float_as_uint(ef));
}

// Raw network outputs (standardised) for caller features: one warp per 32.
__global__ void k_surr_forward(int n, const float* __restrict__ x, const __nv_bfloat16* __restrict__ W,
                               const float* __restrict__ B, float* __restrict__ y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int ii = i < n ? i : 0;
    float f[4], o[3];
    for (int k = 0; k < 4; ++k) f[k] = x[4 * (size_t)ii + k];
    lf_surr_warp(W, B, f, o);
    if (i >= n) return;
    for (int k = 0; k < 3; ++k) y[3 * (size_t)i + k] = o[k];
}

// Inference on caller points (parity entry point): one warp per 32 points.
__global__ void k_surr_eval(LfmmComp c, LfmmSurrMeta m, int n, const double* __restrict__ rho,
                            const double* __restrict__ ht, const double* __restrict__ hs,
                            const __nv_bfloat16* __restrict__ W, const float* __restrict__ B,
                            const float* __restrict__ err, float tol, double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const int ii = valid ? i : 0;
    float f[4];
    surr_features(m, (float)rho[ii], (float)ht[ii], (float)hs[ii], f);
    float y[3];
    lf_surr_warp(W, B, f, y);
    if (!valid) return;
    double h = fmax(ht[i] + hs[i], 1e-4);
    double K[3];
    lf_surr_kernels(c, m, rho[i], h, y, K);
    out[4 * (size_t)i + 0] = K[0];
    out[4 * (size_t)i + 1] = K[1];
    out[4 * (size_t)i + 2] = K[2];
    out[4 * (size_t)i + 3] = lf_surr_cell_ok(m, err, (float)rho[i], (float)ht[i], (float)hs[i], tol) ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------
// Host driver.
// ---------------------------------------------------------------------------
static void layer_depths(const lfmm_ctx* ctx, const LfmmComp& c, float& Tt, float& Ts)
{
    // depth ranges of the training samples: the middle layer's thickness, or
    // for the half-spaces the same span (charges are expected within it)
    double D = (ctx->L == 2) ? ctx->d[0] - ctx->d[1] : 1.0;
    Tt = (float)D;
    Ts = (float)D;
    (void)c;
}

static uint64_t splitmix(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double unif(uint64_t& s) { return (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

LfErr lf_surrogate_train(lfmm_ctx* ctx, int64_t nsamples, int epochs, uint64_t seed)
{
    if (ctx->L != 2) return "EINVAL: the surrogate is built for three-layer media";
    if (nsamples < 1000 || epochs < 1) return "EINVAL: need nsamples >= 1000 and epochs >= 1";
    cudaStream_t st = ctx->s_main;
    std::vector<int> comps;
    for (int c = 0; c < ctx->ncomp; ++c)
        if (!ctx->comp[c].is_free && ctx->comp[c].has_rem) comps.push_back(c);
    if (comps.empty()) return "EINVAL: no reaction component with a remainder to learn";
    const int nc = (int)comps.size();
    if (nsamples > (1 << 26)) return "EINVAL: at most 2^26 samples per component";
    const int ntrain = (int)std::max<int64_t>(TRAIN_B, nsamples);
    const int nval = std::max(4096, ntrain / 10);
    const int per = ntrain + nval;
    // samples (host, splitmix64): rho log-uniform in [1e-3, 3]; the two depths
    // uniform in [0, T] for half the samples and log-uniform in [1e-4, T] for
    // the other half (near-field reaction pairs sit close to an interface);
    // pairs with h_t + h_s below SURR_HMIN are drawn again
    std::vector<double> hr((size_t)nc * per), hht((size_t)nc * per), hhs((size_t)nc * per);
    uint64_t s = seed;
    std::vector<LfmmSurrMeta> meta(ctx->ncomp);
    for (int k = 0; k < nc; ++k) {
        LfmmSurrMeta& m = meta[comps[k]];
        memset(&m, 0, sizeof(m));
        layer_depths(ctx, ctx->comp[comps[k]], m.Tt, m.Ts);
        const double lt0 = log(1e-4), ltt = log((double)m.Tt), lts = log((double)m.Ts);
        for (int i = 0; i < per; ++i) {
            size_t j = (size_t)k * per + i;
            hr[j] = pow(10.0, -3.0 + unif(s) * 3.4771212547196626);
            do {
                if (i & 1) {
                    hht[j] = exp(lt0 + unif(s) * (ltt - lt0));
                    hhs[j] = exp(lt0 + unif(s) * (lts - lt0));
                } else {
                    hht[j] = unif(s) * m.Tt;
                    hhs[j] = unif(s) * m.Ts;
                }
            } while (hht[j] + hhs[j] < (double)SURR_HMIN);
        }
    }
    DevBuf drho, dht, dhs, dx, dy, dk;
    auto cleanup = [&]() {
        DevBuf* b[] = {&drho, &dht, &dhs, &dx, &dy, &dk};
        for (DevBuf* p : b)
            if (p->ptr) cudaFree(p->ptr);
    };
    const size_t ntot = (size_t)nc * per;
    LfErr e = lf_reserve(drho, ntot * 8);
    if (e.empty()) e = lf_reserve(dht, ntot * 8);
    if (e.empty()) e = lf_reserve(dhs, ntot * 8);
    if (e.empty()) e = lf_reserve(dx, ntot * 16);
    if (e.empty()) e = lf_reserve(dy, ntot * 12);
    if (e.empty()) e = lf_reserve(dk, ntot * 24);
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(drho.ptr, hr.data(), ntot * 8, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dht.ptr, hht.data(), ntot * 8, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dhs.ptr, hhs.data(), ntot * 8, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (!e.empty()) {
        cleanup();
        return e;
    }
    // labels by the FP64 quadrature
    for (int k = 0; k < nc; ++k) {
        size_t o = (size_t)k * per;
        ++ctx->launches, k_surr_labels<<<lf_blocks(per, 128), 128, 0, st>>>(
            ctx->comp[comps[k]], meta[comps[k]], per, drho.as<double>() + o, dht.as<double>() + o,
            dhs.as<double>() + o, ctx->gl_q_near, ctx->gl_t_near.as<double>(), ctx->gl_w_near.as<double>(),
            dx.as<float>() + 4 * o, dy.as<float>() + 3 * o, dk.as<double>() + 3 * o);
    }
    e = lf_cuda(cudaGetLastError(), "surrogate labels");
    std::vector<float> hy(ntot * 3);
    if (e.empty()) e = lf_cuda(lf_d2h(hy.data(), dy.ptr, ntot * 12, ctx->s_main), "copy labels");
    if (!e.empty()) {
        cleanup();
        return e;
    }
    // output standardisation from the training part
    for (int k = 0; k < nc; ++k) {
        LfmmSurrMeta& m = meta[comps[k]];
        for (int q = 0; q < 3; ++q) {
            double s1 = 0, s2 = 0;
            for (int i = 0; i < ntrain; ++i) {
                double v = hy[((size_t)k * per + i) * 3 + q];
                s1 += v;
                s2 += v * v;
            }
            double mu = s1 / ntrain, var = std::max(s2 / ntrain - mu * mu, 1e-30);
            m.mu[q] = (float)mu;
            m.sd[q] = (float)std::max(sqrt(var), 1e-6);
        }
        m.trained = 1;
    }
    // parameters: Glorot-uniform weights (seeded), zero biases
    const size_t np = (size_t)ctx->ncomp * LFMM_SURR_NP;
    std::vector<float> theta(np, 0.f);
    for (int k = 0; k < nc; ++k) {
        float* th = &theta[(size_t)comps[k] * LFMM_SURR_NP];
        auto init = [&](int off, int nout, int nin) {
            double a = sqrt(6.0 / (nin + nout));
            for (int i = 0; i < nout * nin; ++i) th[off + i] = (float)((2.0 * unif(s) - 1.0) * a);
        };
        init(SO_W1, 64, 4);
        init(SO_W2, 64, 64);
        init(SO_W3, 64, 64);
        init(SO_W4, 3, 64);
    }
    LfErr e2 = lf_reserve(ctx->surr_theta, np * 4);
    if (e2.empty()) e2 = lf_reserve(ctx->surr_grad, np * 4);
    if (e2.empty()) e2 = lf_reserve(ctx->surr_m1, np * 4);
    if (e2.empty()) e2 = lf_reserve(ctx->surr_m2, np * 4);
    if (e2.empty()) e2 = lf_reserve(ctx->surr_w, (size_t)ctx->ncomp * SW_N * 2);
    if (e2.empty()) e2 = lf_reserve(ctx->surr_b, (size_t)ctx->ncomp * SB_N * 4);
    if (e2.empty()) e2 = lf_reserve(ctx->surr_meta, sizeof(LfmmSurrMeta) * ctx->ncomp);
    if (e2.empty()) e2 = lf_reserve(ctx->surr_err, sizeof(float) * ctx->ncomp * LFMM_SURR_CELLS * LFMM_SURR_CELLS);
    if (e2.empty()) e2 = lf_reserve(ctx->surr_comps, sizeof(int) * nc);
    if (e2.empty()) e2 = lf_reserve(ctx->surr_xoff, sizeof(int64_t) * ctx->ncomp + sizeof(int) * ctx->ncomp + 64);
    if (!e2.empty()) {
        cleanup();
        return e2;
    }
    std::vector<int64_t> xoff(ctx->ncomp, 0);
    std::vector<int> nsamp(ctx->ncomp, 1);
    for (int k = 0; k < nc; ++k) {
        xoff[comps[k]] = (int64_t)k * per;
        nsamp[comps[k]] = ntrain;
    }
    int64_t* dxoff = ctx->surr_xoff.as<int64_t>();
    int* dns = reinterpret_cast<int*>(dxoff + ctx->ncomp);
    e = lf_cuda(cudaMemcpyAsync(ctx->surr_theta.ptr, theta.data(), np * 4, cudaMemcpyHostToDevice, ctx->s_main), "copy params");
    if (e.empty()) e = lf_cuda(cudaMemsetAsync(ctx->surr_grad.ptr, 0, np * 4, ctx->s_main), "zero");
    if (e.empty()) e = lf_cuda(cudaMemsetAsync(ctx->surr_m1.ptr, 0, np * 4, ctx->s_main), "zero");
    if (e.empty()) e = lf_cuda(cudaMemsetAsync(ctx->surr_m2.ptr, 0, np * 4, ctx->s_main), "zero");
    if (e.empty())
        e = lf_cuda(cudaMemcpyAsync(ctx->surr_meta.ptr, meta.data(), sizeof(LfmmSurrMeta) * ctx->ncomp, cudaMemcpyHostToDevice, ctx->s_main), "copy meta");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(ctx->surr_comps.ptr, comps.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dxoff, xoff.data(), sizeof(int64_t) * ctx->ncomp, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dns, nsamp.data(), sizeof(int) * ctx->ncomp, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (!e.empty()) {
        cleanup();
        return e;
    }
    // training loop
    const int blocks = 32;
    const int step_n = blocks * TRAIN_B;
    const int64_t steps = (int64_t)epochs * ((ntrain + step_n - 1) / step_n);
    const size_t sm = sizeof(float) * ((size_t)LFMM_SURR_NP + 6 * 64 * TRAIN_S + 7 * TRAIN_S);
    e = lf_cuda(cudaFuncSetAttribute(k_surr_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm), "attr");
    DevBuf dloss;
    if (e.empty()) e = lf_reserve(dloss, sizeof(double) * ctx->ncomp);
    const float b1 = 0.9f, b2 = 0.999f;
    double pb1 = 1.0, pb2 = 1.0;
    const double lr0 = 2e-3, lr1 = 1e-5;
    for (int64_t it = 0; it < steps && e.empty(); ++it) {
        TrainArgs a;
        a.theta = ctx->surr_theta.as<float>();
        a.grad = ctx->surr_grad.as<float>();
        a.x = dx.as<float>();
        a.y = dy.as<float>();
        a.xoff = dxoff;
        a.nsamp = dns;
        a.comps = ctx->surr_comps.as<int>();
        a.meta = ctx->surr_meta.as<LfmmSurrMeta>();
        a.start = (int)((it * step_n) % ntrain);
        a.ntot = step_n;
        a.loss = nullptr;
        if (it == steps - 1) {
            cudaMemsetAsync(dloss.ptr, 0, sizeof(double) * ctx->ncomp, st);
            a.loss = dloss.as<double>();
        }
        ++ctx->launches, k_surr_train<<<dim3(blocks, nc), TRAIN_B, sm, st>>>(a);
        pb1 *= b1;
        pb2 *= b2;
        double lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + cos(M_PI * (double)it / (double)steps));
        ++ctx->launches, k_adam<<<lf_blocks(np, 256), 256, 0, st>>>(
            ctx->surr_theta.as<float>(), ctx->surr_grad.as<float>(), ctx->surr_m1.as<float>(),
            ctx->surr_m2.as<float>(), (int)np, (float)lr, b1, b2, (float)(1.0 - pb1), (float)(1.0 - pb2), 1e-8f);
        if ((it & 63) == 0) e = lf_cuda(cudaGetLastError(), "surrogate training");
    }
    if (e.empty()) e = lf_cuda(cudaGetLastError(), "surrogate training");
    std::vector<double> hloss(ctx->ncomp, 0.0);
    if (e.empty() && steps > 0)
        e = lf_cuda(lf_d2h(hloss.data(), dloss.ptr, sizeof(double) * ctx->ncomp, ctx->s_main), "loss");
    if (dloss.ptr) cudaFree(dloss.ptr);
    // pack inference weights and validate on the held-out samples
    if (e.empty()) {
        ++ctx->launches, k_surr_pack<<<nc, 256, 0, st>>>(ctx->surr_theta.as<float>(), ctx->surr_comps.as<int>(), 0,
                                                          ctx->surr_w.as<__nv_bfloat16>(), ctx->surr_b.as<float>());
        e = lf_cuda(cudaMemsetAsync(ctx->surr_err.ptr, 0,
                                    sizeof(float) * ctx->ncomp * LFMM_SURR_CELLS * LFMM_SURR_CELLS, st),
                    "zero err");
    }
    DevBuf dgmax;  // [ncomp] maxima, then [ncomp][CELLS^2] counts
    const size_t ncell = (size_t)LFMM_SURR_CELLS * LFMM_SURR_CELLS;
    const size_t gbytes = sizeof(unsigned int) * ctx->ncomp * (1 + ncell);
    if (e.empty()) e = lf_reserve(dgmax, gbytes);
    if (e.empty()) e = lf_cuda(cudaMemsetAsync(dgmax.ptr, 0, gbytes, st), "zero");
    for (int k = 0; k < nc && e.empty(); ++k) {
        int c = comps[k];
        size_t o = (size_t)k * per + ntrain;
        ++ctx->launches, k_surr_validate<<<lf_blocks(nval, 128), 128, 0, st>>>(
            ctx->comp[c], meta[c], nval, drho.as<double>() + o, dht.as<double>() + o, dhs.as<double>() + o,
            dk.as<double>() + 3 * o, ctx->surr_w.as<__nv_bfloat16>() + (size_t)c * SW_N,
            ctx->surr_b.as<float>() + (size_t)c * SB_N,
            reinterpret_cast<unsigned int*>(ctx->surr_err.as<float>() + (size_t)c * ncell),
            dgmax.as<unsigned int>() + ctx->ncomp + (size_t)c * ncell, dgmax.as<unsigned int>() + c);
    }
    if (e.empty()) e = lf_cuda(cudaStreamSynchronize(st), "surrogate validation");
    std::vector<unsigned int> gm(ctx->ncomp * (1 + ncell), 0);
    std::vector<float> cells((size_t)ctx->ncomp * ncell);
    if (e.empty()) e = lf_cuda(lf_d2h(gm.data(), dgmax.ptr, gbytes, ctx->s_main), "copy");
    if (e.empty())
        e = lf_cuda(lf_d2h(cells.data(), ctx->surr_err.ptr, sizeof(float) * cells.size(), ctx->s_main),
                    "copy");
    // a cell that no validation sample reached has no estimate: reject it
    for (size_t q = 0; q < cells.size(); ++q)
        if (gm[ctx->ncomp + q] == 0) cells[q] = 1e30f;
    if (e.empty())
        e = lf_cuda(cudaMemcpyAsync(ctx->surr_err.ptr, cells.data(), sizeof(float) * cells.size(), cudaMemcpyHostToDevice, ctx->s_main),
                    "copy");
    if (dgmax.ptr) cudaFree(dgmax.ptr);
    cleanup();
    if (!e.empty()) return e;
    for (int c = 0; c < ctx->ncomp; ++c) {
        float* info = ctx->surr_info[c];
        for (int q = 0; q < 8; ++q) info[q] = 0.f;
        if (!meta[c].trained) continue;
        float gmax;
        memcpy(&gmax, &gm[c], 4);
        int ok = 0;
        double nok = 0, nall = 0;
        const float* ce = &cells[(size_t)c * ncell];
        const unsigned int* cnt = &gm[ctx->ncomp + (size_t)c * ncell];
        for (size_t q = 0; q < ncell; ++q) {
            ok += ce[q] <= ctx->surr_tol;
            nall += cnt[q];
            if (ce[q] <= ctx->surr_tol) nok += cnt[q];
        }
        info[0] = 1.f;
        info[1] = gmax;
        info[2] = (float)ok / (float)ncell;
        info[3] = (float)hloss[c];
        info[4] = (float)ntrain;
        info[5] = (float)nval;
        info[6] = (float)(nall > 0 ? nok / nall : 0.0);
    }
    if (e.empty()) e = lf_cuda(cudaStreamSynchronize(st), "surrogate tables");
    if (!e.empty()) return e;
    for (int c = 0; c < ctx->ncomp; ++c) ctx->surr_meta_h[c] = meta[c];
    ctx->surr_ready = 1;
    return LfErr();
}

LfErr lf_surrogate_eval_dev(lfmm_ctx* ctx, int comp, int n, const double* rho, const double* ht, const double* hs,
                            double* out)
{
    if (!ctx->surr_ready || !ctx->surr_meta_h[comp].trained) return "ESTATE: surrogate not trained";
    ++ctx->launches, k_surr_eval<<<lf_blocks(n, 128), 128, 0, ctx->s_main>>>(
        ctx->comp[comp], ctx->surr_meta_h[comp], n, rho, ht, hs, ctx->surr_w.as<__nv_bfloat16>() + (size_t)comp * SW_N,
        ctx->surr_b.as<float>() + (size_t)comp * SB_N,
        ctx->surr_err.as<float>() + (size_t)comp * LFMM_SURR_CELLS * LFMM_SURR_CELLS, (float)ctx->surr_tol, out);
    return lf_cuda(cudaGetLastError(), "surrogate eval");
}

// Parameter storage for caller-set parameters (gradient and inference checks).
LfErr lf_surrogate_alloc(lfmm_ctx* ctx)
{
    const size_t np = (size_t)ctx->ncomp * LFMM_SURR_NP;
    if (!ctx->surr_theta.ptr) {
        LF_TRY(lf_reserve(ctx->surr_theta, np * 4));
        LF_CHECK(cudaMemsetAsync(ctx->surr_theta.ptr, 0, np * 4, ctx->s_main));
    }
    if (!ctx->surr_w.ptr) LF_TRY(lf_reserve(ctx->surr_w, (size_t)ctx->ncomp * SW_N * 2));
    if (!ctx->surr_b.ptr) LF_TRY(lf_reserve(ctx->surr_b, (size_t)ctx->ncomp * SB_N * 4));
    return LfErr();
}

// Re-derive one component's inference weights from its master parameters.
LfErr lf_surrogate_pack(lfmm_ctx* ctx, int comp)
{
    ++ctx->launches, k_surr_pack<<<1, 256, 0, ctx->s_main>>>(ctx->surr_theta.as<float>(), nullptr, comp,
                                                            ctx->surr_w.as<__nv_bfloat16>(), ctx->surr_b.as<float>());
    return lf_cuda(cudaGetLastError(), "surrogate pack");
}

LfErr lf_surrogate_forward_dev(lfmm_ctx* ctx, int comp, int n, const float* x, float* y)
{
    if (!ctx->surr_w.ptr) return "ESTATE: surrogate parameters not initialised";
    ++ctx->launches, k_surr_forward<<<lf_blocks(n, 128), 128, 0, ctx->s_main>>>(
        n, x, ctx->surr_w.as<__nv_bfloat16>() + (size_t)comp * SW_N, ctx->surr_b.as<float>() + (size_t)comp * SB_N, y);
    return lf_cuda(cudaGetLastError(), "surrogate forward");
}

// Loss and gradient of one component's network on caller samples with the
// current master parameters (gradient check).
LfErr lf_surrogate_grad_dev(lfmm_ctx* ctx, int comp, int n, const float* x, const float* ystd, double* loss,
                            float* grad)
{
    if (!ctx->surr_theta.ptr) return "ESTATE: surrogate parameters not initialised";
    if (n % TRAIN_B) return "EINVAL: the gradient check takes a multiple of 64 samples";
    // identity standardisation for this call
    LfmmSurrMeta m = ctx->surr_meta_h[comp];
    for (int q = 0; q < 3; ++q) {
        m.mu[q] = 0.f;
        m.sd[q] = 1.f;
    }
    DevBuf dmeta, dcomp, doff, dgrad, dl;
    auto cleanup = [&]() {
        DevBuf* b[] = {&dmeta, &dcomp, &doff, &dgrad, &dl};
        for (DevBuf* p : b)
            if (p->ptr) cudaFree(p->ptr);
    };
    std::vector<LfmmSurrMeta> metas(ctx->ncomp, m);
    const size_t np = (size_t)ctx->ncomp * LFMM_SURR_NP;
    LfErr e = lf_reserve(dmeta, sizeof(LfmmSurrMeta) * ctx->ncomp);
    if (e.empty()) e = lf_reserve(dcomp, sizeof(int));
    if (e.empty()) e = lf_reserve(doff, sizeof(int64_t) * ctx->ncomp + sizeof(int) * ctx->ncomp);
    if (e.empty()) e = lf_reserve(dgrad, np * 4);
    if (e.empty()) e = lf_reserve(dl, sizeof(double) * ctx->ncomp);
    std::vector<int64_t> off(ctx->ncomp, 0);
    std::vector<int> ns(ctx->ncomp, n);
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dmeta.ptr, metas.data(), sizeof(LfmmSurrMeta) * ctx->ncomp, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dcomp.ptr, &comp, sizeof(int), cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemcpyAsync(doff.ptr, off.data(), sizeof(int64_t) * ctx->ncomp, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty())
        e = lf_cuda(cudaMemcpyAsync(doff.as<char>() + sizeof(int64_t) * ctx->ncomp, ns.data(), sizeof(int) * ctx->ncomp, cudaMemcpyHostToDevice, ctx->s_main), "copy");
    if (e.empty()) e = lf_cuda(cudaMemsetAsync(dgrad.ptr, 0, np * 4, ctx->s_main), "zero");
    if (e.empty()) e = lf_cuda(cudaMemsetAsync(dl.ptr, 0, sizeof(double) * ctx->ncomp, ctx->s_main), "zero");
    if (!e.empty()) {
        cleanup();
        return e;
    }
    TrainArgs a;
    a.theta = ctx->surr_theta.as<float>();
    a.grad = dgrad.as<float>();
    a.x = x;
    a.y = ystd;
    a.xoff = doff.as<int64_t>();
    a.nsamp = reinterpret_cast<const int*>(doff.as<char>() + sizeof(int64_t) * ctx->ncomp);
    a.comps = dcomp.as<int>();
    a.meta = dmeta.as<LfmmSurrMeta>();
    a.start = 0;
    a.ntot = n;
    a.loss = dl.as<double>();
    const size_t sm = sizeof(float) * ((size_t)LFMM_SURR_NP + 6 * 64 * TRAIN_S + 7 * TRAIN_S);
    e = lf_cuda(cudaFuncSetAttribute(k_surr_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm), "attr");
    if (e.empty()) {
        ++ctx->launches, k_surr_train<<<dim3(n / TRAIN_B, 1), TRAIN_B, sm, ctx->s_main>>>(a);
        e = lf_cuda(cudaStreamSynchronize(ctx->s_main), "surrogate gradient");
    }
    if (e.empty()) e = lf_cuda(lf_d2h(grad, dgrad.as<float>() + (size_t)comp * LFMM_SURR_NP, LFMM_SURR_NP * 4, ctx->s_main), "copy");
    std::vector<double> hl(ctx->ncomp);
    if (e.empty()) e = lf_cuda(lf_d2h(hl.data(), dl.ptr, sizeof(double) * ctx->ncomp, ctx->s_main), "copy");
    if (e.empty()) *loss = hl[comp];
    cleanup();
    return e;
}

// ---------------------------------------------------------------------------
// Near-field use: called by the P2P kernel (lfmm_near.cu) through these
// pointers; see lf_surr_pair_batch there.
// ---------------------------------------------------------------------------
LfErr lf_surrogate_device_view(lfmm_ctx* ctx, LfmmSurrView* v)
{
    v->ready = ctx->surr_ready && ctx->use_surr;
    v->W = ctx->surr_w.ptr;
    v->B = ctx->surr_b.as<float>();
    v->err = ctx->surr_err.as<float>();
    v->meta = ctx->surr_meta.as<LfmmSurrMeta>();
    v->tol = (float)ctx->surr_tol;
    v->counters = ctx->surr_counters.as<unsigned long long>();
    return LfErr();
}
