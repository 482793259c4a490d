// lfmm_surrogate.cuh -- the surrogate network's layout and its warp-level
// inference (shared by the training/validation kernels and the near-field
// P2P kernel).  See lfmm_surrogate.cu for the design.
#pragma once

#include <cuda_bf16.h>

#include "lfmm_internal.cuh"

// parameter vector of one component (float32 master copy)
#define SO_W1 0
#define SO_B1 256
#define SO_W2 320
#define SO_B2 4416
#define SO_W3 4480
#define SO_B3 8576
#define SO_W4 8640
#define SO_B4 8832
// packed inference weights (bfloat16) in mma.sync B-fragment order: one
// fragment (16 k x 8 n) is 32 lanes x 4 values, lane (g, t) holding
// W[n = 8 nt + g][k = 16 ks + 2t, 2t + 1, 2t + 8, 2t + 9]; fragments
// layer 1: nt (K padded 4 -> 16), layer 2: 8 + 4 nt + ks, layer 3: 40 + 4 nt + ks,
// output: 72 + ks (3 outputs padded to 8)
#define SW_F1 0
#define SW_F2 8
#define SW_F3 40
#define SW_F4 72
#define SW_NFRAG 76
#define SW_N (SW_NFRAG * 128)
// float32 biases: b1 [64], b2 [64], b3 [64], b4 [8]
#define SB_N 200
#define TRAIN_B 64  // samples per training block
#define TRAIN_S 65  // padded row stride of the per-sample buffers

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
// inference form: fast division (the result is split to ~16 bits anyway)
__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z)
{
    float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// smallest pair depth h = h_t + h_s the network serves (below it: quadrature)
#define SURR_HMIN 1e-4f

// features of one pair (see the header comment)
__host__ __device__ __forceinline__ void surr_features(const LfmmSurrMeta& m, float rho, float ht, float hs,
                                                       float f[4])
{
    // log10 rho over [-3, log10 3]; the depths over their trained ranges;
    // log10(rho / h) over about [-4.5, 4.5]
    const float r = fmaxf(rho, 1e-3f), h = fmaxf(ht + hs, SURR_HMIN);
    f[0] = (log10f(r) + 1.2614394f) * (1.0f / 1.7385606f);
    f[1] = 2.0f * ht / m.Tt - 1.0f;
    f[2] = 2.0f * hs / m.Ts - 1.0f;
    f[3] = log10f(r / h) * (1.0f / 4.5f);
}

// error-table cell of a pair: log10 rho in [-3, log10 3] by log10 h in
// [-4, log10(T_t + T_s)], LFMM_SURR_CELLS x LFMM_SURR_CELLS
__host__ __device__ __forceinline__ int surr_cell(const LfmmSurrMeta& m, float rho, float h)
{
    const float lh1 = log10f(m.Tt + m.Ts), lh0 = -4.0f;
    float lr = log10f(fmaxf(rho, 1e-3f));
    float lh = log10f(fmaxf(h, SURR_HMIN));
    int ix = (int)((lr + 3.0f) * (LFMM_SURR_CELLS / 3.4771213f));
    int iy = (int)((lh - lh0) * (LFMM_SURR_CELLS / (lh1 - lh0)));
    ix = ix < 0 ? 0 : (ix > LFMM_SURR_CELLS - 1 ? LFMM_SURR_CELLS - 1 : ix);
    iy = iy < 0 ? 0 : (iy > LFMM_SURR_CELLS - 1 ? LFMM_SURR_CELLS - 1 : iy);
    return iy * LFMM_SURR_CELLS + ix;
}

// lead terms and remainder scales of one pair (double)
__device__ __forceinline__ void surr_lead(const LfmmComp& c, double rho, double h, double lead[3], double sc[3])
{
    double H = h + c.zeta;
    double R2 = rho * rho + H * H, R = sqrt(R2);
    lead[0] = c.C / R;
    lead[1] = c.C * H / (R2 * R);
    lead[2] = c.C * rho / (R2 * R);
    double Hr = h + c.zeta_r;
    double Rr = sqrt(rho * rho + Hr * Hr);
    double cr = fabs(c.rem[0]);
    sc[0] = cr / Rr;
    sc[1] = cr / (Rr * Rr);
    sc[2] = sc[1];
}

// magnitude scales of (I_00, I_10 and I_11) of a pair, against which the
// network's error is measured: leading image plus remainder's leading term
__device__ __forceinline__ void surr_err_scale(const LfmmComp& c, double rho, double h, double& s0, double& s1)
{
    double H = h + c.zeta, Hr = h + c.zeta_r;
    double R2 = rho * rho + H * H, Rr2 = rho * rho + Hr * Hr;
    double cr = c.has_rem ? fabs(c.rem[0]) : 0.0;
    s0 = fabs(c.C) / sqrt(R2) + cr / sqrt(Rr2);
    s1 = fabs(c.C) / R2 + cr / Rr2;
}

// ---------------------------------------------------------------------------
// Warp inference with mma.sync m16n8k16 (bf16 x bf16 -> f32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// split two floats into (hi, lo) bfloat16 pairs
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo)
{
    __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
    float r0 = x0 - __bfloat162float(h0), r1 = x1 - __bfloat162float(h1);
    __nv_bfloat162 h;
    h.x = h0;
    h.y = h1;
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = pack_bf16(r0, r1);
}

// B fragment `frag` of this lane
__device__ __forceinline__ uint2 ldfrag(const __nv_bfloat16* W, int frag, int lane)
{
    return __ldg(reinterpret_cast<const uint2*>(W) + frag * 32 + lane);
}

// One warp: standardised outputs y[3] of this lane's pair (features f[4]).
// All 32 lanes must call it.
static __device__ __noinline__ void lf_surr_warp(const __nv_bfloat16* __restrict__ W, const float* __restrict__ B, const float f[4],
                             float y[3])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int mt = 0; mt < 2; ++mt) {
        const int rowA = 16 * mt + g, rowB = rowA + 8;
        // layer 1: input A fragment (only columns 0..3 are non-zero); the
        // shuffled value is the sender's, so all four features travel
        float fa[4], fb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            fa[k] = __shfl_sync(0xffffffffu, f[k], rowA);
            fb[k] = __shfl_sync(0xffffffffu, f[k], rowB);
        }
        uint32_t ahi[4] = {0, 0, 0, 0}, alo[4] = {0, 0, 0, 0};
        if (t == 0) {
            split2(fa[0], fa[1], ahi[0], alo[0]);
            split2(fb[0], fb[1], ahi[1], alo[1]);
        } else if (t == 1) {
            split2(fa[2], fa[3], ahi[0], alo[0]);
            split2(fb[2], fb[3], ahi[1], alo[1]);
        }
        float C[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float b0 = B[nt * 8 + 2 * t], b1 = B[nt * 8 + 2 * t + 1];
            C[nt][0] = b0;
            C[nt][1] = b1;
            C[nt][2] = b0;
            C[nt][3] = b1;
            const uint2 w = ldfrag(W, SW_F1 + nt, lane);
            mma_bf16(C[nt], ahi, w.x, w.y);
            mma_bf16(C[nt], alo, w.x, w.y);
        }
        // hidden layers 2 and 3
        uint32_t Ah[4][4], Al[4][4];
#pragma unroll
        for (int layer = 0; layer < 2; ++layer) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                split2(silu_fast(C[2 * ks][0]), silu_fast(C[2 * ks][1]), Ah[ks][0], Al[ks][0]);
                split2(silu_fast(C[2 * ks][2]), silu_fast(C[2 * ks][3]), Ah[ks][1], Al[ks][1]);
                split2(silu_fast(C[2 * ks + 1][0]), silu_fast(C[2 * ks + 1][1]), Ah[ks][2], Al[ks][2]);
                split2(silu_fast(C[2 * ks + 1][2]), silu_fast(C[2 * ks + 1][3]), Ah[ks][3], Al[ks][3]);
            }
            const int fl = (layer == 0 ? SW_F2 : SW_F3);
            const float* Bl = B + (layer == 0 ? 64 : 128);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                float b0 = Bl[nt * 8 + 2 * t], b1 = Bl[nt * 8 + 2 * t + 1];
                C[nt][0] = b0;
                C[nt][1] = b1;
                C[nt][2] = b0;
                C[nt][3] = b1;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint2 w = ldfrag(W, fl + 4 * nt + ks, lane);
                    mma_bf16(C[nt], Ah[ks], w.x, w.y);
                    mma_bf16(C[nt], Al[ks], w.x, w.y);
                }
            }
        }
        // output layer (3 outputs padded to 8)
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            split2(silu_fast(C[2 * ks][0]), silu_fast(C[2 * ks][1]), Ah[ks][0], Al[ks][0]);
            split2(silu_fast(C[2 * ks][2]), silu_fast(C[2 * ks][3]), Ah[ks][1], Al[ks][1]);
            split2(silu_fast(C[2 * ks + 1][0]), silu_fast(C[2 * ks + 1][1]), Ah[ks][2], Al[ks][2]);
            split2(silu_fast(C[2 * ks + 1][2]), silu_fast(C[2 * ks + 1][3]), Ah[ks][3], Al[ks][3]);
        }
        float O[4];
        {
            float b0 = B[192 + 2 * t], b1 = B[192 + 2 * t + 1];
            O[0] = b0;
            O[1] = b1;
            O[2] = b0;
            O[3] = b1;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint2 w = ldfrag(W, SW_F4 + ks, lane);
                mma_bf16(O, Ah[ks], w.x, w.y);
                mma_bf16(O, Al[ks], w.x, w.y);
            }
        }
        // row r of this m-tile: outputs 0, 1 at thread (r%8, t=0), output 2 at (r%8, t=1)
        const int r = lane - 16 * mt;
        const int src = (r & 7) * 4;
        float v0a = __shfl_sync(0xffffffffu, O[0], src), v0b = __shfl_sync(0xffffffffu, O[2], src);
        float v1a = __shfl_sync(0xffffffffu, O[1], src), v1b = __shfl_sync(0xffffffffu, O[3], src);
        float v2a = __shfl_sync(0xffffffffu, O[0], src + 1), v2b = __shfl_sync(0xffffffffu, O[2], src + 1);
        if (r >= 0 && r < 16) {
            const bool up = r >= 8;
            y[0] = up ? v0b : v0a;
            y[1] = up ? v1b : v1a;
            y[2] = up ? v2b : v2a;
        }
    }
}

// Kernel values from the network for one pair; returns false when the pair
// must fall back to the quadrature (outside the trained range or cell error
// above the tolerance).  `y` are the standardised network outputs.
__device__ __forceinline__ bool lf_surr_cell_ok(const LfmmSurrMeta& m, const float* __restrict__ err, float rho,
                                                float ht, float hs, float tol)
{
    if (!(ht >= 0.f && ht <= m.Tt && hs >= 0.f && hs <= m.Ts)) return false;
    if (!(rho <= 3.0f) || ht + hs < SURR_HMIN) return false;
    return err[surr_cell(m, rho, ht + hs)] <= tol;
}

// kernel values from the standardised network outputs y: leading image plus
// the scaled remainder, in the caller's precision R
template <typename R>
__device__ __forceinline__ void lf_surr_kernels(const LfmmComp& c, const LfmmSurrMeta& m, R rho, R h,
                                                const float y[3], R K[3])
{
    typedef LfMath<R> F;
    R H = h + (R)c.zeta;
    R ir = F::Rsqrt(rho * rho + H * H);
    R ir3 = ir * ir * ir;
    R Hr = h + (R)c.zeta_r;
    R irr = F::Rsqrt(rho * rho + Hr * Hr);
    R cr = (R)fabs(c.rem[0]);
    R s0 = cr * irr, s1 = s0 * irr;
    K[0] = (R)c.C * ir + s0 * ((R)m.mu[0] + (R)m.sd[0] * (R)y[0]);
    K[1] = (R)c.C * H * ir3 + s1 * ((R)m.mu[1] + (R)m.sd[1] * (R)y[1]);
    K[2] = (R)c.C * rho * ir3 + s1 * ((R)m.mu[2] + (R)m.sd[2] * (R)y[2]);
}
