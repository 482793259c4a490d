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

#include <algorithm>
#include <cmath>

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
    const void* q;    // charges [nr][qstride]
    double* phi;      // [nr][qstride]
    double* fld;      // [nr][qstride][3]
    int64_t qstride;  // charges per right-hand side (n)
    int nr;           // right-hand sides of this launch (<= the kernel's batch)
    int split;        // near list of a leaf shared by this many warps / blocks (1: whole list, stored;
                      // > 1: interleaved entries, partial sums added atomically into zeroed outputs)
    int Qn;
    const LfmmComp* comps;  // the context's components
    const double* gl_t;     // near-field quadrature rule (Qn nodes and weights)
    const double* gl_w;
    const double* ntab;  // remainder tables [component][LF_NT_PER], or null: the quadrature
    const float4* ntab4;  // their float32 copy [component][w][s] {T00, T10, T11, 0} for the float32 kernels
    LfmmSurrView sv;  // learned near-field kernels (sv.ready = 0: quadrature only)
    // float32 warp kernel on a leaf level whose polarization images are grid
    // cells: box grid cells and per component (s, K, is_free) in leaf units,
    // so that every centre offset is an exact small integer times hleaf (null:
    // offsets from the FP64 centres)
    const int4* grid;
    const float4* pcon;
    float hleaf;
};
#define LF_CTAB(a, c) ((a).ntab ? (a).ntab + (size_t)(c) * LF_NT_PER : nullptr)
#define LF_CTAB4(a, c) ((a).ntab4 ? (a).ntab4 + (size_t)(c) * LF_NT_NS * LF_NT_NW : nullptr)

#define P2P_T 128

// Sums of one target over a batch of RB right-hand sides: compensated
// (LfSum) across source boxes, plain (LfPlain) within one source box.
template <typename R>
struct LfPlain {
    R s = 0;
    __device__ __forceinline__ void add(R x) { s += x; }
};
template <typename S, int RB>
struct P2PAccT {
    S P[RB], Ex[RB], Ey[RB], Ez[RB];
};
template <typename R, int RB>
using P2PAcc = P2PAccT<LfSum<R>, RB>;
template <typename R, int RB>
using P2PPart = P2PAccT<LfPlain<R>, RB>;

// add one source box's partial sums into the compensated totals and clear them
template <typename R, int RB>
__device__ __forceinline__ void p2p_flush(P2PPart<R, RB>& part, P2PAcc<R, RB>& A)
{
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        A.P[k].add(part.P[k].s);
        A.Ex[k].add(part.Ex[k].s);
        A.Ey[k].add(part.Ey[k].s);
        A.Ez[k].add(part.Ez[k].s);
        part.P[k].s = part.Ex[k].s = part.Ey[k].s = part.Ez[k].s = R(0);
    }
}

// Free-space kernel of one pair, applied to the nr charges qs[k * qsk] of the batch.
template <typename R, int RB, typename S>
__device__ __forceinline__ void p2p_free_add(R dx, R dy, R dz, const R* qs, int qsk, int nr, P2PAccT<S, RB>& A)
{
    typedef LfMath<R> F;
    R r2 = dx * dx + dy * dy + dz * dz;
    if (r2 > R(0)) {
        R ir = F::Rsqrt(r2);
        R ir3 = ir * ir * ir;
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            if (k >= nr) break;
            const R q = qs[k * qsk];
            const R q3 = q * ir3;
            A.P[k].add(q * ir);
            A.Ex[k].add(q3 * dx);
            A.Ey[k].add(q3 * dy);
            A.Ez[k].add(q3 * dz);
        }
    }
}

// Reaction kernels of one pair by the quadrature, or by the component's
// remainder table ctab where given (once), applied to the batch.
template <typename R, int RB, bool GEN = false, typename S>
__device__ __forceinline__ void p2p_reaction_add(const LfmmComp& cp, R dx, R dy, R dz, const R* qs, int qsk, int nr,
                                                 int Qn, const double* gl_t, const double* gl_w, P2PAccT<S, RB>& A,
                                                 const double* ctab, const float4* ctab4 = nullptr)
{
    typedef LfMath<R> F;
    R h = (cp.a == 1) ? dz : -dz;
    R rho = F::Sqrt(dx * dx + dy * dy);
    R k00, k10, k11;
    lf_reaction_pair<R, GEN>(cp, rho, h, Qn, gl_t, gl_w, k00, k10, k11, ctab, ctab4);
    const R k10s = (cp.a == 1) ? k10 : -k10;
    const R g = rho > R(0) ? k11 / rho : R(0);
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (k >= nr) break;
        const R q = qs[k * qsk];
        A.P[k].add(q * k00);
        A.Ez[k].add(q * k10s);
        if (rho > R(0)) {
            A.Ex[k].add(q * g * dx);
            A.Ey[k].add(q * g * dy);
        }
    }
}

template <typename R, int RB>
__device__ __forceinline__ void p2p_store(const P2PArgs& a, int i, const P2PAcc<R, RB>& A)
{
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (k >= a.nr) break;
        const size_t o = (size_t)k * a.qstride + i;
        if (a.split > 1) {
            atomicAdd(a.phi + o, (double)A.P[k].s);
            atomicAdd(a.fld + 3 * o + 0, (double)A.Ex[k].s);
            atomicAdd(a.fld + 3 * o + 1, (double)A.Ey[k].s);
            atomicAdd(a.fld + 3 * o + 2, (double)A.Ez[k].s);
        } else {
            a.phi[o] = (double)A.P[k].s;
            a.fld[3 * o + 0] = (double)A.Ex[k].s;
            a.fld[3 * o + 1] = (double)A.Ey[k].s;
            a.fld[3 * o + 2] = (double)A.Ez[k].s;
        }
    }
}

// One block per target leaf (FP64 form), a batch of RB right-hand sides.
// GEN: media of four or five layers (both forms, one right-hand side per launch).
template <typename R, int RB, bool GEN = false>
__global__ void __launch_bounds__(P2P_T) k_p2p(P2PArgs a)
{
    __shared__ R sx[P2P_T], sy[P2P_T], sz[P2P_T], sq[RB][P2P_T];
    const R* q = reinterpret_cast<const R*>(a.q);
    const int t = a.leaf_off + (int)blockIdx.x / a.split;
    const int part0 = (int)blockIdx.x % a.split;
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
        P2PAcc<R, RB> A;
        for (int e = a.nbeg[t] + part0; e < a.nend[t]; e += a.split) {
            const uint32_t ent = a.nent[e];
            const int c = (int)(ent >> LFMM_ENT_SHIFT);
            const int s = (int)(ent & LFMM_ENT_MASK);
            const LfmmComp& cp = a.comps[c];
            const int sb = a.pbeg[s], se = a.pend[s];
            for (int cb = sb; cb < se; cb += P2P_T) {
                const int j = cb + tid;
                __syncthreads();
                if (j < se) {
                    sx[tid] = (R)(a.xs[j] - ct.x);
                    sy[tid] = (R)(a.ys[j] - ct.y);
                    double zj = cp.is_free ? a.zs[j] : cp.s * a.zs[j] + cp.o;
                    sz[tid] = (R)(zj - ct.z);
#pragma unroll
                    for (int k = 0; k < RB; ++k)
                        if (k < a.nr) sq[k][tid] = q[(size_t)k * a.qstride + j];
                }
                __syncthreads();
                if (!valid) continue;
                const int cnt = min(P2P_T, se - cb);
                if (cp.is_free) {
                    for (int u = 0; u < cnt; ++u)
                        p2p_free_add<R, RB>(xi - sx[u], yi - sy[u], zi - sz[u], &sq[0][u], P2P_T, a.nr, A);
                } else {
                    for (int u = 0; u < cnt; ++u)
                        p2p_reaction_add<R, RB, GEN>(cp, xi - sx[u], yi - sy[u], zi - sz[u], &sq[0][u], P2P_T,
                                                     a.nr, a.Qn, a.gl_t, a.gl_w, A, LF_CTAB(a, c),
                                                     sizeof(R) == 4 ? LF_CTAB4(a, c) : nullptr);
                }
            }
        }
        if (valid) p2p_store<R, RB>(a, i, A);
    }
}

// Float32 near field: one warp per target leaf (leaves hold ~20 charges, so a
// warp is the natural unit), no block-wide barriers.  Positions come as
// float offsets from each particle's own leaf centre (computed once per
// build); the offset between two box centres (or a source box's
// polarization image and the target box) is formed in double once per warp
// and entry, so no double arithmetic remains per particle or pair.
#define PW_WARPS 4

__global__ void k_rel_pos(int leaf_off, int nleaf, const LfD4* __restrict__ cen, const int* __restrict__ pbeg,
                          const int* __restrict__ pend, const double* __restrict__ xs, const double* __restrict__ ys,
                          const double* __restrict__ zs, float4* __restrict__ rel, int* __restrict__ leaf_of)
{
    const int li = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (li >= nleaf) return;
    const int b = leaf_off + li;
    const LfD4 c = cen[b];
    for (int i = pbeg[b] + lane; i < pend[b]; i += 32) {
        rel[i] = make_float4((float)(xs[i] - c.x), (float)(ys[i] - c.y), (float)(zs[i] - c.z), 0.f);
        leaf_of[i] = b;
    }
}

// A leaf of at most 16 (8) charges gives each target 2 (4) lanes, each
// taking a contiguous part of every staged source box; their sums meet by
// shuffles at the end.
template <int RB>
__global__ void __launch_bounds__(32 * PW_WARPS) k_p2p_warp(P2PArgs a, const float4* __restrict__ rel, int nleaf)
{
    // one charge vector: sources staged as (x, y, z, q), one 16-byte shared load per pair
    constexpr bool ONE = (RB == 1);
    __shared__ float sx[PW_WARPS][ONE ? 1 : 32], sy[PW_WARPS][ONE ? 1 : 32], sz[PW_WARPS][ONE ? 1 : 32],
        sq[PW_WARPS][RB][ONE ? 1 : 32];
    __shared__ float4 sp[PW_WARPS][ONE ? 32 : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int wi = blockIdx.x * PW_WARPS + w;
    if (wi >= nleaf * a.split) return;  // whole warp
    const int li = wi / a.split, part0 = wi - li * a.split;
    const float* q = reinterpret_cast<const float*>(a.q);
    const int t = a.leaf_off + li;
    const LfD4 ct = a.grid ? LfD4{0.0, 0.0, 0.0, 0.0} : a.cen[t];
    const int4 gt = a.grid ? a.grid[t] : make_int4(0, 0, 0, 0);
    const int tb = a.pbeg[t], te = a.pend[t];
    const int eb = a.nbeg[t], ee = a.nend[t];
    const int nt = te - tb;
    const int G = nt <= 8 ? 4 : (nt <= 16 ? 2 : 1);  // lanes per target (warp-uniform)
    const int T = 32 / G;                             // targets per pass
    const int ti = lane % T, slice = lane / T;
    for (int base = tb; base < te; base += T) {
        const int i = base + ti;
        const bool valid = i < te;
        float xi = 0.f, yi = 0.f, zi = 0.f;
        if (valid) {
            const float4 r = rel[i];
            xi = r.x;
            yi = r.y;
            zi = r.z;
        }
        P2PAcc<float, RB> A;
        P2PPart<float, RB> part;
        for (int e = eb + part0; e < ee; e += a.split) {
            const uint32_t ent = a.nent[e];
            const int c = (int)(ent >> LFMM_ENT_SHIFT);
            const int s = (int)(ent & LFMM_ENT_MASK);
            const LfmmComp& cp = a.comps[c];
            // source box centre (free) or its polarization image (reaction), relative to the target box
            float dx0, dy0, dz0, szs;
            if (a.grid) {
                // (z_t - z'') / h = (iz_t + 1/2) - s (iz_s + 1/2) - K with K an integer on this level
                const int4 gs = a.grid[s];
                const float4 pc = a.pcon[c];
                szs = pc.x;
                dx0 = (float)(gs.x - gt.x) * a.hleaf;
                dy0 = (float)(gs.y - gt.y) * a.hleaf;
                dz0 = (pc.x * ((float)gs.z + 0.5f) - ((float)gt.z + 0.5f) + pc.y) * a.hleaf;
            } else {
                const LfD4 cs = a.cen[s];
                dx0 = (float)(cs.x - ct.x);
                dy0 = (float)(cs.y - ct.y);
                dz0 = (float)(cp.is_free ? cs.z - ct.z : cp.s * cs.z + cp.o - ct.z);
                szs = cp.is_free ? 1.f : (float)cp.s;
            }
            const int sb = a.pbeg[s], se = a.pend[s];
            for (int cb = sb; cb < se; cb += 32) {
                const int j = cb + lane;
                __syncwarp();
                if (j < se) {
                    const float4 r = rel[j];
                    if constexpr (ONE) {
                        sp[w][lane] = make_float4(r.x + dx0, r.y + dy0, szs * r.z + dz0, q[j]);
                    } else {
                        sx[w][lane] = r.x + dx0;
                        sy[w][lane] = r.y + dy0;
                        sz[w][lane] = szs * r.z + dz0;
#pragma unroll
                        for (int k = 0; k < RB; ++k)
                            if (k < a.nr) sq[w][k][lane] = q[(size_t)k * a.qstride + j];
                    }
                }
                __syncwarp();
                if (!valid) continue;
                const int cnt = min(32, se - cb);
                // this lane's contiguous share of the staged sources
                const int u0 = (slice * cnt) / G, u1 = ((slice + 1) * cnt) / G;
                if constexpr (ONE) {
                    if (cp.is_free) {
                        float& P = part.P[0].s;
                        float& Ex = part.Ex[0].s;
                        float& Ey = part.Ey[0].s;
                        float& Ez = part.Ez[0].s;
#pragma unroll 4
                        for (int u = u0; u < u1; ++u) {
                            const float4 v = sp[w][u];
                            const float dx = xi - v.x, dy = yi - v.y, dz = zi - v.z;
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            const float ir = (r2 > 0.f) ? rsqrtf(r2) : 0.f;  // the target itself: no term
                            const float q3 = v.w * ir * ir * ir;
                            P += v.w * ir;
                            Ex += q3 * dx;
                            Ey += q3 * dy;
                            Ez += q3 * dz;
                        }
                    } else {
                        for (int u = u0; u < u1; ++u) {
                            const float4 v = sp[w][u];
                            p2p_reaction_add<float, 1>(cp, xi - v.x, yi - v.y, zi - v.z, &sp[w][u].w, 0, 1, a.Qn,
                                                       a.gl_t, a.gl_w, part, LF_CTAB(a, c), LF_CTAB4(a, c));
                        }
                    }
                    continue;
                }
                if (cp.is_free) {
                    for (int u = u0; u < u1; ++u)
                        p2p_free_add<float, RB>(xi - sx[w][u], yi - sy[w][u], zi - sz[w][u], &sq[w][0][u], 32, a.nr,
                                                part);
                } else {
                    for (int u = u0; u < u1; ++u)
                        p2p_reaction_add<float, RB>(cp, xi - sx[w][u], yi - sy[w][u], zi - sz[w][u], &sq[w][0][u],
                                                    32, a.nr, a.Qn, a.gl_t, a.gl_w, part, LF_CTAB(a, c),
                                                    LF_CTAB4(a, c));
                }
            }
            p2p_flush<float, RB>(part, A);
        }
        if (G > 1) {
            // the lanes of one target meet (every lane takes part in the shuffles)
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                float v0 = A.P[k].s - A.P[k].c, v1 = A.Ex[k].s - A.Ex[k].c;
                float v2 = A.Ey[k].s - A.Ey[k].c, v3 = A.Ez[k].s - A.Ez[k].c;
                for (int off = T; off < 32; off <<= 1) {
                    v0 += __shfl_xor_sync(0xffffffffu, v0, off);
                    v1 += __shfl_xor_sync(0xffffffffu, v1, off);
                    v2 += __shfl_xor_sync(0xffffffffu, v2, off);
                    v3 += __shfl_xor_sync(0xffffffffu, v3, off);
                }
                A.P[k].s = v0;
                A.Ex[k].s = v1;
                A.Ey[k].s = v2;
                A.Ez[k].s = v3;
            }
        }
        if (valid && slice == 0) p2p_store<float, RB>(a, i, A);
    }
}

// Float32 free-space near field, one charge vector, when no near list holds
// a reaction entry (the benchmark-size trees): one warp per target leaf, as
// k_p2p_warp, but the warp first stages its whole near list in shared memory
// (as float offsets from the target leaf centre, with the charge), the
// leaf's own box first, and then runs one tight loop over the staged sources
// for each pass of targets.  Only the leaf's own box can hold the target
// itself, so only its pairs keep the r > 0 test.  Lists of more than PF_CAP
// sources are staged in rounds of whole boxes (a box larger than PF_CAP in
// pieces).  Partial sums are compensated every 32 sources.  Box centre
// offsets come from the integer grid cells (leaf levels whose images are
// grid cells; this kernel serves free-space entries only).
#define PF_WARPS 4
#define PF_CAP 512
#define PF_UNR 2  // staging loads in flight per lane

struct PfCursor {
    int k;    // next entry of this warp (index into its strided subsequence), -1: the own box
    int off;  // sources of that box already staged
};

// Stage sources from the cursor on, whole boxes while they fit (a box larger
// than the capacity in pieces).  Returns the staged count; *nself is the
// number of own-box sources at the front; *more is set if sources remain.
__device__ __noinline__ int pf_fill(const P2PArgs& a, const float4* __restrict__ rel, const float* __restrict__ q,
                                       float4* S, int t, int4 gt, int tb, int te, int eb, int nmine, int part0,
                                       PfCursor& cur, int& nself, bool& more, int lane)
{
    int fill = 0;
    nself = 0;
    if (cur.k < 0) {  // the own box (zero centre offset)
        const int n = min(te - tb - cur.off, PF_CAP);
        for (int u = lane; u < n; u += 32) {
            const int j = tb + cur.off + u;
            const float4 r = rel[j];
            S[u] = make_float4(r.x, r.y, r.z, q[j]);
        }
        fill = nself = n;
        cur.off += n;
        if (tb + cur.off >= te) {
            cur.k = 0;
            cur.off = 0;
        }
    }
    // the other boxes, up to 32 entries at a time: lane j reads entry cur.k + j
    // (all metadata loads in flight at once), a warp scan places the boxes,
    // and a flattened copy fills the staging area
    while (cur.k >= 0 && cur.k < nmine && fill < PF_CAP) {
        const int j = cur.k + lane;
        int b0 = 0, n = 0;
        float dx0 = 0.f, dy0 = 0.f, dz0 = 0.f;
        if (j < nmine) {
            const uint32_t ent = a.nent[eb + part0 + j * a.split];
            const int sb = (int)(ent & LFMM_ENT_MASK);
            if (sb != t) {  // the own box: staged by the part-0 warp at the front
                b0 = a.pbeg[sb];
                n = a.pend[sb] - b0;
                const int4 gs = a.grid[sb];
                dx0 = (float)(gs.x - gt.x) * a.hleaf;
                dy0 = (float)(gs.y - gt.y) * a.hleaf;
                dz0 = (float)(gs.z - gt.z) * a.hleaf;
            }
            if (lane == 0) {  // a box begun in the previous round
                b0 += cur.off;
                n -= cur.off;
            }
        }
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int excl = incl - n;
        const int room = PF_CAP - fill;
        // entries that fit whole (incl is non-decreasing over the lanes)
        const int m = min(__popc(__ballot_sync(0xffffffffu, incl <= room)), nmine - cur.k);
        if (m == 0) {
            // the first box alone overflows: next round, or a piece of it
            if (fill > 0) break;
            const int n0 = __shfl_sync(0xffffffffu, n, 0), b00 = __shfl_sync(0xffffffffu, b0, 0);
            const float x0 = __shfl_sync(0xffffffffu, dx0, 0), y0 = __shfl_sync(0xffffffffu, dy0, 0),
                        z0 = __shfl_sync(0xffffffffu, dz0, 0);
            const int take = min(n0, room);
            for (int u = lane; u < take; u += 32) {
                const float4 r = rel[b00 + u];
                S[u] = make_float4(r.x + x0, r.y + y0, r.z + z0, q[b00 + u]);
            }
            fill = take;
            cur.off += take;
            break;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, m - 1);
        // slot u of [0, tot) belongs to the entry e with excl_e <= u < incl_e
        for (int base = 0; base < tot; base += 32 * PF_UNR) {
            int src[PF_UNR];
            float ox[PF_UNR], oy[PF_UNR], oz[PF_UNR];
#pragma unroll
            for (int h = 0; h < PF_UNR; ++h) {
                const int u = base + 32 * h + lane;
                int lo = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int c = lo + step;
                    const int ex = __shfl_sync(0xffffffffu, excl, c & 31);
                    if (c < m && ex <= u) lo = c;
                }
                src[h] = __shfl_sync(0xffffffffu, b0, lo) + (u - __shfl_sync(0xffffffffu, excl, lo));
                ox[h] = __shfl_sync(0xffffffffu, dx0, lo);
                oy[h] = __shfl_sync(0xffffffffu, dy0, lo);
                oz[h] = __shfl_sync(0xffffffffu, dz0, lo);
                if (u >= tot) src[h] = -1;
            }
            float4 r[PF_UNR];
            float qq[PF_UNR];
#pragma unroll
            for (int h = 0; h < PF_UNR; ++h)
                if (src[h] >= 0) {
                    r[h] = rel[src[h]];
                    qq[h] = q[src[h]];
                }
#pragma unroll
            for (int h = 0; h < PF_UNR; ++h)
                if (src[h] >= 0)
                    S[fill + base + 32 * h + lane] = make_float4(r[h].x + ox[h], r[h].y + oy[h], r[h].z + oz[h], qq[h]);
        }
        fill += tot;
        cur.k += m;
        cur.off = 0;
    }
    more = (cur.k < 0) || (cur.k < nmine);
    return fill;
}

// pairs of this lane's R targets with staged sources [u0, u1), compensated
// every 32 sources; each staged source is read once for all R targets
template <bool SELF, int R>
__device__ __forceinline__ void pf_pairs(const float4* S, int u0, int u1, const float* xi, const float* yi,
                                         const float* zi, P2PAcc<float, R>& A)
{
    for (int c0 = u0; c0 < u1; c0 += 32) {
        const int c1 = min(c0 + 32, u1);
        P2PPart<float, R> part;
#pragma unroll
        for (int r = 0; r < R; ++r) part.P[r].s = part.Ex[r].s = part.Ey[r].s = part.Ez[r].s = 0.f;
#pragma unroll 2
        for (int u = c0; u < c1; ++u) {
            const float4 v = S[u];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float dx = xi[r] - v.x, dy = yi[r] - v.y, dz = zi[r] - v.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                float ir = rsqrtf(r2);
                if (SELF) ir = (r2 > 0.f) ? ir : 0.f;  // the target itself: no term
                const float qi = v.w * ir;
                const float q3 = qi * ir * ir;
                part.P[r].s += qi;
                part.Ex[r].s += q3 * dx;
                part.Ey[r].s += q3 * dy;
                part.Ez[r].s += q3 * dz;
            }
        }
        p2p_flush<float, R>(part, A);
    }
}

// One pass over targets base + ti + G r (r < R) of the leaf [tb, te): the
// lane's slice of the staged near list (restaged in rounds when it did not
// fit), the slices of a target slot summed by shuffles, stored by slice 0.
template <int R>
__device__ __forceinline__ void pf_pass(const P2PArgs& a, const float4* __restrict__ rel, const float* __restrict__ q,
                                        float4* S, int t, int4 gt, int tb, int te, int eb, int nmine, int part0,
                                        int base, int lg, int lane, bool once, bool first, PfCursor start,
                                        PfCursor& cur, int& fill, int& nself, bool& more)
{
    const int G = 32 >> lg;
    const int ti = lane & (G - 1), slice = lane >> (5 - lg);
    float xi[R], yi[R], zi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = base + ti + G * r;
        xi[r] = yi[r] = zi[r] = 0.f;
        if (i < te) {
            const float4 v = rel[i];
            xi[r] = v.x;
            yi[r] = v.y;
            zi[r] = v.z;
        }
    }
    P2PAcc<float, R> A;
    if (!once && !first) {  // stage the first round again
        cur = start;
        __syncwarp();
        fill = pf_fill(a, rel, q, S, t, gt, tb, te, eb, nmine, part0, cur, nself, more, lane);
        __syncwarp();
    }
    for (;;) {
        // this lane's contiguous share of the own-box part and of the rest
        const int a0 = (slice * nself) >> lg, a1 = ((slice + 1) * nself) >> lg;
        const int nr = fill - nself;
        const int b0 = nself + ((slice * nr) >> lg), b1 = nself + (((slice + 1) * nr) >> lg);
        pf_pairs<true, R>(S, a0, a1, xi, yi, zi, A);
        pf_pairs<false, R>(S, b0, b1, xi, yi, zi, A);
        if (once || !more) break;
        __syncwarp();
        fill = pf_fill(a, rel, q, S, t, gt, tb, te, eb, nmine, part0, cur, nself, more, lane);
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        // the slices of one target slot meet (every lane takes part in the shuffles)
        float v0 = A.P[r].s - A.P[r].c, v1 = A.Ex[r].s - A.Ex[r].c;
        float v2 = A.Ey[r].s - A.Ey[r].c, v3 = A.Ez[r].s - A.Ez[r].c;
        for (int off = G; off < 32; off <<= 1) {
            v0 += __shfl_xor_sync(0xffffffffu, v0, off);
            v1 += __shfl_xor_sync(0xffffffffu, v1, off);
            v2 += __shfl_xor_sync(0xffffffffu, v2, off);
            v3 += __shfl_xor_sync(0xffffffffu, v3, off);
        }
        const int i = base + ti + G * r;
        if (slice == 0 && i < te) {
            if (a.split > 1) {
                atomicAdd(a.phi + i, (double)v0);
                atomicAdd(a.fld + 3 * (size_t)i + 0, (double)v1);
                atomicAdd(a.fld + 3 * (size_t)i + 1, (double)v2);
                atomicAdd(a.fld + 3 * (size_t)i + 2, (double)v3);
            } else {
                a.phi[i] = (double)v0;
                a.fld[3 * (size_t)i + 0] = (double)v1;
                a.fld[3 * (size_t)i + 1] = (double)v2;
                a.fld[3 * (size_t)i + 2] = (double)v3;
            }
        }
    }
}

// Lanes as G = 32 / 2^lg target slots times 2^lg source slices, each lane
// holding R <= PF_R targets: per staged source a lane spends one shared load
// and R pair evaluations, so the choice minimises (1 load + R pairs) / 2^lg
// over the layouts that cover the leaf's nt targets in one pass (about 3 and
// 15 issue slots; leaves of more than 32 PF_R charges take passes of 32 PF_R).
#define PF_R 3
__device__ __forceinline__ void pf_layout(int nt, int& lg, int& R)
{
    lg = 0;
    R = PF_R;
    if (nt > 32 * PF_R) return;
    int best = 1 << 30;
    for (int l = 0; l <= 5; ++l) {
        const int g = 32 >> l, r = (nt + g - 1) / g;
        if (r > PF_R) continue;
        const int cost = (3 + 15 * r) << (5 - l);
        if (cost < best) {
            best = cost;
            lg = l;
            R = r;
        }
    }
}

__global__ void __launch_bounds__(32 * PF_WARPS, 4) k_p2p_free_staged(P2PArgs a, const float4* __restrict__ rel,
                                                                    int nleaf)
{
    __shared__ float4 sp[PF_WARPS][PF_CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int wi = blockIdx.x * PF_WARPS + w;
    if (wi >= nleaf * a.split) return;  // whole warp
    const int li = wi / a.split, part0 = wi - li * a.split;
    const float* q = reinterpret_cast<const float*>(a.q);
    float4* S = sp[w];
    const int t = a.leaf_off + li;
    const int4 gt = a.grid[t];
    const int tb = a.pbeg[t], te = a.pend[t];
    const int eb = a.nbeg[t], ee = a.nend[t];
    const int nmine = (ee - eb > part0) ? (ee - eb - part0 + a.split - 1) / a.split : 0;
    int lg, R;  // warp-uniform
    pf_layout(te - tb, lg, R);
    const int per = (32 >> lg) * R;  // targets per pass
    const PfCursor start{part0 == 0 ? -1 : 0, 0};
    // the first round stages everything when the list fits: later passes reuse it
    PfCursor cur = start;
    int nself = 0;
    bool more = false;
    int fill = pf_fill(a, rel, q, S, t, gt, tb, te, eb, nmine, part0, cur, nself, more, lane);
    const bool once = !more;
    __syncwarp();
    for (int base = tb; base < te; base += per) {
        const bool first = base == tb;
#define PF_PASS(RR) \
    pf_pass<RR>(a, rel, q, S, t, gt, tb, te, eb, nmine, part0, base, lg, lane, once, first, start, cur, fill, nself, more)
        if (R == 1) PF_PASS(1);
#if PF_R >= 2
        else if (R == 2) PF_PASS(2);
#endif
#if PF_R >= 3
        else if (R == 3) PF_PASS(3);
#endif
#if PF_R >= 4
        else PF_PASS(4);
#endif
#undef PF_PASS
    }
}

LfErr lf_near_prepare(lfmm_ctx* ctx, cudaStream_t st)
{
    const LfmmLevel& leaf = ctx->levels[ctx->depth];
    LF_TRY(lf_reserve(ctx->pos_rel, (size_t)ctx->n * sizeof(float4) + 16));
    LF_TRY(lf_reserve(ctx->leaf_of, (size_t)ctx->n * sizeof(int) + 16));
    if (leaf.nbox > 0)
        ++ctx->launches, k_rel_pos<<<lf_blocks(leaf.nbox, 4), 128, 0, st>>>(
            leaf.off, leaf.nbox, ctx->box_center.as<LfD4>(), ctx->box_pbeg.as<int>(), ctx->box_pend.as<int>(),
            ctx->xs.as<double>(), ctx->ys.as<double>(), ctx->zs.as<double>(), ctx->pos_rel.as<float4>(),
            ctx->leaf_of.as<int>());
    return lf_cuda(cudaGetLastError(), "relative positions");
}

// Near field with the learned reaction kernels.  For a trained component each
// warp first looks its 32 pairs (one source against the warp's 32 targets) up
// in the error table; if any lane accepts, the warp evaluates the network for
// all 32 (tensor-core MMAs need the whole warp).  Rejected pairs are not
// integrated in place (that would stall the warp on the slowest lane):
// they go to a per-warp queue of (target lane, source) entries that is drained
// 32 at a time, one pair per lane, the results added into per-target
// shared-memory accumulators.
#define P2P_W (P2P_T / 32)
#define P2P_QCAP 64

template <typename R>
__device__ __forceinline__ void p2p_drain(const LfmmComp& cp, const uint16_t* qe, int count, int lane, int wbase,
                                          const R* tx, const R* ty, const R* tz, const R* sx, const R* sy,
                                          const R* sz, const R* sq, R (*acc)[4], int Qn, const double* gl_t,
                                          const double* gl_w, const double* ctab)
{
    typedef LfMath<R> F;
    if (lane >= count) return;
    const int ent = qe[lane];
    const int o = wbase + (ent >> 7), u = ent & 127;
    R dx = tx[o] - sx[u], dy = ty[o] - sy[u], dz = tz[o] - sz[u];
    R h = (cp.a == 1) ? dz : -dz;
    R rho = F::Sqrt(dx * dx + dy * dy);
    R k00, k10, k11;
    lf_reaction_pair<R>(cp, rho, h, Qn, gl_t, gl_w, k00, k10, k11, ctab);
    R qs = sq[u];
    atomicAdd(&acc[o][0], qs * k00);
    atomicAdd(&acc[o][3], (cp.a == 1) ? qs * k10 : -qs * k10);
    if (rho > R(0)) {
        R g = qs * k11 / rho;
        atomicAdd(&acc[o][1], g * dx);
        atomicAdd(&acc[o][2], g * dy);
    }
}

template <typename R>
__global__ void __launch_bounds__(P2P_T) k_p2p_net(P2PArgs a)
{
    typedef LfMath<R> F;
    __shared__ R sx[P2P_T], sy[P2P_T], sz[P2P_T], sq[P2P_T];
    __shared__ R tx[P2P_T], ty[P2P_T], tz[P2P_T];
    __shared__ R acc[P2P_T][4];  // deferred (phi, Ex, Ey, Ez) per target
    __shared__ uint16_t qbuf[P2P_W][P2P_QCAP];
    const R* q = reinterpret_cast<const R*>(a.q);
    const int t = a.leaf_off + (int)blockIdx.x / a.split;
    const int part0 = (int)blockIdx.x % a.split;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, wbase = tid & ~31;
    const LfD4 ct = a.cen[t];
    const int tb = a.pbeg[t], te = a.pend[t];
    unsigned long long n_net = 0, n_quad = 0;
    for (int base = tb; base < te; base += P2P_T) {
        const int i = base + tid;
        const bool valid = i < te;
        R xi = 0, yi = 0, zi = 0;
        if (valid) {
            xi = (R)(a.xs[i] - ct.x);
            yi = (R)(a.ys[i] - ct.y);
            zi = (R)(a.zs[i] - ct.z);
        }
        tx[tid] = xi;
        ty[tid] = yi;
        tz[tid] = zi;
        acc[tid][0] = acc[tid][1] = acc[tid][2] = acc[tid][3] = R(0);
        __syncwarp();
        P2PAcc<R, 1> A;
        LfSum<R>&P = A.P[0], &Ex = A.Ex[0], &Ey = A.Ey[0], &Ez = A.Ez[0];
        for (int e = a.nbeg[t] + part0; e < a.nend[t]; e += a.split) {
            const uint32_t ent = a.nent[e];
            const int c = (int)(ent >> LFMM_ENT_SHIFT);
            const int s = (int)(ent & LFMM_ENT_MASK);
            const LfmmComp& cp = a.comps[c];
            const int sb = a.pbeg[s], se = a.pend[s];
            const bool use_net = !cp.is_free && a.sv.meta[c].trained;
            LfmmSurrMeta sm;
            const __nv_bfloat16* sW = nullptr;
            const float *sB = nullptr, *serr = nullptr;
            float ht = 0.f;
            if (use_net) {
                sm = a.sv.meta[c];
                sW = reinterpret_cast<const __nv_bfloat16*>(a.sv.W) + (size_t)c * SW_N;
                sB = a.sv.B + (size_t)c * SB_N;
                serr = a.sv.err + (size_t)c * LFMM_SURR_CELLS * LFMM_SURR_CELLS;
                // depth of the target below (a = 1) or above (a = 2) its interface
                const double zt = valid ? a.zs[i] : ct.z;
                ht = (float)((cp.a == 1) ? zt - cp.iface : cp.iface - zt);
            }
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
                const int cnt = min(P2P_T, se - cb);
                if (!use_net) {
                    if (!valid) continue;
                    if (cp.is_free) {
                        for (int u = 0; u < cnt; ++u)
                            p2p_free_add<R, 1>(xi - sx[u], yi - sy[u], zi - sz[u], &sq[u], 0, 1, A);
                    } else {
                        for (int u = 0; u < cnt; ++u)
                            p2p_reaction_add<R, 1>(cp, xi - sx[u], yi - sy[u], zi - sz[u], &sq[u], 0, 1, a.Qn, a.gl_t, a.gl_w, A, LF_CTAB(a, c));
                        n_quad += cnt;
                    }
                    continue;
                }
                // every lane of the warp runs this loop (valid or not)
                int qn = 0;
                for (int u = 0; u < cnt; ++u) {
                    R dx = xi - sx[u], dy = yi - sy[u], dz = zi - sz[u];
                    R h = (cp.a == 1) ? dz : -dz;
                    R rho = F::Sqrt(dx * dx + dy * dy);
                    const float hs = (float)h - ht;
                    const bool net = valid && lf_surr_cell_ok(sm, serr, (float)rho, ht, hs, a.sv.tol);
                    if (__any_sync(0xffffffffu, net)) {
                        float f[4], y[3];
                        surr_features(sm, (float)rho, ht, hs, f);
                        __syncwarp();
                        lf_surr_warp(sW, sB, f, y);
                        if (net) {
                            R K[3];
                            lf_surr_kernels<R>(cp, sm, rho, h, y, K);
                            R qs = sq[u];
                            P.add(qs * K[0]);
                            Ez.add((cp.a == 1) ? qs * K[1] : -qs * K[1]);
                            if (rho > R(0)) {
                                R g = qs * K[2] / rho;
                                Ex.add(g * dx);
                                Ey.add(g * dy);
                            }
                            ++n_net;
                        }
                    }
                    const bool rej = valid && !net;
                    n_quad += rej;
                    const unsigned m = __ballot_sync(0xffffffffu, rej);
                    if (m) {
                        if (rej) qbuf[wid][qn + __popc(m & ((1u << lane) - 1u))] = (uint16_t)((lane << 7) | u);
                        qn += __popc(m);
                        if (qn >= 32) {
                            __syncwarp();
                            qn -= 32;
                            p2p_drain<R>(cp, &qbuf[wid][qn], 32, lane, wbase, tx, ty, tz, sx, sy, sz, sq, acc, a.Qn, a.gl_t, a.gl_w, LF_CTAB(a, c));
                            __syncwarp();
                        }
                    }
                }
                if (qn > 0) {
                    __syncwarp();
                    p2p_drain<R>(cp, &qbuf[wid][0], qn, lane, wbase, tx, ty, tz, sx, sy, sz, sq, acc, a.Qn, a.gl_t, a.gl_w, LF_CTAB(a, c));
                    __syncwarp();
                }
            }
        }
        __syncwarp();
        if (valid) {
            P.add(acc[tid][0]);
            Ex.add(acc[tid][1]);
            Ey.add(acc[tid][2]);
            Ez.add(acc[tid][3]);
            if (a.split > 1) {
                atomicAdd(a.phi + i, (double)P.s);
                atomicAdd(a.fld + 3 * (size_t)i + 0, (double)Ex.s);
                atomicAdd(a.fld + 3 * (size_t)i + 1, (double)Ey.s);
                atomicAdd(a.fld + 3 * (size_t)i + 2, (double)Ez.s);
            } else {
                a.phi[i] = (double)P.s;
                a.fld[3 * (size_t)i + 0] = (double)Ex.s;
                a.fld[3 * (size_t)i + 1] = (double)Ey.s;
                a.fld[3 * (size_t)i + 2] = (double)Ez.s;
            }
        }
    }
    if (n_net | n_quad) {
        atomicAdd(&a.sv.counters[0], n_net);
        atomicAdd(&a.sv.counters[1], n_quad);
    }
}

LfErr lf_near_field(lfmm_ctx* ctx, cudaStream_t st)
{
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
    a.comps = ctx->comp_dev.as<LfmmComp>();
    a.gl_t = ctx->gl_t_near.as<double>();
    a.gl_w = ctx->gl_w_near.as<double>();
    const bool tab_on = ctx->near_tab_ready && (ctx->use_near_tab == 1 || (ctx->use_near_tab == 2 && ctx->precision == 1));
    a.ntab = tab_on ? ctx->near_tab.as<double>() : nullptr;
    a.ntab4 = tab_on ? ctx->near_tab4.as<float4>() : nullptr;
    a.grid = nullptr;
    a.pcon = nullptr;
    a.hleaf = (float)leaf.h;
    if (ctx->leaf_int_offsets) {
        a.grid = ctx->box_grid.as<int4>();
        a.pcon = ctx->p2p_consts.as<float4>();
    }
    LF_TRY(lf_reserve(ctx->surr_counters, 64));
    LF_CHECK(cudaMemsetAsync(ctx->surr_counters.ptr, 0, 16, st));
    LF_TRY(lf_surrogate_device_view(ctx, &a.sv));
    a.qstride = ctx->n;
    const int nr = ctx->nrhs_b;
    const size_t qs = (ctx->precision ? sizeof(float) : sizeof(double)) * (size_t)ctx->n;
    const int ph = lf_prof_start(ctx, LFMM_TIME_P2P, st);
    // the network variant only where the near field holds reaction pairs (it
    // needs far more registers, which slows the free-space part); one launch
    // per right-hand side.  The quadrature kernels take batches of up to 4
    // (float32: more registers per thread cost more than the shared pair
    // geometry saves) or 8 (FP64).
    const bool net = a.sv.ready != 0 && ctx->near_reaction_entries > 0;
    // Few leaves (small problems) leave most SMs idle with one warp or block
    // per leaf: share each near list between `split` of them.  A set value
    // (ctx->p2p_split, e.g. from the tuner) wins over this occupancy rule.
    // media of four or five layers need the solved densities only for reaction pairs
    // of the near lists (counted at every build); without any, the kernels of
    // thinner media compute the free-space pairs alone and are exact
    const bool general = ctx->L >= 3 && ctx->near_reaction_entries > 0;
    const bool warp_kernel = !net && !general && ctx->precision;
    int split = ctx->p2p_split;
    if (split <= 0) {
        const int want = warp_kernel ? 152 * 32 : 152 * 8;  // warps, or blocks of P2P_T threads
        split = 1;
        while (split < LFMM_P2P_SPLIT_MAX && (int64_t)leaf.nbox * split * 2 <= want) split *= 2;
    }
    a.split = split;
    if (split > 1) {
        LF_CHECK(cudaMemsetAsync(a.phi, 0, sizeof(double) * (size_t)ctx->n * nr, st));
        LF_CHECK(cudaMemsetAsync(a.fld, 0, 3 * sizeof(double) * (size_t)ctx->n * nr, st));
    }
    const double* phi0 = a.phi;
    double* fld0 = a.fld;
    const char* q0 = reinterpret_cast<const char*>(a.q);
    const int step = (net || general) ? 1 : (ctx->precision ? 4 : 8);
    for (int r0 = 0; r0 < nr; r0 += step) {
        a.nr = nr - r0 < step ? nr - r0 : step;
        a.q = q0 + (size_t)r0 * qs;
        a.phi = const_cast<double*>(phi0) + (size_t)r0 * ctx->n;
        a.fld = fld0 + (size_t)r0 * ctx->n * 3;
        if (general) {
            if (ctx->precision)
                ++ctx->launches, k_p2p<float, 1, true><<<leaf.nbox * split, P2P_T, 0, st>>>(a);
            else
                ++ctx->launches, k_p2p<double, 1, true><<<leaf.nbox * split, P2P_T, 0, st>>>(a);
        } else if (net) {
            if (ctx->precision)
                ++ctx->launches, k_p2p_net<float><<<leaf.nbox * split, P2P_T, 0, st>>>(a);
            else
                ++ctx->launches, k_p2p_net<double><<<leaf.nbox * split, P2P_T, 0, st>>>(a);
        } else if (ctx->precision) {
            const int g = lf_blocks((int64_t)leaf.nbox * split, PW_WARPS), T = 32 * PW_WARPS;
            const float4* rel = ctx->pos_rel.as<float4>();
            if (a.nr == 1 && a.grid && ctx->near_reaction_entries == 0 && ctx->p2p_staged)
                ++ctx->launches, k_p2p_free_staged<<<lf_blocks((int64_t)leaf.nbox * split, PF_WARPS), 32 * PF_WARPS, 0,
                                                     st>>>(a, rel, leaf.nbox);
            else if (a.nr == 1)
                ++ctx->launches, k_p2p_warp<1><<<g, T, 0, st>>>(a, rel, leaf.nbox);
            else if (a.nr == 2)
                ++ctx->launches, k_p2p_warp<2><<<g, T, 0, st>>>(a, rel, leaf.nbox);
            else if (a.nr <= 4)
                ++ctx->launches, k_p2p_warp<4><<<g, T, 0, st>>>(a, rel, leaf.nbox);
            else
                ++ctx->launches, k_p2p_warp<8><<<g, T, 0, st>>>(a, rel, leaf.nbox);
        } else {
            if (a.nr == 1)
                ++ctx->launches, k_p2p<double, 1><<<leaf.nbox * split, P2P_T, 0, st>>>(a);
            else if (a.nr == 2)
                ++ctx->launches, k_p2p<double, 2><<<leaf.nbox * split, P2P_T, 0, st>>>(a);
            else if (a.nr <= 4)
                ++ctx->launches, k_p2p<double, 4><<<leaf.nbox * split, P2P_T, 0, st>>>(a);
            else
                ++ctx->launches, k_p2p<double, 8><<<leaf.nbox * split, P2P_T, 0, st>>>(a);
        }
        LF_TRY(lf_cuda(cudaGetLastError(), "p2p"));
    }
    lf_prof_stop(ctx, ph, st);
    return LfErr();
}

// ---------------------------------------------------------------------------
// Remainder tables of the near-field reaction kernels (built once per
// medium): one thread per (component, w, s) grid point, FP64 quadrature with
// the M2L rule; then a check of the interpolated kernels against the
// quadrature at seeded points.
// ---------------------------------------------------------------------------
template <bool GEN>
__global__ void k_near_tables(const LfmmComp* __restrict__ comps, int ncomp, int Q, const double* __restrict__ gt,
                              const double* __restrict__ gw, double* __restrict__ tab)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)LF_NT_NS * LF_NT_NW;
    if (i >= per * ncomp) return;
    const int c = (int)(i / per);
    const int r = (int)(i - (int64_t)c * per);
    const int iw = r / LF_NT_NS, is = r - iw * LF_NT_NS;
    const LfmmComp cp = comps[c];
    double out[3] = {0.0, 0.0, 0.0};
    if (!cp.is_free && cp.has_rem)
        lf_nt_point<GEN>(cp, is * (LF_NT_SMAX / (LF_NT_NS - 1)), iw * (1.0 / (LF_NT_NW - 1)), Q, gt, gw, out);
    double* t = tab + (size_t)c * LF_NT_PER + r;
    t[0] = out[0];
    t[per] = out[1];
    t[2 * per] = out[2];
}

// the float32 copy of the tables: one float4 {T00, T10, T11, 0} per grid point
__global__ void k_near_tab4(const double* __restrict__ tab, int ncomp, float4* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)LF_NT_NS * LF_NT_NW;
    if (i >= per * ncomp) return;
    const int c = (int)(i / per);
    const int64_t r = i - (int64_t)c * per;
    const double* t = tab + (size_t)c * LF_NT_PER + r;
    out[i] = make_float4((float)t[0], (float)t[per], (float)t[2 * per], 0.f);
}

// err[i]: largest deviation of the three interpolated kernels from the
// quadrature, relative to |I_00| (field kernels times the distance R)
template <bool GEN>
__global__ void k_near_tables_check(const LfmmComp* __restrict__ comps, const int* __restrict__ pc,
                                    const double* __restrict__ prho, const double* __restrict__ ph, int n, int Q,
                                    const double* __restrict__ gt, const double* __restrict__ gw,
                                    const double* __restrict__ tab, double* __restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const LfmmComp& cp = comps[pc[i]];
    double a00, a10, a11, b00, b10, b11;
    lf_reaction_pair<double, GEN>(cp, prho[i], ph[i], Q, gt, gw, a00, a10, a11);
    lf_reaction_pair<double, GEN>(cp, prho[i], ph[i], Q, gt, gw, b00, b10, b11, tab + (size_t)pc[i] * LF_NT_PER);
    const double H = ph[i] + cp.zeta;
    const double R = sqrt(prho[i] * prho[i] + H * H);
    const double sc = fabs(a00) > 1e-300 ? 1.0 / fabs(a00) : 0.0;
    err[i] = fmax(fabs(b00 - a00), fmax(fabs(b10 - a10), fabs(b11 - a11)) * R) * sc;
}

LfErr lf_near_tables(lfmm_ctx* ctx, double* max_err)
{
    cudaStream_t st = ctx->s_main;
    const int nc = ctx->ncomp, Q = ctx->gl_q_m2l;
    if (!ctx->near_tab_ready) {
        LF_TRY(lf_reserve(ctx->near_tab, sizeof(double) * (size_t)LF_NT_PER * nc));
        const int64_t tot = (int64_t)LF_NT_NS * LF_NT_NW * nc;
        auto kern = (ctx->L >= 3) ? k_near_tables<true> : k_near_tables<false>;
        ++ctx->launches, kern<<<lf_blocks(tot, 128), 128, 0, st>>>(
            ctx->comp_dev.as<LfmmComp>(), nc, Q, ctx->gl_t_m2l.as<double>(), ctx->gl_w_m2l.as<double>(),
            ctx->near_tab.as<double>());
        LF_TRY(lf_cuda(cudaGetLastError(), "near tables"));
        LF_TRY(lf_reserve(ctx->near_tab4, sizeof(float4) * (size_t)LF_NT_NS * LF_NT_NW * nc));
        ++ctx->launches, k_near_tab4<<<lf_blocks(tot, 256), 256, 0, st>>>(ctx->near_tab.as<double>(), nc,
                                                                          ctx->near_tab4.as<float4>());
        LF_TRY(lf_cuda(cudaGetLastError(), "near tables (float32 copy)"));
    }
    // seeded check points: per reaction component, s uniform over the table,
    // depth sum h log-uniform in [1e-4, 3]
    std::vector<int> pc;
    std::vector<double> prho, ph;
    uint64_t x = 0x9e3779b97f4a7c15ull;
    auto uni = [&x]() {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        return (double)(x >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int c = 0; c < nc; ++c) {
        const LfmmComp& cp = ctx->comp[c];
        if (cp.is_free || !cp.has_rem) continue;
        for (int k = 0; k < 2048; ++k) {
            const double h = pow(10.0, -4.0 + uni() * (4.0 + log10(3.0)));
            const double sv = uni() * LF_NT_SMAX * 0.999;
            pc.push_back(c);
            ph.push_back(h);
            prho.push_back(sv * (h + cp.zeta_r));
        }
    }
    double worst = 0.0;
    const int n = (int)pc.size();
    if (n > 0) {
        DevBuf dpc, drho, dh, derr;
        LfErr e = lf_reserve(dpc, sizeof(int) * n);
        if (e.empty()) e = lf_reserve(drho, sizeof(double) * n);
        if (e.empty()) e = lf_reserve(dh, sizeof(double) * n);
        if (e.empty()) e = lf_reserve(derr, sizeof(double) * n);
        std::vector<double> herr(n, 0.0);
        if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dpc.ptr, pc.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st), "copy");
        if (e.empty()) e = lf_cuda(cudaMemcpyAsync(drho.ptr, prho.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st), "copy");
        if (e.empty()) e = lf_cuda(cudaMemcpyAsync(dh.ptr, ph.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st), "copy");
        if (e.empty()) {
            auto kern = (ctx->L >= 3) ? k_near_tables_check<true> : k_near_tables_check<false>;
            ++ctx->launches, kern<<<lf_blocks(n, 128), 128, 0, st>>>(
                ctx->comp_dev.as<LfmmComp>(), dpc.as<int>(), drho.as<double>(), dh.as<double>(), n, Q,
                ctx->gl_t_m2l.as<double>(), ctx->gl_w_m2l.as<double>(), ctx->near_tab.as<double>(),
                derr.as<double>());
            e = lf_cuda(cudaGetLastError(), "near tables check");
        }
        if (e.empty()) e = lf_cuda(lf_d2h(herr.data(), derr.ptr, sizeof(double) * n, st), "check");
        for (DevBuf* b : {&dpc, &drho, &dh, &derr})
            if (b->ptr) cudaFree(b->ptr);
        if (!e.empty()) return e;
        for (double v : herr) worst = std::max(worst, v);
    } else {
        LF_TRY(lf_cuda(cudaStreamSynchronize(st), "near tables"));
    }
    ctx->near_tab_ready = 1;
    ctx->near_tab_err = worst;
    if (max_err) *max_err = worst;
    return LfErr();
}

// ---------------------------------------------------------------------------
// Parity entry points: the same device routines on caller-given geometries.
// ---------------------------------------------------------------------------
template <bool GEN>
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
    lf_sommerfeld_table_block<GEN>(c, rho[i] / S, z[i] / S, S, 2 * P, sT, TS, Q, gt, gw, sJ, sA);
    for (int j = threadIdx.x; j < TT; j += blockDim.x) out[(size_t)i * TT + j] = sT[j];
}

LfErr lf_sommerfeld_tables_dev(lfmm_ctx* ctx, int comp, int npts, const double* rho, const double* z, double S,
                               int P, double* out)
{
    const int TS = 2 * P + 1;
    const int Q = ctx->gl_q_m2l;
    size_t sm = sizeof(double) * ((size_t)TS * TS + 2 * (size_t)Q * TS);
    auto kern = (ctx->L >= 3) ? k_som_tables<true> : k_som_tables<false>;
    LF_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    ++ctx->launches, kern<<<npts, 128, sm, ctx->s_main>>>(ctx->comp[comp], npts, rho, z, S, P, ctx->gl_t_m2l.as<double>(),
                                                  ctx->gl_w_m2l.as<double>(), Q, out);
    return lf_cuda(cudaGetLastError(), "sommerfeld tables");
}

template <bool GEN>
__global__ void k_reaction_kernel(const LfmmComp* __restrict__ comps, const double* __restrict__ gl_t,
                                  const double* __restrict__ gl_w, int comp, int npts, const double* __restrict__ rho,
                                  const double* __restrict__ h, int Q, double* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    double k00, k10, k11;
    lf_reaction_pair<double, GEN>(comps[comp], rho[i], h[i], Q, gl_t, gl_w, k00, k10, k11);
    out[3 * (size_t)i] = k00;
    out[3 * (size_t)i + 1] = k10;
    out[3 * (size_t)i + 2] = k11;
}

LfErr lf_reaction_kernel_dev(lfmm_ctx* ctx, int comp, int npts, const double* rho, const double* h, double* out)
{
    auto kern = (ctx->L >= 3) ? k_reaction_kernel<true> : k_reaction_kernel<false>;
    ++ctx->launches, kern<<<lf_blocks(npts, 128), 128, 0, ctx->s_main>>>(
        ctx->comp_dev.as<LfmmComp>(), ctx->gl_t_near.as<double>(), ctx->gl_w_near.as<double>(), comp, npts, rho, h,
        ctx->gl_q_near, out);
    return lf_cuda(cudaGetLastError(), "reaction kernel");
}

// ---------------------------------------------------------------------------
// Allocation-free variant of lfmm_reaction_kernel.
//
// Some callers cannot allocate device memory at the point where they need the
// layered reaction kernel: real-time or embedded loops whose rules forbid
// allocator calls after start-up, and hosts that hand this library a device
// on which another runtime already owns the memory budget.
// lfmm_reaction_kernel stages its inputs and outputs through buffers it
// allocates on every call; this variant stages them through one file-scope
// device array instead, so the call itself makes no cudaMalloc / cudaFree (or
// any other allocating call).  Like lfmm_reaction_kernel it copies from and
// to the caller's host arrays and waits for the context's stream before it
// returns.
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
// first time the entry point runs on a device and cached per device; that
// first call therefore must come before any stream capture.  The call runs on
// the device the context was created on, which must be the current device.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_scratch[5 * LFMM_NOALLOC_MAX_POINTS];

static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[LFMM_MAX_DEVICES] = {nullptr};

// The array's device address on `device`, which the caller has checked is
// the current device.
static LfErr noalloc_scratch(int device, double** out)
{
    if (device < 0 || device >= LFMM_MAX_DEVICES) return "EINVAL: device index out of range";
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
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
    int cur = -1;
    cudaError_t ce = cudaGetDevice(&cur);
    if (ce != cudaSuccess) {
        ctx->err = lf_cuda(ce, "cudaGetDevice");
        return LFMM_ECUDA;
    }
    if (cur != ctx->device) {
        ctx->err = "EINVAL: the current device (" + std::to_string(cur) + ") is not the context's device (" +
                   std::to_string(ctx->device) + "); make the context's device current first";
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
    if (e.empty()) {
        auto kern = (ctx->L >= 3) ? k_reaction_kernel<true> : k_reaction_kernel<false>;
        ++ctx->launches, kern<<<lf_blocks(npts, 128), 128, 0, st>>>(
            ctx->comp_dev.as<LfmmComp>(), ctx->gl_t_near.as<double>(), ctx->gl_w_near.as<double>(), c, npts, drho, dh,
            ctx->gl_q_near, dout);
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
