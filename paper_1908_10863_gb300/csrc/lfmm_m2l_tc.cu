// lfmm_m2l_tc.cu -- free-space M2L (eq. metole) on the tcgen05 tensor cores.
//
// The same per-offset real-linear maps A_o as the CUDA-core GEMM in
// lfmm_m2l.cu, evaluated as D[r][j] = sum_o sum_k A_o[r][k] X_o[j][k] with
//   r = output coefficient (M = 128 rows, expansions with (p+1)^2 <= 128),
//   j = target box of the tile (N = 256 columns, one level and octant class),
//   k = input coefficient of the source at offset o (K = 128 in chunks of
//       TC_KC, only the chunks that hold the (p+1)^2 inputs),
// accumulated in tensor memory (128 lanes x 256 float32 columns).  The wide
// form takes 128 < (p+1)^2 <= 256 (p = 11 .. 14): two 128-row halves of r,
// K = 256, tiles of 128 targets (see k_m2l_tc<true>).
//
// Precision: float32 operands as sums of two TF32 pieces, the operator
// (a1 + a2, from its FP64 values) and the multipoles (x1 + x2, split once per
// evaluation), with the three products a1 x1 + a1 x2 + a2 x1 ("3xTF32",
// ~2^-21 of |a||x| per product).  What limits the result is the tensor
// core's float32 accumulation: its error grows with the number of MMAs
// summed into one accumulator, so each CTA takes only 7 of the 189 offsets
// (27 CTAs per tile, joined by float atomics), which keeps the far field
// within the CUDA-core float32 GEMM's error (measured: Err2 of the potential
// against the FP64 path 2.0e-6 with 7 offsets per CTA, 1.2e-5 with 63,
// 3.3e-5 with 189; 1.4e-6 for the CUDA-core float32 GEMM).
//
// One CTA = (tile of 256 targets, one third of its 189 offsets):
//   warps 0..7  gather the 256 pre-split source multipoles of a (offset,
//               K chunk) stage with 16-byte cp.async into the swizzled
//               K-major layout (zeros where a target has no source there), ahead
//               of the tensor cores; thread 0 also starts the bulk
//               copy of the matching operator chunk (stored pre-split and
//               pre-swizzled in HBM);
//   warp 8      one thread issues the MMAs of a stage (3 products x K chunk / 8) and commits them to
//               the stage's "empty" barrier;
//   epilogue    warps 0..7 read the accumulator (tcgen05.ld), scale by 1/h and
//               add into the local expansions (float atomics: the CTAs of a
//               tile's offset groups meet there).
// Two stages of 48 KB (K chunks of 16, 64-byte swizzle) per CTA buffer the
// operands, handed to the tensor cores one stage after their copies start;
// two CTAs share an SM, so four stages are in flight per SM.  (K chunks of 8
// with 32-byte swizzle, or one CTA per SM with four stages, measured slower.)
// Tiles of one octant class share their offset list; each tile walks it from a different starting offset so
// that concurrent CTAs read different operator chunks.  Every barrier wait is
// bounded; on a timeout the CTA records an error, stops issuing work, waits
// (bounded) for its copies in flight and frees its tensor memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "lfmm_ctx.h"
#include "lfmm_tc.cuh"

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

#define TC_N 256                     // targets per tile (MMA N)
#define TC_M 128                     // output coefficients (MMA M)
#define TC_NKC (128 / TC_KC)         // K chunks (K = 128)
#define TC_RCH (TC_ROWB / 16)        // 16-byte chunks per row
#define TC_NOFF 189                  // offsets per octant class
#define TC_NALL 343
#define TC_PROD_WARPS 8
#define TC_THREADS (32 * TC_PROD_WARPS + 32)
#define TC_A_BYTES (TC_M * TC_ROWB)  // one operator piece of a stage
#define TC_X_BYTES (TC_N * TC_ROWB)  // one multipole piece of a stage
#define TC_AP 2                      // operator pieces
#define TC_XP 2                      // multipole pieces
#define TC_STAGE_BYTES (TC_AP * TC_A_BYTES + TC_XP * TC_X_BYTES)
#define TC_MROW 128                  // floats per multipole piece row in the split copy (512 B)
// Two CTAs per SM (97 KB of shared memory and 256 tensor-memory columns
// each), two 48 KB stages apiece: one CTA's prologue, gathers and atomic
// epilogue overlap the other's MMAs.  Measured at N = 1M, p = 10: 2.39 ms
// against 2.63 ms for one CTA per SM with four stages.
#ifndef TC_STAGES
#define TC_STAGES 2
#endif
#ifndef TC_LAG
#define TC_LAG (TC_STAGES / 2)           // stages between a stage's copies and its hand-over
#endif
#ifndef TC_MINB
#define TC_MINB 2                        // resident CTAs per SM
#endif
#define TC_SMEM (TC_STAGES * TC_STAGE_BYTES + 1024)
#define TC_TMEM_COLS 256
#define TC_WIDE_STAGES 4             // wide form: one CTA per SM
#define TC_WIDE_SMEM (TC_WIDE_STAGES * TC_STAGE_BYTES + 1024)
#define TC_MSEG LFMM_TC_MSEG

struct TcArgs {
    const int4* tiles;      // level, class, start, count
    const int* sorted;      // target boxes grouped by (level, class), or null: targets start .. start + count - 1
    const int* slots;       // [box][noff] source box at each offset of the class, or -1
    const int* cls;         // [class][noff] operator index of each class position
    int noff;               // offsets per class: 189 (M2L), 8 (M2M: children), 1 (L2L: parent)
    int unit_scale;         // 1: add D as it is (M2M, L2L); 0: add D / h_level (M2L)
    const double* levelh;   // box size per level
    const int4* mseg;       // merged tiles' runs [merged tile][TC_MSEG]: (level, start, count, 0)
    const unsigned char* A; // [343][4 chunks][2 pieces x 16 KB], pre-swizzled
    const float* Ms;        // split multipoles [box + 1][2 pieces][128] (last box: zeros)
    int zero_row;           // index of the zero box of Ms
    float* L;               // locals [box][nc]
    int nc;
    int nkc;                // K chunks of TC_KC coefficients that hold the nc inputs: ceil(nc / TC_KC)
    size_t ms_stride;       // per right-hand side (blockIdx.y): split multipoles, in floats
    size_t l_stride;        // per right-hand side: local expansions, in floats
    int groups;             // CTAs per tile (offset groups; divides noff)
    int* err;               // [0]: timeouts
};

// Target t of a tile (a box id, or -1 past the tile's count) and its output
// scale (1 for M2M and L2L, 1/h of the target's level for M2L).  A tile with
// level < 0 is a merged tile: the leftover runs (fewer targets than a tile)
// of one octant class on several levels, listed at mseg[-1 - level] with
// tile.z runs; its columns take the runs in order, each with its level's
// scale (the operators depend only on the class and the offset).
__device__ __forceinline__ int tc_tile_target(const TcArgs& g, const int4& tile, int t, float& ih)
{
    ih = 0.f;
    if (t >= tile.w) return -1;
    if (tile.x >= 0) {
        ih = g.unit_scale ? 1.f : 1.f / (float)g.levelh[tile.x];
        return g.sorted ? g.sorted[tile.z + t] : tile.z + t;
    }
    const int4* sg = g.mseg + (size_t)(-1 - tile.x) * TC_MSEG;
    for (int k = 0; k < tile.z; ++k) {
        const int4 r = sg[k];
        if (t < r.z) {
            ih = g.unit_scale ? 1.f : 1.f / (float)g.levelh[r.x];
            return g.sorted[r.y + t];
        }
        t -= r.z;
    }
    return -1;
}

// WIDE: expansions with 128 < (p+1)^2 <= 256 (p <= 15): the output rows are
// two 128-row halves (two MMAs per K step), K runs over 16 chunks, and a tile
// holds 128 targets, so a stage keeps its 48 KB.  With twice the MMAs per
// offset, the large product a1 x1 gets an accumulator of its own (256
// columns) and the two correction products share a second one: the float32
// accumulation drift of the tensor cores grows with the MMAs summed into
// one accumulator, and the corrections are 2^-11 of the large product.  The
// 512 columns allow one CTA per SM, which then runs four stages.
template <bool WIDE>
__global__ void __launch_bounds__(TC_THREADS, WIDE ? 1 : TC_MINB) k_m2l_tc(TcArgs g)
{
    constexpr int TN = WIDE ? 128 : TC_N;       // targets per tile (MMA N)
    constexpr int MH = WIDE ? 2 : 1;            // 128-row halves of the output (MMA M = 128 each)
    constexpr int NKC = WIDE ? 16 : TC_NKC;     // K chunks per operator in the blob
    constexpr int MROW = WIDE ? 256 : TC_MROW;  // floats per multipole piece row
    constexpr int ABYTES = MH * TC_A_BYTES;     // one operator piece of a stage
    constexpr int XBYTES = TN * TC_ROWB;        // one multipole piece of a stage
    constexpr int NST = WIDE ? TC_WIDE_STAGES : TC_STAGES;
    constexpr int LAG = WIDE ? TC_WIDE_STAGES / 2 : TC_LAG;
    constexpr uint32_t COLS = WIDE ? 2 * TC_TMEM_COLS : TC_TMEM_COLS;
    constexpr uint32_t SMALL = WIDE ? TC_TMEM_COLS : 0;  // accumulator of the correction products
    static_assert(TC_AP * ABYTES + TC_XP * XBYTES == TC_STAGE_BYTES, "stage size");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[NST], empty_bar[NST], done_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ int s_tb[TC_N];
    __shared__ float s_ih[TC_N];  // output scale of each target column

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int item = blockIdx.x;
    const int4 tile = g.tiles[item / g.groups];
    const int grp = item % g.groups;
    const int goff = g.noff / g.groups;
    const int cl = tile.y, cnt = tile.w;
    const int nc = g.nc;
    const int nkc = g.nkc;  // K chunks that hold coefficients (the rest are zero)
    const int nstage = goff * nkc;

    if (tid < TN) {
        float ih;
        s_tb[tid] = tc_tile_target(g, tile, tid, ih);
        s_ih[tid] = ih;
    }
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full_bar[s], TC_PROD_WARPS + 1);  // one arrival per producer warp + the bulk copy's
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == TC_PROD_WARPS) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp < TC_PROD_WARPS) {
        // ---------------- producers ----------------
        // stage it is filled at iteration it and handed to the tensor cores at
        // iteration it + TC_LAG, once its copies have landed
        const int ptid = tid;  // 0 .. 255
        const int rot = (item / g.groups) % goff;
        int armed = 0;         // stages with a bulk copy issued by this thread, for the bounded drain
        int my_src = -1;       // source of row (warp * 32 + lane) at the current offset
        // the source at the next offset is loaded one offset ahead (its
        // latency hides behind the current offset's gathers)
        const int my_tb = s_tb[(WIDE ? (warp & 3) : warp) * 32 + lane];
        int nxt_src = (my_tb >= 0) ? g.slots[(size_t)my_tb * g.noff + grp * goff + rot % goff] : -1;
        int it = 0;
        for (; it < nstage; ++it) {
            const int s = it % NST, round = it / NST;
            const int oi = grp * goff + (it / nkc + rot) % goff, kc = it % nkc;
            if (it >= NST) {
                if (!mbar_wait(&empty_bar[s], (round - 1) & 1)) atomicExch(&s_abort, 1);
            }
            if (__any_sync(0xffffffffu, *(volatile int*)&s_abort)) break;  // warp-uniform
            unsigned char* st = sm + (size_t)s * TC_STAGE_BYTES;
            if (ptid == 0) {
                const int o = g.cls[cl * g.noff + oi];
                mbar_arrive_tx(&full_bar[s], TC_AP * ABYTES);
                bulk_g2s(st, g.A + ((size_t)o * NKC + kc) * (TC_AP * ABYTES), TC_AP * ABYTES, &full_bar[s]);
                armed = it + 1;
            }
            if (kc == 0) {
                my_src = nxt_src;
                const int on = it / nkc + 1;
                if (on < goff && my_tb >= 0) nxt_src = g.slots[(size_t)my_tb * g.noff + grp * goff + (on + rot) % goff];
            }
            unsigned char* xs = st + TC_AP * ABYTES;
            const uint32_t xbase = smem_u32(xs);
            // 32 rows x TC_RCH chunks of 16 B per warp and piece: both pieces
            // per warp (256 rows), or warps 4..7 the second piece (128 rows)
            constexpr int NI = WIDE ? TC_RCH : 2 * TC_RCH;
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                const int piece = WIDE ? (warp >> 2) : i / TC_RCH;
                const int flat = (WIDE ? i : i % TC_RCH) * 32 + lane;  // chunk-major over the warp's 32 rows
                const int rl = flat / TC_RCH, chunk = flat % TC_RCH;
                const int src = __shfl_sync(0xffffffffu, my_src, rl);
                const int row = (WIDE ? (warp & 3) : warp) * 32 + rl;
                const uint32_t off = piece * XBYTES + swz(row, chunk * 4);
                if (src >= 0) {
                    const float* gsrc = g.Ms + (size_t)blockIdx.y * g.ms_stride + ((size_t)src * TC_XP + piece) * MROW +
                                        kc * TC_KC + chunk * 4;
                    cp_async16(xbase + off, gsrc);
                } else {
                    *reinterpret_cast<float4*>(xs + off) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            cp_async_commit();
            if (it >= LAG) {
                cp_async_wait<LAG>();
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full_bar[(it - LAG) % NST]);
            }
        }
        cp_async_wait<0>();
        fence_async_smem();
        __syncwarp();
        if (lane == 0)
            for (int j = (it > LAG ? it - LAG : 0); j < it; ++j) mbar_arrive(&full_bar[j % NST]);
        // drain: the bulk copies this thread issued complete on their full barriers
        if (ptid == 0 && *(volatile int*)&s_abort) {
            for (int j = (armed > NST ? armed - NST : 0); j < armed; ++j)
                mbar_wait(&full_bar[j % NST], (j / NST) & 1);
        }
        // ---------------- epilogue ----------------
        const bool ok = mbar_wait(&done_bar, 0);
        tc_fence_after();
        if (ok && !*(volatile int*)&s_abort) {
            const int q = warp & 3, half = warp >> 2;
            // narrow: half = target half of the 256 columns; wide: half = the
            // 128-row half of the outputs, whose accumulator starts at column half * TN
            const int row = (WIDE ? 128 * half : 0) + 32 * q + lane;
#pragma unroll 1
            for (int ch = 0; ch < 4; ++ch) {
                const int col0 = (WIDE ? 0 : half * 128) + ch * 32;  // first target of the chunk
                float v[32];
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((WIDE ? half * TN : 0) + col0);
                tc_ld32(ta, v);
                if (WIDE) {
                    float w[32];
                    tc_ld32(ta + SMALL, w);
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] += w[i];
                }
                if (row < nc) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int j = col0 + i;
                        if (j < cnt) atomicAdd(g.L + (size_t)blockIdx.y * g.l_stride + (size_t)s_tb[j] * nc + row, v[i] * s_ih[j]);
                    }
                }
            }
        } else if (lane == 0) {
            atomicAdd(g.err, 1);
        }
    } else {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = tc_idesc(TC_M, TN);
            bool ok = true;
            for (int it = 0; it < nstage && ok; ++it) {
                const int s = it % NST, round = it / NST;
                if (!mbar_wait(&full_bar[s], round & 1)) {
                    ok = false;
                    atomicExch(&s_abort, 1);
                    break;
                }
                tc_fence_after();
                const uint32_t base = smem_u32(sm + (size_t)s * TC_STAGE_BYTES);
                const uint32_t xb = base + TC_AP * ABYTES;
                // a1 x1, a1 x2, a2 x1
                const int pa[3] = {0, 0, 1}, px[3] = {0, 1, 0};
#pragma unroll
                for (int prod = 0; prod < 3; ++prod) {
                    const uint32_t a = base + pa[prod] * ABYTES;
                    const uint32_t b = xb + px[prod] * XBYTES;
                    // narrow: one accumulator; wide: a1 x1 alone, the corrections in the second
                    const uint32_t acc = (WIDE && prod > 0) ? SMALL : 0u;
                    const int first = WIDE ? (prod == 2 ? 1 : 0) : prod;  // 0: may start its accumulator
#pragma unroll
                    for (int ks = 0; ks < TC_KC / 8; ++ks)
#pragma unroll
                        for (int h = 0; h < MH; ++h)
                            tc_mma(tmem + acc + (uint32_t)(h * TN), smem_desc(a + h * TC_A_BYTES + 32 * ks),
                                   smem_desc(b + 32 * ks), idesc, (it | first | ks) != 0 ? 1u : 0u);
                }
                tc_commit(&empty_bar[s]);
            }
            tc_commit(&done_bar);
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == TC_PROD_WARPS) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Persistent form of the free M2L (one CTA per SM).
//
// The work units are the (tile, offset group) pairs of k_m2l_tc; each CTA
// walks units u = blockIdx.x, blockIdx.x + gridDim.x, ... with one pipeline
// that never drains between units:
//   warps 0..7   producers: operator chunk by bulk copy, multipole rows by
//                16-byte cp.async gathers, TCP_STAGES stages of 48 KB, each
//                handed to the tensor cores TCP_LAG stages after its copies
//                start (stage counter global over the CTA's units);
//   warp 8       one thread issues the MMAs of a unit into one of two
//                256-column tensor-memory accumulators (unit parity), and
//                commits the unit to that accumulator's "full" barrier;
//   warps 9..12  epilogue: read the finished accumulator (tcgen05.ld; warp w
//                reads lanes 32 (w mod 4) .. + 31), scale by 1/h and add into
//                the local expansions, then release the accumulator, while
//                the tensor cores already work on the next unit.
// Same arithmetic, offset groups and error behaviour as k_m2l_tc; every
// barrier wait is bounded as there.
// ---------------------------------------------------------------------------
#ifndef TCP_STAGES
#define TCP_STAGES 4
#endif
#ifndef TCP_LAG
#define TCP_LAG 2
#endif
#define TCP_EPI_WARPS 4
#define TCP_THREADS (32 * (TC_PROD_WARPS + 1 + TCP_EPI_WARPS))
#define TCP_SMEM (TCP_STAGES * TC_STAGE_BYTES + 1024)
#define TCP_TMEM_COLS 512

__global__ void __launch_bounds__(TCP_THREADS, 1) k_m2l_tcp(TcArgs g, int nunits)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[TCP_STAGES], empty_bar[TCP_STAGES], accf_bar[2], acce_bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int goff = g.noff / g.groups;
    const int nstage = goff * g.nkc;  // stages per unit
    const int nc = g.nc;

    if (tid == 0) {
        for (int s = 0; s < TCP_STAGES; ++s) {
            mbar_init(&full_bar[s], TC_PROD_WARPS + 1);  // one arrival per producer warp + the bulk copy's
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf_bar[b], 1);              // the MMA thread's commit
            mbar_init(&acce_bar[b], TCP_EPI_WARPS);  // one arrival per epilogue warp
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == TC_PROD_WARPS) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TCP_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp < TC_PROD_WARPS) {
        // ---------------- producers ----------------
        const int row = warp * 32 + lane;  // this thread's target row of every tile
        int armed = 0;                     // stages with a bulk copy issued by this thread
        int it = 0;                        // global stage counter
        bool stop = false;
        for (int u = blockIdx.x; u < nunits && !stop; u += gridDim.x) {
            const int4 tile = g.tiles[u / g.groups];
            const int grp = u % g.groups;
            const int cl = tile.y;
            float ih_unused;
            const int my_tb = tc_tile_target(g, tile, row, ih_unused);
            const int rot = (u / g.groups) % goff;
            int my_src = -1;
            // the source at the next offset is loaded one offset ahead
            int nxt_src = (my_tb >= 0) ? g.slots[(size_t)my_tb * g.noff + grp * goff + rot % goff] : -1;
            for (int j = 0; j < nstage; ++j, ++it) {
                const int s = it % TCP_STAGES, round = it / TCP_STAGES;
                const int oi = grp * goff + (j / g.nkc + rot) % goff, kc = j % g.nkc;
                if (it >= TCP_STAGES) {
                    if (!mbar_wait(&empty_bar[s], (round - 1) & 1)) atomicExch(&s_abort, 1);
                }
                if (__any_sync(0xffffffffu, *(volatile int*)&s_abort)) {  // warp-uniform
                    stop = true;
                    break;
                }
                unsigned char* st = sm + (size_t)s * TC_STAGE_BYTES;
                if (row == 0) {
                    const int o = g.cls[cl * g.noff + oi];
                    mbar_arrive_tx(&full_bar[s], TC_AP * TC_A_BYTES);
                    bulk_g2s(st, g.A + ((size_t)o * TC_NKC + kc) * (TC_AP * TC_A_BYTES), TC_AP * TC_A_BYTES,
                             &full_bar[s]);
                    armed = it + 1;
                }
                if (kc == 0) {
                    my_src = nxt_src;
                    const int on = j / g.nkc + 1;
                    if (on < goff && my_tb >= 0)
                        nxt_src = g.slots[(size_t)my_tb * g.noff + grp * goff + (on + rot) % goff];
                }
                unsigned char* xs = st + TC_AP * TC_A_BYTES;
                const uint32_t xbase = smem_u32(xs);
#pragma unroll
                for (int i = 0; i < 2 * TC_RCH; ++i) {
                    const int piece = i / TC_RCH;
                    const int flat = (i % TC_RCH) * 32 + lane;  // chunk-major over the warp's 32 rows
                    const int rl = flat / TC_RCH, chunk = flat % TC_RCH;
                    const int src = __shfl_sync(0xffffffffu, my_src, rl);
                    const int r = warp * 32 + rl;
                    const uint32_t off = piece * TC_X_BYTES + swz(r, chunk * 4);
                    if (src >= 0) {
                        const float* gsrc = g.Ms + (size_t)blockIdx.y * g.ms_stride +
                                            ((size_t)src * TC_XP + piece) * TC_MROW + kc * TC_KC + chunk * 4;
                        cp_async16(xbase + off, gsrc);
                    } else {
                        *reinterpret_cast<float4*>(xs + off) = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                cp_async_commit();
                if (it >= TCP_LAG) {
                    cp_async_wait<TCP_LAG>();
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full_bar[(it - TCP_LAG) % TCP_STAGES]);
                }
            }
        }
        cp_async_wait<0>();
        fence_async_smem();
        __syncwarp();
        if (lane == 0)
            for (int j = (it > TCP_LAG ? it - TCP_LAG : 0); j < it; ++j) mbar_arrive(&full_bar[j % TCP_STAGES]);
        // drain: the bulk copies this thread issued complete on their full barriers
        if (row == 0 && *(volatile int*)&s_abort) {
            for (int j = (armed > TCP_STAGES ? armed - TCP_STAGES : 0); j < armed; ++j)
                mbar_wait(&full_bar[j % TCP_STAGES], (j / TCP_STAGES) & 1);
        }
    } else if (warp == TC_PROD_WARPS) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = tc_idesc(TC_M, TC_N);
            int it = 0, ul = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++ul) {
                const int b = ul & 1;
                if (ul >= 2 && !mbar_wait(&acce_bar[b], ((ul >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * TC_N);
                for (int j = 0; j < nstage; ++j, ++it) {
                    const int s = it % TCP_STAGES, round = it / TCP_STAGES;
                    if (!mbar_wait(&full_bar[s], round & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(sm + (size_t)s * TC_STAGE_BYTES);
                    const uint32_t xb = base + TC_AP * TC_A_BYTES;
                    const int pa[3] = {0, 0, 1}, px[3] = {0, 1, 0};  // a1 x1, a1 x2, a2 x1
#pragma unroll
                    for (int prod = 0; prod < 3; ++prod) {
                        const uint32_t a = base + pa[prod] * TC_A_BYTES;
                        const uint32_t bb = xb + px[prod] * TC_X_BYTES;
#pragma unroll
                        for (int ks = 0; ks < TC_KC / 8; ++ks)
                            tc_mma(acc, smem_desc(a + 32 * ks), smem_desc(bb + 32 * ks), idesc,
                                   (j | prod | ks) != 0 ? 1u : 0u);
                    }
                    tc_commit(&empty_bar[s]);
                }
                if (!ok) break;
                tc_commit(&accf_bar[b]);
            }
            if (!ok) atomicExch(&s_abort, 1);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        // (no barrier between the epilogue warps: each decides on its own,
        // so a warp that gives up on a timed-out wait cannot strand another)
        const int q = warp & 3;  // tensor-memory lanes 32 q .. 32 q + 31
        const int r = 32 * q + lane;
        int ul = 0;
        for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++ul) {
            const int b = ul & 1;
            const int4 tile = g.tiles[u / g.groups];
            const int cnt = tile.w;
            const bool ok = mbar_wait(&accf_bar[b], (ul >> 1) & 1);
            tc_fence_after();
            if (!ok || *(volatile int*)&s_abort) {
                if (lane == 0) atomicAdd(g.err, 1);
                atomicExch(&s_abort, 1);
                break;
            }
            float* Lb = g.L + (size_t)blockIdx.y * g.l_stride;
#pragma unroll 1
            for (int ch = 0; ch < TC_N / 32; ++ch) {
                const int col0 = ch * 32;
                if (col0 >= cnt) break;  // warp-uniform
                // target box of column col0 + lane, handed to every lane by shuffles
                const int jl = col0 + lane;
                float ihl;
                const int tbl = tc_tile_target(g, tile, jl, ihl);
                float v[32];
                tc_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * TC_N + col0), v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int tb = __shfl_sync(0xffffffffu, tbl, i);
                    const float ih = __shfl_sync(0xffffffffu, ihl, i);
                    if (r < nc && tb >= 0) atomicAdd(Lb + (size_t)tb * nc + r, v[i] * ih);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce_bar[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == TC_PROD_WARPS) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCP_TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Host: operator blob and launch.
// ---------------------------------------------------------------------------
static inline uint32_t host_tf32(float x)
{
    // round to nearest (ties away from zero) at 10 explicit mantissa bits
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return u;
    u = (u + 0x1000u) & 0xffffe000u;
    return u;
}

// A64: [nops][KP in][RP out] (double) -> the tensor-core operator blob:
// per operator nkc K chunks of two TF32 pieces, each piece mh 128-row halves
// (mh = 2 for the wide form), pre-swizzled
static LfErr tc_blob(const double* A64, int nops, int KP, int RP, int nc, bool wide, DevBuf& out)
{
    const int mh = wide ? 2 : 1, nkc = wide ? 16 : TC_NKC;
    const size_t chunk = (size_t)TC_AP * mh * TC_A_BYTES;
    const size_t per = (size_t)nkc * chunk;
    std::vector<uint32_t> blob((size_t)nops * per / 4, 0u);
    for (int o = 0; o < nops; ++o)
        for (int kc = 0; kc < nkc; ++kc) {
            unsigned char* p0 = reinterpret_cast<unsigned char*>(blob.data()) + (size_t)o * per + (size_t)kc * chunk;
            for (int r = 0; r < mh * TC_M; ++r)
                for (int k = 0; k < TC_KC; ++k) {
                    const int kin = kc * TC_KC + k;
                    double v = (r < nc && kin < nc) ? A64[((size_t)o * KP + kin) * RP + r] : 0.0;
                    for (int q = 0; q < TC_AP; ++q) {
                        uint32_t t = host_tf32((float)v);
                        float tf;
                        memcpy(&tf, &t, 4);
                        memcpy(p0 + ((size_t)q * mh + r / TC_M) * TC_A_BYTES + swz(r % TC_M, k), &t, 4);
                        v -= (double)tf;
                    }
                }
        }
    LF_TRY(lf_reserve(out, blob.size() * 4));
    LF_CHECK(cudaMemcpy(out.ptr, blob.data(), blob.size() * 4, cudaMemcpyHostToDevice));
    return LfErr();
}

// A64: [343][KP][RP] free M2L operators; M2M, L2L: [8][KP][RP] octant operators
LfErr lf_setup_m2l_tc(lfmm_ctx* ctx, const double* A64, const double* M2M64, const double* L2L64, int KP, int RP)
{
    const int nc = lf_nc(ctx->p);
    ctx->m2l_tc_ok = 0;
    ctx->m2l_tc_wide = 0;
    if (nc > 2 * TC_M || KP < nc || RP < nc) return LfErr();
    const bool wide = nc > TC_M;
    // the wide form serves the free M2L only; M2M and L2L stay on the CUDA cores
    LF_TRY(tc_blob(A64, TC_NALL, KP, RP, nc, wide, ctx->m2l_Atc));
    if (!wide) {
        LF_TRY(tc_blob(M2M64, 8, KP, RP, nc, false, ctx->m2m_Atc));
        LF_TRY(tc_blob(L2L64, 8, KP, RP, nc, false, ctx->l2l_Atc));
    }
    LF_CHECK(cudaFuncSetAttribute(k_m2l_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    LF_CHECK(cudaFuncSetAttribute(k_m2l_tc<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    LF_CHECK(cudaFuncSetAttribute(k_m2l_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_WIDE_SMEM));
    LF_CHECK(cudaFuncSetAttribute(k_m2l_tc<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    LF_CHECK(cudaFuncSetAttribute(k_m2l_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize, TCP_SMEM));
    LF_CHECK(cudaFuncSetAttribute(k_m2l_tcp, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int nsm = 0;
    LF_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    ctx->num_sms = nsm > 0 ? nsm : 152;
    ctx->m2l_tc_wide = wide ? 1 : 0;
    ctx->m2l_tc_ok = 1;
    return LfErr();
}

// expansions [box][nc] -> two TF32 pieces per box, rows padded to mrow floats
// (128, or 256 for the wide form), for the boxes b0 .. b0 + count - 1 (the
// arrays hold nbox boxes per right-hand side, blockIdx.y)
__global__ void k_split_m(const float* __restrict__ M, int nbox, int nc, int mrow, int b0, int count,
                          float* __restrict__ Ms)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)count * mrow) return;
    M += (size_t)blockIdx.y * nbox * nc;
    Ms += (size_t)blockIdx.y * (nbox + 1) * TC_XP * mrow;
    const int b = b0 + (int)(i / mrow), k = (int)(i % mrow);
    const float x = (k < nc) ? M[(size_t)b * nc + k] : 0.f;
    const uint32_t hi = to_tf32(x);
    const uint32_t lo = to_tf32(x - __uint_as_float(hi));
    Ms[((size_t)b * TC_XP + 0) * mrow + k] = __uint_as_float(hi);
    Ms[((size_t)b * TC_XP + 1) * mrow + k] = __uint_as_float(lo);
}

static int ms_row(const lfmm_ctx* ctx) { return ctx->m2l_tc_wide ? 2 * TC_MROW : TC_MROW; }

static LfErr split_boxes(lfmm_ctx* ctx, const float* src, int b0, int count, cudaStream_t st)
{
    if (count <= 0) return LfErr();
    const int nb = ctx->nbox_total, nr = ctx->nrhs_b, mrow = ms_row(ctx);
    LF_TRY(lf_reserve(ctx->m2l_Ms, (size_t)(nb + 1) * TC_XP * mrow * sizeof(float) * nr));
    const size_t tot = (size_t)count * mrow;
    ++ctx->launches, k_split_m<<<dim3((unsigned)((tot + 255) / 256), nr), 256, 0, st>>>(
        src, nb, lf_nc(ctx->p), mrow, b0, count, ctx->m2l_Ms.as<float>());
    return lf_cuda(cudaGetLastError(), "split");
}

static TcArgs tc_args(lfmm_ctx* ctx)
{
    const int nb = ctx->nbox_total;
    TcArgs g;
    g.levelh = ctx->m2l_levelh.as<double>();
    g.mseg = ctx->tc_mseg.as<int4>();
    g.Ms = ctx->m2l_Ms.as<float>();
    g.zero_row = nb;
    g.ms_stride = (size_t)(nb + 1) * TC_XP * ms_row(ctx);
    g.l_stride = (size_t)nb * lf_nc(ctx->p);
    g.nc = lf_nc(ctx->p);
    g.nkc = (g.nc + TC_KC - 1) / TC_KC;
    g.err = reinterpret_cast<int*>(ctx->counts.as<char>() + LFMM_TIMEOUT_OFF);
    return g;
}

LfErr lf_m2l_tc(lfmm_ctx* ctx, cudaStream_t st)
{
    if (ctx->m2l_tc_ntiles == 0) return LfErr();
    const int nb = ctx->nbox_total;
    const int nr = ctx->nrhs_b;
    LF_TRY(split_boxes(ctx, ctx->Mexp.as<float>(), 0, nb, st));
    TcArgs g = tc_args(ctx);
    g.tiles = ctx->m2l_tc_tiles.as<int4>();
    g.sorted = ctx->m2l_sorted.as<int>();
    g.slots = ctx->m2l_slots.as<int>();
    g.cls = ctx->m2l_cls.as<int>();
    g.noff = TC_NOFF;
    g.unit_scale = 0;
    g.A = ctx->m2l_Atc.as<unsigned char>();
    g.L = ctx->Lexp.as<float>();
    // automatic: 7 offsets per accumulator, 3 in the wide form, whose float32
    // accumulation adds twice the MMAs per offset (measured at N = 1M, p = 14:
    // Err2 of the potential 1.18e-6 with 7 offsets, 7.5e-7 with 3, for 1.2 ms more)
    g.groups = ctx->tc_groups > 0 ? ctx->tc_groups : (ctx->m2l_tc_wide ? 63 : 27);
    const int nunits = ctx->m2l_tc_ntiles * g.groups;
    // the persistent form pays off when every SM walks many units; a small
    // tree (or one of many problems sharing the GPU in a batch) keeps one
    // CTA per unit, two of which share an SM
    if (ctx->m2l_tc_wide) {
        ++ctx->launches, k_m2l_tc<true><<<dim3(nunits, nr), TC_THREADS, TC_WIDE_SMEM, st>>>(g);
    } else if (ctx->tc_persistent && nunits * nr >= 4 * ctx->num_sms) {
        // one CTA per SM (shared memory and the 512 tensor-memory columns allow
        // no second); all right-hand sides share the SMs
        int per = std::max(1, ctx->num_sms / std::max(1, nr));
        per = std::min(per, nunits);
        ++ctx->launches, k_m2l_tcp<<<dim3(per, nr), TCP_THREADS, TCP_SMEM, st>>>(g, nunits);
    } else {
        ++ctx->launches, k_m2l_tc<false><<<dim3(nunits, nr), TC_THREADS, TC_SMEM, st>>>(g);
    }
    return lf_cuda(cudaGetLastError(), "m2l tensor-core gemm");
}

// M2M into the parents at `level` (from their children one level down), or
// L2L into the boxes at `level` (from their parents), on the tensor cores:
// the source expansions are split into TF32 pieces first; the products are
// added atomically (M2M into zeroed parents, L2L onto the M2L results).
LfErr lf_shift_tc(lfmm_ctx* ctx, int level, bool l2l, cudaStream_t st)
{
    const int t0 = l2l ? ctx->tc_l2l_first[level] : ctx->tc_m2m_first[level];
    const int t1 = l2l ? ctx->tc_l2l_first[level + 1] : ctx->tc_m2m_first[level + 1];
    if (t1 <= t0) return LfErr();
    if (ctx->m2l_tc_wide) return LfErr("internal: tensor-core translations need (p+1)^2 <= 128");
    const int nr = ctx->nrhs_b, nc = lf_nc(ctx->p);
    const LfmmLevel& src = ctx->levels[l2l ? level - 1 : level + 1];
    TcArgs g;
    if (l2l) {
        LF_TRY(split_boxes(ctx, ctx->Lexp.as<float>(), src.off, src.nbox, st));
        g = tc_args(ctx);
        g.sorted = ctx->m2l_sorted.as<int>();
        g.slots = ctx->box_parent.as<int>();
        g.noff = 1;
        g.A = ctx->l2l_Atc.as<unsigned char>();
        g.L = ctx->Lexp.as<float>();
        g.groups = 1;
    } else {
        LF_TRY(split_boxes(ctx, ctx->Mexp.as<float>(), src.off, src.nbox, st));
        const LfmmLevel& lv = ctx->levels[level];
        const size_t ms = (size_t)ctx->nbox_total * nc;
        LF_CHECK(cudaMemset2DAsync(ctx->Mexp.as<float>() + (size_t)lv.off * nc, ms * sizeof(float), 0,
                                   sizeof(float) * (size_t)lv.nbox * nc, nr, st));
        g = tc_args(ctx);
        g.sorted = nullptr;
        g.slots = ctx->m2m_slots.as<int>();
        g.noff = 8;
        g.A = ctx->m2m_Atc.as<unsigned char>();
        g.L = ctx->Mexp.as<float>();
        g.groups = 8;  // one child octant per CTA, summed by the atomics
    }
    g.tiles = ctx->tc_shift_tiles.as<int4>() + t0;
    g.cls = ctx->shift_cls.as<int>();
    g.unit_scale = 1;
    ++ctx->launches, k_m2l_tc<false><<<dim3((t1 - t0) * g.groups, nr), TC_THREADS, TC_SMEM, st>>>(g);
    return lf_cuda(cudaGetLastError(), l2l ? "l2l tensor-core gemm" : "m2m tensor-core gemm");
}

// Self-check of the bounded-wait path: one thread waits on a barrier that
// expects two arrivals and gets one, so the wait must run out after `limit`
// cycles and count a timeout, exactly as a stalled pipeline stage would.
__global__ void k_wait_probe(long long limit, int* err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_arrive(&bar);
    if (!mbar_wait_for(&bar, 0, limit)) atomicAdd(err, 1);
}

LfErr lf_wait_probe(lfmm_ctx* ctx, double limit_ms, int* timed_out)
{
    int khz = 0;  // SM clock; the GB300's maximum (2.07 GHz) if the runtime does not report it
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device) != cudaSuccess) {
        (void)cudaGetLastError();
        khz = 0;
    }
    if (khz <= 0) khz = 2070000;
    const long long limit = (long long)(limit_ms * (double)khz);
    int* err = reinterpret_cast<int*>(ctx->counts.as<char>() + LFMM_TIMEOUT_OFF);
    LF_CHECK(cudaMemsetAsync(err, 0, sizeof(int), ctx->s_main));
    ++ctx->launches, k_wait_probe<<<1, 32, 0, ctx->s_main>>>(limit, err);
    LF_TRY(lf_cuda(cudaGetLastError(), "wait probe"));
    LF_CHECK(lf_d2h(timed_out, err, sizeof(int), ctx->s_main));
    LF_CHECK(cudaMemsetAsync(err, 0, sizeof(int), ctx->s_main));
    return LfErr();
}

int lf_m2l_tc_tile(const lfmm_ctx* ctx) { return ctx->m2l_tc_wide ? 128 : TC_N; }
