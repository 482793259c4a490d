// lfmm_tree.cu -- octree construction and interaction lists on the device.
//
// Algorithm 1 of the paper starts by forming the polarization coordinates and
// an adaptive tree.  Here every layer's charges live in one global uniform
// grid whose planes contain the interfaces whenever their distances share a
// unit (always for up to three layers), so no box of an aligned level
// straddles an interface, which is the centre condition of eq.
// imagecentercond.  Otherwise a box (of one layer: the layer id is part of
// its key) may straddle an interface; the list test below still requires the
// target and image box centres on their own sides.  Polarization boxes are
// the source boxes mapped by z'' = s z + o (eq. eqpolarizedsource); their
// multipoles are the physical ones up to the sign (-1)^{n+m} of a reflection.  Lists come from a dual
// traversal per level: the candidates of a target box are the children of
// its parent's near list; an admissible candidate (one box of separation,
// sides of the interface respected for reaction components) becomes an M2L
// entry, the rest stay near.  At the leaf level the near list is the P2P
// list (free space) or the near-field Sommerfeld list (reaction).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "lfmm_ctx.h"

#define LF_CHECK(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return lf_cuda(e_, #call); \
    } while (0)
#define LF_TRY(expr)                 \
    do {                             \
        LfErr r_ = (expr);           \
        if (!r_.empty()) return r_;  \
    } while (0)

static inline int lf_blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// Exclusive scan of int32 (block of 512 threads x 4 items, recursive on the
// block sums).
// ---------------------------------------------------------------------------
#define SCAN_T 512
#define SCAN_I 4
#define SCAN_TILE (SCAN_T * SCAN_I)

__global__ void k_scan_tile(const int* in, int* out, int64_t n, int* bsum)  // may run in place
{
    __shared__ int warp_tot[SCAN_T / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)tid * SCAN_I;
    int v[SCAN_I];
    int s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_I; ++j) {
        int x = (base + j < n) ? in[base + j] : 0;
        v[j] = s;
        s += x;
    }
    // inclusive warp scan of thread totals
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = (lane < SCAN_T / 32) ? warp_tot[lane] : 0;
        int ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < SCAN_T / 32) warp_tot[lane] = ti - t;  // exclusive warp offsets
        if (lane == SCAN_T / 32 - 1 && bsum) bsum[blockIdx.x] = ti;
    }
    __syncthreads();
    int off = warp_tot[wid] + incl - s;
#pragma unroll
    for (int j = 0; j < SCAN_I; ++j)
        if (base + j < n) out[base + j] = v[j] + off;
}

__global__ void k_scan_add(int* out, int64_t n, const int* boff)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += boff[i / SCAN_TILE];
}

static LfErr scan_rec(lfmm_ctx* ctx, const int* in, int* out, int64_t n, int* tmp, cudaStream_t st)
{
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb <= 1) {
        ++ctx->launches, k_scan_tile<<<1, SCAN_T, 0, st>>>(in, out, n, nullptr);
        return lf_cuda(cudaGetLastError(), "scan");
    }
    int* bs = tmp;
    int* rest = tmp + nb;
    ++ctx->launches, k_scan_tile<<<(int)nb, SCAN_T, 0, st>>>(in, out, n, bs);
    LF_TRY(lf_cuda(cudaGetLastError(), "scan tile"));
    LF_TRY(scan_rec(ctx, bs, bs, nb, rest, st));
    ++ctx->launches, k_scan_add<<<lf_blocks(n, 256), 256, 0, st>>>(out, n, bs);
    return lf_cuda(cudaGetLastError(), "scan add");
}

LfErr lf_scan_i32(lfmm_ctx* ctx, const int* in, int* out, int64_t n, int64_t* total, cudaStream_t st, int set)
{
    if (n <= 0) {
        if (total) *total = 0;
        return LfErr();
    }
    DevBuf& tmp = set ? ctx->scan_tmp2 : ctx->scan_tmp;
    int64_t need = 0, m = n;
    while (m > 1) {
        m = (m + SCAN_TILE - 1) / SCAN_TILE;
        need += m + 1;
    }
    LF_TRY(lf_reserve(tmp, (size_t)(need + 16) * sizeof(int)));
    // the last input is copied before the scan is enqueued, so in-place scans
    // work (into pinned memory: neither copy waits, one synchronisation)
    int* last = lf_pin<int>(ctx, LFMM_PIN_SCAN + 8 * set);
    if (total) LF_CHECK(cudaMemcpyAsync(last, in + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    LF_TRY(scan_rec(ctx, in, out, n, tmp.as<int>(), st));
    if (total) {
        LF_CHECK(cudaMemcpyAsync(last + 1, out + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        LF_CHECK(cudaStreamSynchronize(st));
        *total = (int64_t)last[1] + last[0];
    }
    return LfErr();
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, value) uint32 pairs, 8 bits per pass.
// ---------------------------------------------------------------------------
#define RS_T 256
#define RS_ROUNDS 8
#define RS_TILE (RS_T * RS_ROUNDS)

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, int* __restrict__ hist,
                             int nblocks)
{
    __shared__ int h[256];
    const int tid = threadIdx.x;
    h[tid] = 0;
    __syncthreads();
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = (int64_t)blockIdx.x * RS_TILE + r * RS_T + tid;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[tid * nblocks + blockIdx.x] = h[tid];
}

__global__ void k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
                                const int* __restrict__ hoff, int nblocks)
{
    __shared__ int s_off[256];
    __shared__ int s_wcnt[RS_T / 32][256];
    __shared__ int s_rtot[256];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    s_off[tid] = hoff[tid * nblocks + blockIdx.x];
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = (int64_t)blockIdx.x * RS_TILE + r * RS_T + tid;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        uint32_t val = valid ? vin[i] : 0u;
        int digit = valid ? (int)((key >> shift) & 255u) : 256;
#pragma unroll
        for (int w = 0; w < RS_T / 32; ++w) s_wcnt[w][tid] = 0;
        __syncthreads();
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        int rank = __popc(peers & ((1u << lane) - 1u));
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) s_wcnt[wid][digit] = __popc(peers);
        __syncthreads();
        {
            int run = 0;
#pragma unroll
            for (int w = 0; w < RS_T / 32; ++w) {
                int t = s_wcnt[w][tid];
                s_wcnt[w][tid] = run;
                run += t;
            }
            s_rtot[tid] = run;
        }
        __syncthreads();
        if (valid) {
            int pos = s_off[digit] + s_wcnt[wid][digit] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        s_off[tid] += s_rtot[tid];
        __syncthreads();
    }
}

// Sorts by the key bits [8 first_pass, 8 (first_pass + npass)); the other
// bits are ignored (stable within equal digits).
LfErr lf_radix_sort(lfmm_ctx* ctx, uint32_t* keys, uint32_t* vals, int64_t n, cudaStream_t st, int first_pass,
                    int npass, int set)
{
    int nb = lf_blocks(n, RS_TILE);
    DevBuf& kt = set ? ctx->keys_tmp2 : ctx->keys_tmp;
    DevBuf& vt = set ? ctx->vals_tmp2 : ctx->vals_tmp;
    DevBuf& ht = set ? ctx->hist2 : ctx->hist;
    LF_TRY(lf_reserve(kt, (size_t)n * 4));
    LF_TRY(lf_reserve(vt, (size_t)n * 4));
    LF_TRY(lf_reserve(ht, (size_t)256 * nb * 4));
    uint32_t *ka = keys, *va = vals, *kb = kt.as<uint32_t>(), *vb = vt.as<uint32_t>();
    int* h = ht.as<int>();
    for (int pass = first_pass; pass < first_pass + npass; ++pass) {
        int shift = 8 * pass;
        ++ctx->launches, k_radix_hist<<<nb, RS_T, 0, st>>>(ka, n, shift, h, nb);
        LF_TRY(lf_cuda(cudaGetLastError(), "radix hist"));
        LF_TRY(lf_scan_i32(ctx, h, h, (int64_t)256 * nb, nullptr, st, set));
        ++ctx->launches, k_radix_scatter<<<nb, RS_T, 0, st>>>(ka, va, kb, vb, n, shift, h, nb);
        LF_TRY(lf_cuda(cudaGetLastError(), "radix scatter"));
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (npass & 1) {  // the result sits in the scratch buffers
        LF_CHECK(cudaMemcpyAsync(keys, ka, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
        LF_CHECK(cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    }
    return LfErr();
}

// ---------------------------------------------------------------------------
// Keys, bounds, depth.
// ---------------------------------------------------------------------------
__global__ void k_bounds(const double* __restrict__ xyz, int64_t n, double* __restrict__ part)
{
    __shared__ double s[6][256];
    const int tid = threadIdx.x;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 3; ++k) {
            double v = xyz[3 * i + k];
            mn[k] = fmin(mn[k], v);
            mx[k] = fmax(mx[k], v);
        }
    for (int k = 0; k < 3; ++k) {
        s[k][tid] = mn[k];
        s[3 + k][tid] = mx[k];
    }
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o)
            for (int k = 0; k < 3; ++k) {
                s[k][tid] = fmin(s[k][tid], s[k][tid + o]);
                s[3 + k][tid] = fmax(s[3 + k][tid], s[3 + k][tid + o]);
            }
        __syncthreads();
    }
    if (tid == 0)
        for (int k = 0; k < 6; ++k) part[blockIdx.x * 6 + k] = s[k][0];
}

struct KeyParams {
    int L;
    int fine;  // fine grid level of the keys (lf_fine_level)
    double d[LFMM_MAXL];
    double org[3];
    double hfine, ihfine;  // fine cell size and its reciprocal
    int iz_lo[LFMM_MAXL + 1], iz_hi[LFMM_MAXL + 1];
};

__global__ void k_make_keys(const double* __restrict__ xyz, const int32_t* __restrict__ layer, int64_t n,
                            KeyParams kp, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                            int* __restrict__ err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    int l = layer[i];
    bool bad = (l < 0 || l > kp.L);
    if (!bad) {
        if (l > 0 && !(z < kp.d[l - 1])) bad = true;
        if (l < kp.L && !(z > kp.d[l])) bad = true;
    }
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
        atomicMin(&err[1], (int)min(i, (int64_t)0x7fffffff));
        atomicOr(&err[0], 2);
        l = 0;
    } else if (bad) {
        atomicMin(&err[1], (int)min(i, (int64_t)0x7fffffff));
        atomicOr(&err[0], 1);
        l = 0;
    }
    // cells by a product with the reciprocal (the FP64 divide is costly): a
    // point within rounding of a cell face may take the cell beside it, which
    // only moves it by that rounding outside its box; across an interface the
    // per-layer clamp of iz decides
    const int top = (1 << kp.fine) - 1;
    int ix = (int)floor((x - kp.org[0]) * kp.ihfine);
    int iy = (int)floor((y - kp.org[1]) * kp.ihfine);
    int iz = (int)floor((z - kp.org[2]) * kp.ihfine);
    ix = min(max(ix, 0), top);
    iy = min(max(iy, 0), top);
    iz = min(max(iz, kp.iz_lo[l]), kp.iz_hi[l]);
    keys[i] = ((uint32_t)l << (3 * kp.fine)) | lf_spread3((uint32_t)ix) | (lf_spread3((uint32_t)iy) << 1) |
              (lf_spread3((uint32_t)iz) << 2);
    vals[i] = (uint32_t)i;
}

__global__ void k_level_counts(const uint32_t* __restrict__ keys, int64_t n, int fine, int* __restrict__ counts)
{
    __shared__ int s[LFMM_FINE_LEVEL + 1];
    if (threadIdx.x <= LFMM_FINE_LEVEL) s[threadIdx.x] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        uint32_t k = keys[i], kp = (i > 0) ? keys[i - 1] : 0u;
        for (int l = 0; l <= fine; ++l) {
            int sh = 3 * (fine - l);
            if (i == 0 || (k >> sh) != (kp >> sh)) atomicAdd(&s[l], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x <= fine && s[threadIdx.x]) atomicAdd(&counts[threadIdx.x], s[threadIdx.x]);
}

__global__ void k_gather_sorted(const double* __restrict__ xyz, const uint32_t* __restrict__ vals, int64_t n,
                                double* __restrict__ xs, double* __restrict__ ys, double* __restrict__ zs,
                                int32_t* __restrict__ perm)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t j = vals[i];
    xs[i] = xyz[3 * (int64_t)j];
    ys[i] = xyz[3 * (int64_t)j + 1];
    zs[i] = xyz[3 * (int64_t)j + 2];
    perm[i] = (int32_t)j;
}

// ---------------------------------------------------------------------------
// Boxes.
// ---------------------------------------------------------------------------

// All levels' boxes from the sorted particle keys in four launches.  A box of
// level l is a run of equal key prefixes key >> 3 (fine - l); the particle
// that starts a box of level l starts one at every finer level too, so one
// number per particle, lev(i) (the coarsest level at which particle i starts
// a box; > depth when it starts none), gives every level's run starts.  Box
// ids: level l holds off[l] .. off[l] + nb[l] - 1 (finest level first), in
// order of their first particles.
#define BX_T 256                  // threads per block
#define BX_E 8                    // consecutive particles per thread
#define BX_TILE (BX_T * BX_E)
#define BX_LV 17                  // levels 0 .. 16
struct BoxLevels {
    int depth, fine;
    int off[BX_LV], nb[BX_LV];
    double h[BX_LV];
};

__device__ __forceinline__ int box_lev(const uint32_t* __restrict__ keys, int64_t i, int fine, int depth)
{
    if (i == 0) return 0;
    const uint32_t x = keys[i] ^ keys[i - 1];
    if (x == 0u) return depth + 1;
    const int hb = 31 - __clz((int)x);
    const int l = max(0, fine - hb / 3);
    return l > depth ? depth + 1 : l;
}

// block-wide exclusive scan of one value per thread (BX_T threads); *total gets the sum
__device__ __forceinline__ int box_scan(int v, int* s_w, int& total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    int base = 0;
    total = 0;
#pragma unroll
    for (int k = 0; k < BX_T / 32; ++k) {
        const int t = s_w[k];
        if (k < w) base += t;
        total += t;
    }
    __syncthreads();
    return base + x - v;
}

// per tile of BX_TILE particles, the number of boxes of each level starting in it
__global__ void __launch_bounds__(BX_T) k_box_tile_counts(const uint32_t* __restrict__ keys, int64_t n, int fine,
                                                          int depth, int* __restrict__ tcnt)
{
    __shared__ int s_c[BX_LV];
    if (threadIdx.x < BX_LV) s_c[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * BX_TILE + (int64_t)threadIdx.x * BX_E;
    int lev[BX_E];
#pragma unroll
    for (int e = 0; e < BX_E; ++e) lev[e] = (i0 + e < n) ? box_lev(keys, i0 + e, fine, depth) : depth + 1;
    for (int l = 0; l <= depth; ++l) {
        int c = 0;
#pragma unroll
        for (int e = 0; e < BX_E; ++e) c += lev[e] <= l;
        c = __reduce_add_sync(0xffffffffu, c);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_c[l], c);
    }
    __syncthreads();
    if (threadIdx.x <= depth) tcnt[(size_t)blockIdx.x * BX_LV + threadIdx.x] = s_c[threadIdx.x];
}

// exclusive scan over the tiles, per level (one block)
__global__ void __launch_bounds__(BX_T) k_box_tile_scan(int* __restrict__ tcnt, int ntile, int depth)
{
    __shared__ int s_w[BX_T / 32];
    for (int l = 0; l <= depth; ++l) {
        int carry = 0;
        for (int t0 = 0; t0 < ntile; t0 += BX_T) {
            const int t = t0 + (int)threadIdx.x;
            const int v = (t < ntile) ? tcnt[(size_t)t * BX_LV + l] : 0;
            int total;
            const int ex = box_scan(v, s_w, total);
            if (t < ntile) tcnt[(size_t)t * BX_LV + l] = carry + ex;
            carry += total;
        }
    }
}

// every box's key, first particle, parent and first child
__global__ void __launch_bounds__(BX_T) k_box_write(const uint32_t* __restrict__ keys, int64_t n, BoxLevels L,
                                                    const int* __restrict__ toff, uint32_t* __restrict__ bkey,
                                                    int* __restrict__ pbeg, int* __restrict__ parent,
                                                    int* __restrict__ cbeg)
{
    __shared__ int s_w[BX_T / 32];
    const int depth = L.depth, fine = L.fine;
    const int64_t i0 = (int64_t)blockIdx.x * BX_TILE + (int64_t)threadIdx.x * BX_E;
    int lev[BX_E];
    int mn = depth + 1;
#pragma unroll
    for (int e = 0; e < BX_E; ++e) {
        lev[e] = (i0 + e < n) ? box_lev(keys, i0 + e, fine, depth) : depth + 1;
        mn = min(mn, lev[e]);
    }
    // base[l]: boxes of level l that start before this thread's particles
    int base[BX_LV];
    for (int l = 0; l <= depth; ++l) {
        int c = 0;
#pragma unroll
        for (int e = 0; e < BX_E; ++e) c += lev[e] <= l;
        int total;
        base[l] = toff[(size_t)blockIdx.x * BX_LV + l] + box_scan(c, s_w, total);
    }
    if (mn > depth) return;  // no box starts here (after the block-wide scans)
#pragma unroll
    for (int e = 0; e < BX_E; ++e) {
        const int le = lev[e];
        if (le > depth) continue;
        // inc[l] = boxes of level l starting at or before particle i0 + e: the
        // counts of levels >= le include this particle
        const uint32_t key = keys[i0 + e];
        for (int l = le; l <= depth; ++l) {
            int inc_l = base[l];
            for (int f = 0; f <= e; ++f) inc_l += lev[f] <= l;
            const int b = L.off[l] + inc_l - 1;
            bkey[b] = key >> (3 * (fine - l));
            pbeg[b] = (int)(i0 + e);
            if (l > 0) {
                int inc_p = base[l - 1];
                for (int f = 0; f <= e; ++f) inc_p += lev[f] <= l - 1;
                parent[b] = L.off[l - 1] + inc_p - 1;
            }
            if (l < depth) {  // the first child starts at the same particle
                int inc_c = base[l + 1];
                for (int f = 0; f <= e; ++f) inc_c += lev[f] <= l + 1;
                cbeg[b] = L.off[l + 1] + inc_c - 1;
            }
        }
    }
}

// per box: particle and child ranges' ends, the roots' parents, leaves'
// child ranges, centres and grid cells
__global__ void k_box_finish(int nbox, int64_t n, BoxLevels L, double ox, double oy, double oz,
                             const uint32_t* __restrict__ bkey, const int* __restrict__ pbeg, int* __restrict__ pend,
                             int* __restrict__ cbeg, int* __restrict__ cend, int* __restrict__ parent,
                             LfD4* __restrict__ cen, int4* __restrict__ grid)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int level = L.depth;
    while (level > 0 && b >= L.off[level - 1]) --level;
    const int i = b - L.off[level];
    const bool last = i + 1 == L.nb[level];
    pend[b] = last ? (int)n : pbeg[b + 1];
    if (level == L.depth) {
        cbeg[b] = -1;
        cend[b] = -1;
    } else {
        cend[b] = last ? L.off[level + 1] + L.nb[level + 1] : cbeg[b + 1];
    }
    if (level == 0) parent[b] = -1;
    const double h = L.h[level];
    const uint32_t k = bkey[b];
    const uint32_t layer = k >> (3 * level);
    const uint32_t mort = (level > 0) ? (k & ((1u << (3 * level)) - 1u)) : 0u;
    const uint32_t ix = lf_compact3(mort), iy = lf_compact3(mort >> 1), iz = lf_compact3(mort >> 2);
    cen[b] = LfD4{ox + (ix + 0.5) * h, oy + (iy + 0.5) * h, oz + (iz + 0.5) * h, (double)layer};
    grid[b] = make_int4((int)ix, (int)iy, (int)iz, (int)layer);
}

// ---------------------------------------------------------------------------
// Lists.
// ---------------------------------------------------------------------------
// The medium as the list kernels see it: the context's components and, per
// (component, level), in units of the level's box size h, with the box
// centre of grid cell i at origin + (i + 1/2) h:
//   K = (o + (s - 1) oz) / h    so that (z_t - z'') / h = (iz_t + 1/2) - s (iz_s + 1/2) - K,
//   F = (iface - oz) / h        so that (z_t - iface) / h = (iz_t + 1/2) - F,
//   G = (s oz + o - iface) / h  so that (z'' - iface) / h = s (iz_s + 1/2) + G,
//   Z = zeta_r / h
// (lc[c * 16 + level]); sep = 1 also requires a centre distance of sqrt(6) boxes.
struct LfListMedium {
    const LfmmComp* comps;
    const float4* lc;
    int sep;
};

// Far-field admissibility of a (target box, source box) pair of one level, in
// grid units.  Free space: not neighbours (|di|_inf >= 2).  Reaction: the
// polarization image of the source box at least 2h away (|.|_inf), target
// and image on their own sides of the interface, and rho <= |dz| + zeta_r.
// At levels where interfaces are grid planes the tested quantities are
// integers or half-integers, so single precision decides them exactly; the
// small margin on the 2h test only matters on coarser levels.
__device__ __forceinline__ bool lf_admissible(const LfmmComp& c, float4 k, int sep, int4 gt, int4 gs)
{
    const int ix = abs(gt.x - gs.x), iy = abs(gt.y - gs.y);
    if (c.is_free) {
        const int iz = abs(gt.z - gs.z);
        if (sep && ix * ix + iy * iy + iz * iz < 6) return false;
        return max(ix, max(iy, iz)) >= 2;
    }
    const float s = (float)c.s;
    const float zt = (float)gt.z + 0.5f, zs = s * ((float)gs.z + 0.5f);
    const float uz = zt - zs - k.x;
    const float ux = (float)ix, uy = (float)iy;
    if (fmaxf(ux, fmaxf(uy, fabsf(uz))) < 2.0f - 1e-3f) return false;
    if (sep && ux * ux + uy * uy + uz * uz < 6.0f - 1e-3f) return false;
    const float tside = zt - k.y, pside = zs + k.z;
    if (c.a == 1) {
        if (!(tside > 0.f && pside < 0.f)) return false;
    } else {
        if (!(tside < 0.f && pside > 0.f)) return false;
    }
    // keep the remainder integral on the real axis (rho <= z + zeta_r)
    if (c.has_rem && sqrtf(ux * ux + uy * uy) > fabsf(uz) + k.w) return false;
    return true;
}

// Where the lists of one level go: entries are appended to the three arrays
// at positions taken from device counters, so no level waits for the host.
struct ListOut {
    uint32_t* near_ent;  // parents' near entries are read from here too
    uint32_t* m2l_ent;
    uint32_t* m2r_ent;
    unsigned* used;      // [0] near, [1] free M2L, [2] reaction M2L entries taken so far
    unsigned cap0, cap1, cap2;
    int* overflow;       // set when an array's capacity would be exceeded (nothing is written past it)
    int *nbeg, *nend, *mbeg, *mend, *rbeg, *rend;
};

// Candidates of the near entries [e0, e0 + 32) of a parent list (ending at
// ee), in slots q = lane + 32 m (m < 8): entry e0 + q / 8, child q mod 8 --
// the order of taking them 4 entries at a time.  Each lane loads one entry and
// its child range, and then the eight child cells of its slots, so a chunk
// costs three rounds of dependent loads rather than three per 4 entries.
// kind: 0 free M2L, 1 reaction M2L, 2 near, -1 no candidate.
__device__ __forceinline__ void list_chunk(const LfListMedium& med, const ListOut& o, int level, int e0, int ee,
                                           int4 gt, const int* __restrict__ cbeg, const int* __restrict__ cend,
                                           const int4* __restrict__ grid, int lane, int kind[8], uint32_t v[8],
                                           int sc[8], int4 gs[8])
{
    const int e = e0 + lane;
    uint32_t ent = 0;
    int cb = 0, ce = 0;
    if (e < ee) {
        ent = o.near_ent[e];
        const int s = (int)(ent & LFMM_ENT_MASK);
        cb = cbeg[s];
        ce = cend[s];
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int src = 4 * m + (lane >> 3);  // lane holding the slot's entry
        const uint32_t en = __shfl_sync(0xffffffffu, ent, src);
        const int b = __shfl_sync(0xffffffffu, cb, src), bend = __shfl_sync(0xffffffffu, ce, src);
        const int ch = b + (lane & 7);
        sc[m] = (e0 + src < ee && ch < bend) ? ch : -1;
        v[m] = (en & ~LFMM_ENT_MASK) | (uint32_t)max(sc[m], 0);
        if (sc[m] >= 0) gs[m] = grid[sc[m]];
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        kind[m] = -1;
        if (sc[m] >= 0) {
            const int c = (int)(v[m] >> LFMM_ENT_SHIFT);
            const LfmmComp& cp = med.comps[c];
            kind[m] = lf_admissible(cp, med.lc[c * 16 + level], med.sep, gt, gs[m]) ? (cp.is_free ? 0 : 1) : 2;
        }
    }
}

// One warp per target box.  The candidates (children of the parent's near
// entries) are taken 32 at a time as 4 entries x 8 child slots.  A first pass
// classifies them (every candidate costs dependent loads: entry, child
// range, child cell) and keeps the accepted ones in candidate order in a
// shared-memory stash of LST_CAP entries per warp; lane 0 then takes
// positions in each array for the counted entries, and the second pass
// copies the stash out through a ballot prefix per category, so each box's
// lists are deterministic (the boxes' segments are placed in whatever order
// the warps reach the counters).  A box with more accepted candidates than
// the stash holds classifies them again in the second pass.  With `slots`,
// the first pass also records each free M2L source at its position in the
// target's octant-class offset list (slots[t][189], inv[class][343]:
// position or -1).
#define LST_WARPS 4
#define LST_CAP 1024
__global__ void __launch_bounds__(32 * LST_WARPS) k_list_level(LfListMedium med, int level_off, int nb, int level,
                                                               const int* __restrict__ parent,
                                                               const int* __restrict__ cbeg, const int* __restrict__ cend,
                                                               const int4* __restrict__ grid, ListOut o,
                                                               unsigned long long* __restrict__ stat,
                                                               const uint32_t* __restrict__ bkey,
                                                               const int* __restrict__ inv, int* __restrict__ slots,
                                                               int* __restrict__ slot_err, int leaf)
{
    __shared__ uint32_t s_v[LST_WARPS][LST_CAP];
    __shared__ unsigned char s_k[LST_WARPS][LST_CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * LST_WARPS + w;
    if (i >= nb) return;  // whole warp
    const int t = level_off + i;
    const int pt = parent[t];
    const int4 gt = grid[t];
    const unsigned lt_mask = (1u << lane) - 1u;
    const int cls = slots ? (int)(bkey[t] & 7u) : 0;
    const int eb = o.nbeg[pt], ee = o.nend[pt];
    int wf = 0, wr = 0, wn = 0;
    int nst = 0;  // accepted candidates (stashed while nst <= LST_CAP)
    if (slots) {
        for (int j = lane; j < 189; j += 32) slots[(size_t)t * 189 + j] = -1;
        __syncwarp();
    }
    for (int pass = 0; pass < 2; ++pass) {
        int nf = 0, nr = 0, nn = 0;  // warp-uniform running counts
        int nrn = 0;                 // leaf level: near entries of reaction components
        if (pass == 1 && nst <= LST_CAP) {
            // copy the stash out, in candidate order within each category
            for (int j0 = 0; j0 < nst; j0 += 32) {
                const int j = j0 + lane;
                const int kind = (j < nst) ? (int)s_k[w][j] : -1;
                const uint32_t v = (j < nst) ? s_v[w][j] : 0u;
                const unsigned bf = __ballot_sync(0xffffffffu, kind == 0);
                const unsigned br = __ballot_sync(0xffffffffu, kind == 1);
                const unsigned bn = __ballot_sync(0xffffffffu, kind == 2);
                if (kind == 0)
                    o.m2l_ent[wf + nf + __popc(bf & lt_mask)] = v;
                else if (kind == 1)
                    o.m2r_ent[wr + nr + __popc(br & lt_mask)] = v;
                else if (kind == 2)
                    o.near_ent[wn + nn + __popc(bn & lt_mask)] = v;
                if (leaf) nrn += __popc(__ballot_sync(0xffffffffu, kind == 2 && !med.comps[v >> LFMM_ENT_SHIFT].is_free));
                nf += __popc(bf);
                nr += __popc(br);
                nn += __popc(bn);
            }
        } else {
            for (int e0 = eb; e0 < ee; e0 += 32) {
                int kinds[8], scs[8];
                uint32_t vs[8];
                int4 gss[8];
                list_chunk(med, o, level, e0, ee, gt, cbeg, cend, grid, lane, kinds, vs, scs, gss);
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int kind = kinds[m];
                    const uint32_t v = vs[m];
                    const unsigned bf = __ballot_sync(0xffffffffu, kind == 0);
                    const unsigned br = __ballot_sync(0xffffffffu, kind == 1);
                    const unsigned bn = __ballot_sync(0xffffffffu, kind == 2);
                    if (pass == 0) {
                        const unsigned ba = bf | br | bn;
                        const int pos = nst + __popc(ba & lt_mask);
                        if (kind >= 0 && pos < LST_CAP) {
                            s_v[w][pos] = v;
                            s_k[w][pos] = (unsigned char)kind;
                        }
                        nst += __popc(ba);
                        if (kind == 0 && slots) {
                            const int4 gs = gss[m];
                            const int ox = gt.x - gs.x, oy = gt.y - gs.y, oz = gt.z - gs.z;
                            int loc = -1;
                            if (ox >= -3 && ox <= 3 && oy >= -3 && oy <= 3 && oz >= -3 && oz <= 3)
                                loc = inv[cls * 343 + (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3)];
                            if (loc < 0)
                                atomicAdd(slot_err, 1);
                            else
                                slots[(size_t)t * 189 + loc] = scs[m];
                        }
                    } else {
                        if (kind == 0)
                            o.m2l_ent[wf + nf + __popc(bf & lt_mask)] = v;
                        else if (kind == 1)
                            o.m2r_ent[wr + nr + __popc(br & lt_mask)] = v;
                        else if (kind == 2)
                            o.near_ent[wn + nn + __popc(bn & lt_mask)] = v;
                        if (leaf)
                            nrn += __popc(__ballot_sync(0xffffffffu,
                                                        kind == 2 && !med.comps[v >> LFMM_ENT_SHIFT].is_free));
                    }
                    nf += __popc(bf);
                    nr += __popc(br);
                    nn += __popc(bn);
                }
            }
        }
        if (pass == 1) {
            if (lane == 0 && stat) {
                if (nf) atomicAdd(&stat[0], (unsigned long long)nf);
                if (nr) atomicAdd(&stat[1], (unsigned long long)nr);
                if (nrn) atomicAdd(&stat[4], (unsigned long long)nrn);
            }
            break;
        }
        __syncwarp();  // the stash is complete before the second pass reads it
        // take the positions, and publish the ranges (empty where an array is full)
        int ok = 0;
        if (lane == 0) {
            wn = (int)atomicAdd(&o.used[0], (unsigned)nn);
            wf = (int)atomicAdd(&o.used[1], (unsigned)nf);
            wr = (int)atomicAdd(&o.used[2], (unsigned)nr);
            ok = (unsigned)wn + nn <= o.cap0 && (unsigned)wf + nf <= o.cap1 && (unsigned)wr + nr <= o.cap2;
            if (!ok) atomicExch(o.overflow, 1);
            o.nbeg[t] = ok ? wn : 0;
            o.nend[t] = ok ? wn + nn : 0;
            o.mbeg[t] = ok ? wf : 0;
            o.mend[t] = ok ? wf + nf : 0;
            o.rbeg[t] = ok ? wr : 0;
            o.rend[t] = ok ? wr + nr : 0;
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) return;  // whole warp
        wn = __shfl_sync(0xffffffffu, wn, 0);
        wf = __shfl_sync(0xffffffffu, wf, 0);
        wr = __shfl_sync(0xffffffffu, wr, 0);
    }
}

// particle-pair statistics of the leaf-level near lists (one warp per leaf,
// lanes over its entries)
__global__ void k_p2p_stats(const LfmmComp* __restrict__ comps, int level_off, int nb, const int* __restrict__ nbeg,
                            const int* __restrict__ nend, const uint32_t* __restrict__ ent,
                            const int* __restrict__ pbeg, const int* __restrict__ pend,
                            unsigned long long* __restrict__ stat)
{
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= nb) return;  // whole warp
    const int t = level_off + i;
    const unsigned long long nt = (unsigned long long)(pend[t] - pbeg[t]);
    unsigned long long f = 0, r = 0;
    for (int e = nbeg[t] + lane; e < nend[t]; e += 32) {
        const uint32_t v = ent[e];
        const int c = (int)(v >> LFMM_ENT_SHIFT);
        const int s = (int)(v & LFMM_ENT_MASK);
        const unsigned long long ns = (unsigned long long)(pend[s] - pbeg[s]);
        if (comps[c].is_free) f += nt * ns; else r += nt * ns;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        f += __shfl_down_sync(0xffffffffu, f, d);
        r += __shfl_down_sync(0xffffffffu, r, d);
    }
    if (lane == 0) {
        if (f) atomicAdd(&stat[2], f);
        if (r) atomicAdd(&stat[3], r);
    }
}

// The particle-pair counts of the last build's leaf-level near lists (free
// and reaction components), computed on request: the build only needs to
// know whether any reaction entry is near.
LfErr lf_p2p_pair_stats(lfmm_ctx* ctx)
{
    if (!ctx->p2p_stats_stale || !ctx->built) return LfErr();
    cudaStream_t st = ctx->s_main;
    const LfmmLevel& lf = ctx->levels[ctx->depth];
    const int nb = ctx->nbox_total;
    unsigned long long* stat = reinterpret_cast<unsigned long long*>(ctx->counts.as<char>() + 20480);
    LF_CHECK(cudaMemsetAsync(stat + 2, 0, 2 * sizeof(unsigned long long), st));
    if (lf.nbox > 0)
        ++ctx->launches, k_p2p_stats<<<lf_blocks(lf.nbox, 8), 256, 0, st>>>(
            ctx->comp_dev.as<LfmmComp>(), lf.off, lf.nbox, ctx->near_off.as<int>(), ctx->near_off.as<int>() + nb,
            ctx->near_ent.as<uint32_t>(), ctx->box_pbeg.as<int>(), ctx->box_pend.as<int>(), stat);
    LF_TRY(lf_cuda(cudaGetLastError(), "p2p stats"));
    unsigned long long* h = lf_pin<unsigned long long>(ctx, LFMM_PIN_LIST);
    LF_CHECK(cudaMemcpyAsync(h, stat + 2, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    LF_CHECK(cudaStreamSynchronize(st));
    ctx->stats[LFMM_STAT_P2P_FREE] = (int64_t)h[0];
    ctx->stats[LFMM_STAT_P2P_REACTION] = (int64_t)h[1];
    ctx->p2p_stats_stale = 0;
    return LfErr();
}

// grow a buffer keeping its first `keep` bytes
static LfErr grow_keep(DevBuf& b, size_t bytes, size_t keep, cudaStream_t st)
{
    if (bytes <= b.cap) return LfErr();
    size_t nc = std::max(bytes, b.cap + b.cap / 2);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, nc);
    if (e != cudaSuccess) return lf_cuda(e, "cudaMalloc (grow)");
    if (keep && b.ptr) {
        e = cudaMemcpyAsync(p, b.ptr, keep, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return lf_cuda(e, "cudaMemcpyAsync (grow)");
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return lf_cuda(e, "sync (grow)");
    }
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = p;
    b.cap = nc;
    return LfErr();
}

// ---------------------------------------------------------------------------
// Host driver.
// ---------------------------------------------------------------------------
LfErr lf_build_tree(lfmm_ctx* ctx, const double* xyz, const int32_t* layer, int64_t n, cudaStream_t st)
{
    if (n > (int64_t)LFMM_ENT_MASK) return "too many charges for this build (max 2^25)";
    // ---- bounds ----
    const int nbb = 256;
    LF_TRY(lf_reserve(ctx->counts, 65536));  // [0,16K) bounds partials, 16K level counts, 20K stats
    // the bounded-wait counter reads zero until an evaluation's waits run out
    // (the buffer may reuse memory that held anything)
    LF_CHECK(cudaMemsetAsync(ctx->counts.as<char>() + LFMM_TIMEOUT_OFF, 0, sizeof(int), st));
    double* part = ctx->counts.as<double>();
    ++ctx->launches, k_bounds<<<nbb, 256, 0, st>>>(xyz, n, part);
    LF_TRY(lf_cuda(cudaGetLastError(), "bounds"));
    static_assert(LFMM_PIN_BOUNDS + 256 * 6 * sizeof(double) <= LFMM_PIN_M2R, "pinned regions");
    const double* hp = lf_pin<double>(ctx, LFMM_PIN_BOUNDS);
    LF_CHECK(cudaMemcpyAsync(lf_pin<double>(ctx, LFMM_PIN_BOUNDS), part, sizeof(double) * 6 * nbb,
                             cudaMemcpyDeviceToHost, st));
    LF_CHECK(cudaStreamSynchronize(st));
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nbb; ++b)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], hp[b * 6 + k]);
            hi[k] = std::max(hi[k], hp[b * 6 + 3 + k]);
        }
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(lo[k]) || !std::isfinite(hi[k])) return "non-finite coordinates";
    double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    ext = std::max(ext, 1e-12) * (1.0 + 1e-9) + 1e-300;

    // ---- grid: interfaces are planes of every level >= the alignment level ----
    // With two or more interfaces whose distances from d0 are multiples of a
    // common unit u (at most 8 units per inner layer), u is the alignment unit;
    // other media get a grid whose cells may straddle an interface (the layer
    // id in the box key keeps the layers apart, and reaction pairs of such
    // boxes fail the side test of the lists and stay in the near field).
    double H, oz;
    double unit = 0.0;
    if (ctx->L >= 2) {
        double dmin = INFINITY;
        for (int j = 1; j < ctx->L; ++j) dmin = std::min(dmin, ctx->d[j - 1] - ctx->d[j]);
        for (int m = 1; m <= 8 && unit == 0.0; ++m) {
            const double u = dmin / m;
            bool ok = true;
            for (int j = 1; j < ctx->L; ++j) {
                const double r = (ctx->d[0] - ctx->d[j]) / u;
                if (fabs(r - std::round(r)) > 1e-9 * r || r > 8.0 * m * ctx->L) ok = false;
            }
            if (ok) unit = u;
        }
    }
    if (unit > 0.0) {
        const double D = unit;
        H = D;
        for (;;) {
            // origin: a multiple of D below d0 such that [oz, oz + H] covers [lo, hi]
            double c = std::ceil((ctx->d[0] - lo[2]) / D - 1e-12);
            if (c < 0) c = 0;
            oz = ctx->d[0] - c * D;
            if (oz > lo[2]) oz -= D;
            if (H >= ext && oz + H > hi[2] + 1e-12 * H) break;
            H *= 2.0;
        }
    } else if (ctx->L == 1) {
        H = 1.0;
        while (H < ext) H *= 2.0;
        while (H * 0.5 >= ext) H *= 0.5;
        // d0 is a plane of every level >= 2
        for (;;) {
            double u = H / 4.0;
            double c = std::ceil((ctx->d[0] - lo[2]) / u - 1e-12);
            if (c < 0) c = 0;
            oz = ctx->d[0] - c * u;
            if (oz > lo[2]) oz -= u;
            if (oz + H > hi[2] + 1e-12 * H) break;
            H *= 2.0;
        }
    } else {
        H = ext * (1.0 + 1e-6);
        oz = lo[2] - 1e-7 * H;
    }
    double pad = 1e-7 * H;
    ctx->H = H;
    ctx->origin[0] = lo[0] - pad;
    ctx->origin[1] = lo[1] - pad;
    ctx->origin[2] = oz;
    if (ctx->origin[0] + H < hi[0] || ctx->origin[1] + H < hi[1]) {
        // widen so the padded box still holds every point
        ctx->H = H = H * 2.0;
    }

    KeyParams kp;
    kp.L = ctx->L;
    const int fine = lf_fine_level(ctx->L);
    kp.fine = fine;
    for (int j = 0; j < LFMM_MAXL; ++j) kp.d[j] = (j < ctx->L) ? ctx->d[j] : 0.0;
    for (int k = 0; k < 3; ++k) kp.org[k] = ctx->origin[k];
    kp.hfine = H / (double)(1 << fine);
    kp.ihfine = 1.0 / kp.hfine;
    const int top = (1 << fine) - 1;
    // fine cells a layer's points may take: interfaces on cell planes (L == 1 or
    // an alignment unit) bound them exactly; otherwise the straddling cells count
    const bool planes = ctx->L == 1 || unit > 0.0;
    for (int l = 0; l <= LFMM_MAXL; ++l) {
        kp.iz_lo[l] = 0;
        kp.iz_hi[l] = top;
        if (l <= ctx->L) {
            if (planes) {
                if (l < ctx->L) kp.iz_lo[l] = std::max(0, (int)std::llround((ctx->d[l] - oz) / kp.hfine));
                if (l > 0) kp.iz_hi[l] = std::min(top, (int)std::llround((ctx->d[l - 1] - oz) / kp.hfine) - 1);
            } else {
                if (l < ctx->L) kp.iz_lo[l] = std::max(0, std::min(top, (int)std::floor((ctx->d[l] - oz) / kp.hfine)));
                if (l > 0) kp.iz_hi[l] = std::max(0, std::min(top, (int)std::floor((ctx->d[l - 1] - oz) / kp.hfine)));
            }
            if (kp.iz_hi[l] < kp.iz_lo[l]) kp.iz_hi[l] = kp.iz_lo[l];
        }
    }

    // ---- keys and sort ----
    LF_TRY(lf_reserve(ctx->keys, (size_t)n * 4));
    LF_TRY(lf_reserve(ctx->vals_tmp, (size_t)n * 4));
    LF_TRY(lf_reserve(ctx->err_flag, 64));
    int init_err[4] = {0, 0x7fffffff, 0, 0};
    LF_CHECK(cudaMemcpyAsync(ctx->err_flag.ptr, init_err, sizeof(init_err), cudaMemcpyHostToDevice, st));
    // values live in idx (uint32)
    LF_TRY(lf_reserve(ctx->idx, (size_t)std::max<int64_t>(n, 1024) * 4));
    uint32_t* keys = ctx->keys.as<uint32_t>();
    uint32_t* vals = ctx->idx.as<uint32_t>();
    ++ctx->launches, k_make_keys<<<lf_blocks(n, 256), 256, 0, st>>>(xyz, layer, n, kp, keys, vals, ctx->err_flag.as<int>());
    LF_TRY(lf_cuda(cudaGetLastError(), "make keys"));
    // the flags come back (into pinned memory, without waiting) with the level
    // counts: a rejected point gets a clamped, valid key, so the sort and the
    // counts below stay in bounds
    int* herr = lf_pin<int>(ctx, LFMM_PIN_ERR);
    LF_CHECK(cudaMemcpyAsync(herr, ctx->err_flag.ptr, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    LF_TRY(lf_radix_sort(ctx, keys, vals, n, st));

    // sorted particle arrays
    LF_TRY(lf_reserve(ctx->xs, (size_t)n * 8));
    LF_TRY(lf_reserve(ctx->ys, (size_t)n * 8));
    LF_TRY(lf_reserve(ctx->zs, (size_t)n * 8));
    LF_TRY(lf_reserve(ctx->perm, (size_t)n * 4));
    ++ctx->launches, k_gather_sorted<<<lf_blocks(n, 256), 256, 0, st>>>(xyz, vals, n, ctx->xs.as<double>(), ctx->ys.as<double>(),
                                                        ctx->zs.as<double>(), ctx->perm.as<int32_t>());
    LF_TRY(lf_cuda(cudaGetLastError(), "gather"));

    // ---- depth ----
    int* cnt = reinterpret_cast<int*>(ctx->counts.as<char>() + 16384);
    LF_CHECK(cudaMemsetAsync(cnt, 0, sizeof(int) * 16, st));
    ++ctx->launches, k_level_counts<<<lf_blocks(n, 256), 256, 0, st>>>(keys, n, fine, cnt);
    LF_TRY(lf_cuda(cudaGetLastError(), "level counts"));
    const int* hc = lf_pin<int>(ctx, LFMM_PIN_LEVELS);
    LF_CHECK(cudaMemcpyAsync(lf_pin<int>(ctx, LFMM_PIN_LEVELS), cnt, sizeof(int) * 16, cudaMemcpyDeviceToHost, st));
    LF_CHECK(cudaStreamSynchronize(st));
    if (herr[0] & 2) {
        char buf[160];
        snprintf(buf, sizeof buf, "EINVAL: non-finite coordinate at charge %d", herr[1]);
        return buf;
    }
    if (herr[0] & 1) {
        char buf[160];
        snprintf(buf, sizeof buf, "EINVAL: charge %d has an invalid layer id or lies outside its layer", herr[1]);
        return buf;
    }

    // the level whose mean leaf occupancy is nearest (in ratio) to half the
    // capacity, among the levels whose mean stays within the capacity
    int depth = fine;
    {
        const double want = 0.5 * ctx->leaf_cap;
        double best = INFINITY;
        for (int l = 0; l <= fine; ++l) {
            const double mean = (double)n / (double)hc[l];
            if (mean > ctx->leaf_cap) continue;
            const double d = fabs(log(mean / want));
            if (d < best) {
                best = d;
                depth = l;
            }
            if (mean < want) break;  // finer levels only move further away
        }
    }
    ctx->depth = depth;
    ctx->levels.assign(depth + 1, LfmmLevel());
    for (int l = 0; l <= depth; ++l) {
        ctx->levels[l].nbox = hc[l];
        ctx->levels[l].h = H / (double)(1 << l);
    }
    // global ids: finest level first
    int tot = 0;
    for (int l = depth; l >= 0; --l) {
        ctx->levels[l].off = tot;
        tot += hc[l];
    }
    ctx->nbox_total = tot;
    if ((int64_t)tot > (int64_t)LFMM_ENT_MASK) return "too many boxes";

    size_t nb = (size_t)tot;
    LF_TRY(lf_reserve(ctx->box_key, nb * 4));
    LF_TRY(lf_reserve(ctx->box_pbeg, nb * 4));
    LF_TRY(lf_reserve(ctx->box_pend, nb * 4));
    LF_TRY(lf_reserve(ctx->box_parent, nb * 4));
    LF_TRY(lf_reserve(ctx->box_cbeg, nb * 4));
    LF_TRY(lf_reserve(ctx->box_cend, nb * 4));
    LF_TRY(lf_reserve(ctx->box_center, nb * sizeof(LfD4)));
    LF_TRY(lf_reserve(ctx->box_grid, nb * sizeof(int4)));
    uint32_t* bkey = ctx->box_key.as<uint32_t>();
    int *pbeg = ctx->box_pbeg.as<int>(), *pend = ctx->box_pend.as<int>(), *par = ctx->box_parent.as<int>();
    int *cbeg = ctx->box_cbeg.as<int>(), *cend = ctx->box_cend.as<int>();
    {
        if (depth >= BX_LV) return "internal: tree deeper than 16 levels";
        BoxLevels bl;
        bl.depth = depth;
        bl.fine = fine;
        for (int l = 0; l < BX_LV; ++l) {
            bl.off[l] = (l <= depth) ? ctx->levels[l].off : 0;
            bl.nb[l] = (l <= depth) ? ctx->levels[l].nbox : 0;
            bl.h[l] = (l <= depth) ? ctx->levels[l].h : 0.0;
        }
        const int ntile = (int)((n + BX_TILE - 1) / BX_TILE);
        LF_TRY(lf_reserve(ctx->flags, (size_t)ntile * BX_LV * sizeof(int) + 64));
        int* tcnt = ctx->flags.as<int>();
        ++ctx->launches, k_box_tile_counts<<<ntile, BX_T, 0, st>>>(keys, n, fine, depth, tcnt);
        ++ctx->launches, k_box_tile_scan<<<1, BX_T, 0, st>>>(tcnt, ntile, depth);
        ++ctx->launches, k_box_write<<<ntile, BX_T, 0, st>>>(keys, n, bl, tcnt, bkey, pbeg, par, cbeg);
        ++ctx->launches, k_box_finish<<<lf_blocks(tot, 256), 256, 0, st>>>(
            tot, n, bl, ctx->origin[0], ctx->origin[1], ctx->origin[2], bkey, pbeg, pend, cbeg, cend, par,
            ctx->box_center.as<LfD4>(), ctx->box_grid.as<int4>());
    }
    LF_TRY(lf_cuda(cudaGetLastError(), "boxes"));
    {
        // per (component, level) constants of the admissibility test
        // host staging owned by the context: the copy needs no synchronisation
        std::vector<float4>& lc = ctx->level_consts_h;
        lc.assign((size_t)LFMM_MAXCOMP * 16, make_float4(0.f, 0.f, 0.f, 0.f));
        const double oz = ctx->origin[2];
        for (int c = 0; c < ctx->ncomp; ++c)
            for (int l = 0; l <= depth && l < 16; ++l) {
                const LfmmComp& cp = ctx->comp[c];
                const double h = ctx->levels[l].h;
                lc[(size_t)c * 16 + l] = make_float4((float)((cp.o + (cp.s - 1.0) * oz) / h), (float)((cp.iface - oz) / h),
                                                     (float)((cp.s * oz + cp.o - cp.iface) / h), (float)(cp.zeta_r / h));
            }
        LF_TRY(lf_reserve(ctx->level_consts, sizeof(float4) * lc.size()));
        LF_CHECK(cudaMemcpyAsync(ctx->level_consts.ptr, lc.data(), sizeof(float4) * lc.size(), cudaMemcpyHostToDevice,
                                 st));
        // the leaf level's image offsets for the float32 near field: exact
        // when every K is an integer (interfaces on leaf grid planes)
        std::vector<float4>& pc = ctx->p2p_consts_h;
        pc.assign((size_t)LFMM_MAXCOMP, make_float4(0.f, 0.f, 0.f, 0.f));
        bool integral = depth < 16;
        const double hl = ctx->levels[depth].h;
        for (int c = 0; c < ctx->ncomp && integral; ++c) {
            const LfmmComp& cp = ctx->comp[c];
            const double K = cp.is_free ? 0.0 : (cp.o + (cp.s - 1.0) * oz) / hl;
            if (!(std::fabs(K - std::nearbyint(K)) <= 1e-9 * (1.0 + std::fabs(K))) || std::fabs(K) > 1e6) integral = false;
            pc[c] = make_float4(cp.is_free ? 1.f : (float)cp.s, (float)std::nearbyint(K), (float)cp.is_free, 0.f);
        }
        ctx->leaf_int_offsets = integral ? 1 : 0;
        if (integral) {
            LF_TRY(lf_reserve(ctx->p2p_consts, sizeof(float4) * pc.size()));
            LF_CHECK(cudaMemcpyAsync(ctx->p2p_consts.ptr, pc.data(), sizeof(float4) * pc.size(),
                                     cudaMemcpyHostToDevice, st));
        }
    }

    // ---- lists ----
    const LfListMedium med{ctx->comp_dev.as<LfmmComp>(), ctx->level_consts.as<float4>(), ctx->sep_ext};
    LF_TRY(lf_reserve(ctx->near_off, nb * 4 * 2));  // beg, end
    LF_TRY(lf_reserve(ctx->m2l_off, nb * 4 * 2));
    LF_TRY(lf_reserve(ctx->m2r_off, nb * 4 * 2));
    int* nbeg = ctx->near_off.as<int>();
    int* nend = nbeg + nb;
    int* mbeg = ctx->m2l_off.as<int>();
    int* mend = mbeg + nb;
    int* rbeg = ctx->m2r_off.as<int>();
    int* rend = rbeg + nb;
    // level 0: near(root_t) = root of the source layer of every component
    int64_t near_used = 0;
    {
        const LfmmLevel& r = ctx->levels[0];
        if (r.nbox > 128) return "internal: more than 128 root boxes";
        const uint32_t* rk = lf_pin<uint32_t>(ctx, LFMM_PIN_ROOT);
        LF_CHECK(cudaMemcpyAsync(lf_pin<uint32_t>(ctx, LFMM_PIN_ROOT), bkey + r.off, 4 * r.nbox, cudaMemcpyDeviceToHost,
                                 st));
        LF_CHECK(cudaStreamSynchronize(st));
        int root_of[LFMM_MAXL + 1];
        for (int l = 0; l <= LFMM_MAXL; ++l) root_of[l] = -1;
        for (int i = 0; i < r.nbox; ++i) root_of[rk[i]] = r.off + i;
        for (int l = 0; l <= LFMM_MAXL; ++l) ctx->nlayer_used[l] = root_of[l] >= 0;
        // staged in the pinned buffer (the bounds region, read long before):
        // the copies are queued without waiting, and the buffer is not
        // written again before the build's final synchronisation
        constexpr int MAXE = 2048;  // root entries: roots x components
        uint32_t* ent = lf_pin<uint32_t>(ctx, LFMM_PIN_UP);
        int* hb = lf_pin<int>(ctx, LFMM_PIN_UP + 4 * MAXE);
        int* he = hb + 128;
        int* zero = he + 128;
        static_assert(4 * MAXE + 3 * 128 * 4 + 8 * 16 <= LFMM_PIN_M2R - LFMM_PIN_UP, "pinned regions");
        int ne = 0;
        for (int i = 0; i < r.nbox; ++i) {
            int tl = (int)rk[i];
            hb[i] = ne;
            zero[i] = 0;
            for (int c = 0; c < ctx->ncomp; ++c) {
                const LfmmComp& cp = ctx->comp[c];
                if (cp.l != tl) continue;
                int src = root_of[cp.lp];
                if (src < 0) continue;
                if (ne >= MAXE) return "internal: too many root list entries";
                ent[ne++] = ((uint32_t)c << LFMM_ENT_SHIFT) | (uint32_t)src;
            }
            he[i] = ne;
        }
        LF_TRY(grow_keep(ctx->near_ent, std::max<size_t>((size_t)ne, 1) * 4, 0, st));
        if (ne > 0) LF_CHECK(cudaMemcpyAsync(ctx->near_ent.ptr, ent, (size_t)ne * 4, cudaMemcpyHostToDevice, st));
        LF_CHECK(cudaMemcpyAsync(nbeg + r.off, hb, 4 * r.nbox, cudaMemcpyHostToDevice, st));
        LF_CHECK(cudaMemcpyAsync(nend + r.off, he, 4 * r.nbox, cudaMemcpyHostToDevice, st));
        LF_CHECK(cudaMemcpyAsync(mbeg + r.off, zero, 4 * r.nbox, cudaMemcpyHostToDevice, st));
        LF_CHECK(cudaMemcpyAsync(mend + r.off, zero, 4 * r.nbox, cudaMemcpyHostToDevice, st));
        LF_CHECK(cudaMemcpyAsync(rbeg + r.off, zero, 4 * r.nbox, cudaMemcpyHostToDevice, st));
        LF_CHECK(cudaMemcpyAsync(rend + r.off, zero, 4 * r.nbox, cudaMemcpyHostToDevice, st));
        near_used = ne;
        ctx->levels[0].near_base = 0;
        ctx->levels[0].near_count = near_used;
    }
    unsigned long long* stat = reinterpret_cast<unsigned long long*>(ctx->counts.as<char>() + 20480);
    // free M2L slot table [box][189] (for the gathered GEMMs), filled with the lists
    int* slot_err = reinterpret_cast<int*>(ctx->counts.as<char>() + 24576);
    const bool want_slots = ctx->m2l_rm > 0 && depth >= 2;
    if (want_slots) LF_TRY(lf_reserve(ctx->m2l_slots, (size_t)nb * 189 * sizeof(int)));
    // list counters [3], overflow flag, and the counters after each level [17][3]
    unsigned* used = reinterpret_cast<unsigned*>(ctx->counts.as<char>() + 28672);
    int* overflow = reinterpret_cast<int*>(used + 3);
    unsigned* snap = used + 4;
    const int64_t nroot = near_used;
    // capacities: the last build's, at least a per-box estimate; one more pass
    // with the measured totals when an array overflows (first builds)
    for (int k = 0; k < 3; ++k)
        if (ctx->list_cap[k] == 0) ctx->list_cap[k] = (int64_t)nb * (k == 0 ? 64 : (k == 1 ? 189 : 16)) + nroot + 1024;
    // read-backs of the list phase, in the pinned buffer
    unsigned long long* hs = lf_pin<unsigned long long>(ctx, LFMM_PIN_LIST);       // 8 statistics
    int* hovp = lf_pin<int>(ctx, LFMM_PIN_LIST + 64);                              // overflow flag
    unsigned* hused = lf_pin<unsigned>(ctx, LFMM_PIN_LIST + 80);                   // 3 counters
    unsigned* hsnap = lf_pin<unsigned>(ctx, LFMM_PIN_LIST + 128);                  // 3 (depth + 1)
    static_assert(LFMM_PIN_LIST + 128 + 3 * 17 * sizeof(unsigned) <= LFMM_PIN_M2L, "pinned regions");
    for (int attempt = 0;; ++attempt) {
        if (ctx->list_cap[0] > 0x7fffffffLL || ctx->list_cap[1] > 0x7fffffffLL || ctx->list_cap[2] > 0x7fffffffLL)
            return "interaction lists too long";
        // the root entries were uploaded to the front of near_ent: keep them if it grows
        LF_TRY(grow_keep(ctx->near_ent, (size_t)ctx->list_cap[0] * 4 + 16, (size_t)nroot * 4, st));
        LF_TRY(lf_reserve(ctx->m2l_ent, (size_t)ctx->list_cap[1] * 4 + 16));
        LF_TRY(lf_reserve(ctx->m2r_ent, (size_t)ctx->list_cap[2] * 4 + 16));
        // one pinned slot per attempt (an attempt's upload may still be queued)
        unsigned* init = lf_pin<unsigned>(ctx, LFMM_PIN_UP + 4 * 2048 + 3 * 128 * 4 + 16 * (attempt % 8));
        init[0] = (unsigned)nroot;
        init[1] = init[2] = init[3] = 0u;
        LF_CHECK(cudaMemcpyAsync(used, init, 4 * sizeof(unsigned), cudaMemcpyHostToDevice, st));
        LF_CHECK(cudaMemsetAsync(stat, 0, 8 * 8, st));
        LF_CHECK(cudaMemsetAsync(slot_err, 0, sizeof(int), st));
        // (the list kernel clears each box's slots of levels >= 2 before filling them)
        ListOut o;
        o.near_ent = ctx->near_ent.as<uint32_t>();
        o.m2l_ent = ctx->m2l_ent.as<uint32_t>();
        o.m2r_ent = ctx->m2r_ent.as<uint32_t>();
        o.used = used;
        o.cap0 = (unsigned)ctx->list_cap[0];
        o.cap1 = (unsigned)ctx->list_cap[1];
        o.cap2 = (unsigned)ctx->list_cap[2];
        o.overflow = overflow;
        o.nbeg = nbeg;
        o.nend = nend;
        o.mbeg = mbeg;
        o.mend = mend;
        o.rbeg = rbeg;
        o.rend = rend;
        LF_CHECK(cudaMemcpyAsync(snap, used, 3 * sizeof(unsigned), cudaMemcpyDeviceToDevice, st));
        for (int l = 1; l <= depth; ++l) {
            const LfmmLevel& lv = ctx->levels[l];
            if (lv.nbox > 0)
                ++ctx->launches, k_list_level<<<lf_blocks(lv.nbox, LST_WARPS), 32 * LST_WARPS, 0, st>>>(
                    med, lv.off, lv.nbox, l, par, cbeg, cend, ctx->box_grid.as<int4>(), o, stat,
                    ctx->box_key.as<uint32_t>(), ctx->m2l_inv.as<int>(),
                    (want_slots && l >= 2) ? ctx->m2l_slots.as<int>() : nullptr, slot_err, l == depth ? 1 : 0);
            LF_CHECK(cudaMemcpyAsync(snap + 3 * l, used, 3 * sizeof(unsigned), cudaMemcpyDeviceToDevice, st));
        }
        LF_TRY(lf_cuda(cudaGetLastError(), "lists"));
        LF_CHECK(cudaMemcpyAsync(hs, stat, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        LF_CHECK(cudaMemcpyAsync(hovp, overflow, sizeof(int), cudaMemcpyDeviceToHost, st));
        LF_CHECK(cudaMemcpyAsync(hused, used, 3 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        LF_CHECK(cudaMemcpyAsync(hsnap, snap, sizeof(unsigned) * 3 * (size_t)(depth + 1), cudaMemcpyDeviceToHost, st));
        LF_CHECK(cudaStreamSynchronize(st));
        if (!*hovp) break;
        if (attempt >= 8) return "internal: interaction lists keep overflowing";
        // the counters kept counting past the capacities, but boxes below a
        // full array found no candidates: grow to at least the counted totals
        // and at least double what overflowed
        for (int k = 0; k < 3; ++k) {
            const int64_t need = (int64_t)hused[k] + hused[k] / 8 + 1024;
            if (need > ctx->list_cap[k]) ctx->list_cap[k] = std::max(need, 2 * ctx->list_cap[k]);
        }
    }
    for (int l = 1; l <= depth; ++l) {
        LfmmLevel& lv = ctx->levels[l];
        const unsigned* a0 = &hsnap[3 * (size_t)(l - 1)];
        const unsigned* a1 = &hsnap[3 * (size_t)l];
        lv.near_base = a0[0];
        lv.near_count = (int64_t)a1[0] - a0[0];
        lv.m2l_base = a0[1];
        lv.m2l_count = (int64_t)a1[1] - a0[1];
        lv.m2r_base = a0[2];
        lv.m2r_count = (int64_t)a1[2] - a0[2];
    }
    ctx->near_total = hsnap[3 * (size_t)depth + 0];
    ctx->m2l_total = hsnap[3 * (size_t)depth + 1];
    ctx->m2r_total = hsnap[3 * (size_t)depth + 2];
    ctx->stats[LFMM_STAT_N] = n;
    ctx->stats[LFMM_STAT_DEPTH] = depth;
    ctx->stats[LFMM_STAT_BOXES] = tot;
    ctx->stats[LFMM_STAT_LEAVES] = ctx->levels[depth].nbox;
    ctx->stats[LFMM_STAT_M2L_FREE] = (int64_t)hs[0];
    ctx->stats[LFMM_STAT_M2L_REACTION] = (int64_t)hs[1];
    // particle-pair counts only on request (lf_p2p_pair_stats); the near field
    // needs to know whether any leaf's near list holds a reaction entry
    ctx->near_reaction_entries = (int64_t)hs[4];
    ctx->p2p_stats_stale = 1;
    ctx->stats[LFMM_STAT_P2P_FREE] = 0;
    ctx->stats[LFMM_STAT_P2P_REACTION] = 0;
    ctx->stats[LFMM_STAT_COMPONENTS] = ctx->ncomp;
    ctx->stats[LFMM_STAT_M2M_EDGES] = tot - ctx->levels[0].nbox;
    ctx->n = n;
    ctx->stats[LFMM_STAT_REACTION_KEYS] = 0;
    // the reaction M2L keys and the near field's relative positions go on the
    // second stream, beside the free M2L classes and slots on this one (their
    // scratch buffers and pinned read-back regions are disjoint)
    cudaStream_t s2 = ctx->s_near;
    LF_CHECK(cudaEventRecord(ctx->ev_fork, st));
    LF_CHECK(cudaStreamWaitEvent(s2, ctx->ev_fork, 0));
    LF_TRY(lf_prepare_m2r(ctx, s2));
    LF_TRY(lf_near_prepare(ctx, s2));
    LF_TRY(lf_prepare_m2l(ctx, st));
    LF_TRY(lf_prepare_m2r_finish(ctx, s2));
    LF_CHECK(cudaEventRecord(ctx->ev_join, s2));
    LF_CHECK(cudaStreamWaitEvent(st, ctx->ev_join, 0));
    return LfErr();
}
