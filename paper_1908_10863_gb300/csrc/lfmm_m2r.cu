// lfmm_m2r.cu -- reaction-component M2L (eqs. metoleimage1, coefintable)
// grouped by geometry key.
//
// On a level whose grid planes contain the interfaces, every polarization
// box is a grid box, so the offset o = (t - P(s))/h of a reaction M2L pair is
// an integer vector in [-3,3]^3.  The translation operator then depends only
// on the key (component, level, offset): the Sommerfeld table of the pair
// (leading image in closed form + Gauss-Laguerre remainder, all (N, mu)) is
// computed once per key at build time, and at evaluation time the pairs of
// one key are applied as batched GEMMs Y = A_key X (X = 64 gathered source
// multipoles), added atomically into the targets' local expansions.  The
// reflection sign (-1)^{n+m} of the multipole (s = -1 maps) and the
// (-1)^{N+mu} of an a = 2 component are folded into A_key.
// Pairs on coarser, non-aligned levels keep the per-pair kernel.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
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

static inline int lf_blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

#define R_TB 64   // pairs per batch
#define R_T 256   // threads: 16 row groups x 16 column groups
#define KEY_NONE 0xffffffffu


// key = level (4 bits) | comp (7 bits) | offset index (12 bits, offsets in
// [-7, 7]^3): sorted keys group a level's keys together, so the keys of the
// levels left to the per-pair kernel are a prefix
#define R_OR 7
#define R_OW (2 * R_OR + 1)
__host__ __device__ __forceinline__ uint32_t rkey(int c, int l, int ox, int oy, int oz)
{
    return ((uint32_t)l << 19) | ((uint32_t)c << 12) | (uint32_t)(((ox + R_OR) * R_OW + (oy + R_OR)) * R_OW + (oz + R_OR));
}
__host__ __device__ __forceinline__ void rkey_decode(uint32_t key, int& c, int& l, int& ox, int& oy, int& oz)
{
    c = (int)((key >> 12) & 127u);
    l = (int)(key >> 19);
    int oi = (int)(key & 4095u);
    ox = oi / (R_OW * R_OW) - R_OR;
    oy = (oi / R_OW) % R_OW - R_OR;
    oz = oi % R_OW - R_OR;
}

// Keys of the reaction M2L entries of one level, from the boxes' grid cells.
// Lateral offsets are exact integers.  The vertical offset of the source's
// polarization image, in box units, (iz_t + 1/2) - s (iz_s + 1/2) - K, is
// n + f with the integer n = iz_t - s iz_s + base and the fraction f fixed per
// (component, level) (0 on levels where the interfaces are grid planes); the
// key holds n, the table is taken at n + f.  An entry outside the key's
// offset range counts in bad[level] (its level then stays per pair).
__global__ void k_m2r_keys(const LfmmComp* __restrict__ comps, int off, int nb, const int4* __restrict__ grid,
                           const int* __restrict__ zbase,
                           const int* __restrict__ rbeg, const int* __restrict__ rend,
                           const uint32_t* __restrict__ rent, int level, uint32_t* __restrict__ keys,
                           uint32_t* __restrict__ vals, int* __restrict__ tgt, int* __restrict__ bad)
{
    // one warp per target box, lanes over its entries
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= nb) return;
    const int t = off + i;
    const int4 gt = grid[t];
    for (int e = rbeg[t] + (threadIdx.x & 31); e < rend[t]; e += 32) {
        uint32_t v = rent[e];
        int c = (int)(v >> LFMM_ENT_SHIFT);
        int s = (int)(v & LFMM_ENT_MASK);
        const LfmmComp& cp = comps[c];
        const int4 gs = grid[s];
        const int sz = cp.s > 0.0 ? 1 : -1;
        const int ox = gt.x - gs.x, oy = gt.y - gs.y, oz = gt.z - sz * gs.z + zbase[c * 16 + level];
        const bool ok = ox >= -R_OR && ox <= R_OR && oy >= -R_OR && oy <= R_OR && oz >= -R_OR && oz <= R_OR;
        if (!ok) atomicAdd(bad + level, 1);
        keys[e] = ok ? rkey(c, level, ox, oy, oz) : KEY_NONE;
        vals[e] = (uint32_t)e;
        tgt[e] = t;
    }
}

__global__ void k_key_flags(const uint32_t* __restrict__ keys, int n, int* __restrict__ f)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    f[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_key_starts(const uint32_t* __restrict__ keys, int n, const int* __restrict__ f,
                             const int* __restrict__ idx, int* __restrict__ kstart, uint32_t* __restrict__ kval)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !f[i]) return;
    kstart[idx[i]] = i;
    kval[idx[i]] = keys[i];
}

// One block per key: the box-unit table (lead + remainder) with the a = 2 sign.
// One Sommerfeld table per (component, level, rho^2, oz): the table depends on
// the lateral distance only; the azimuth enters through the phases applied
// when the operator is assembled.
template <bool GEN>
__global__ void k_m2r_tables(const LfmmComp* __restrict__ comps, const int4* __restrict__ tdesc, int ntab,
                             const double* __restrict__ levelh, const double* __restrict__ zfrac, int P,
                             const double* __restrict__ gt, const double* __restrict__ gw, int Q,
                             double* __restrict__ tables)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TS = 2 * P + 1, TT = TS * TS;
    double* sT = reinterpret_cast<double*>(smem_raw);
    double* sJ = sT + TT;
    double* sA = sJ + Q * TS;
    const int k = blockIdx.x;
    const int4 d = tdesc[k];
    const int c = d.x, l = d.y, oz = d.w;
    const LfmmComp cp = comps[c];
    const double rho = sqrt((double)d.z);
    const double vz = (double)oz + zfrac[c * 16 + l];  // image offset n + f in box units
    const double zz = (cp.a == 1) ? vz : -vz;
    for (int j = threadIdx.x; j < TT; j += blockDim.x) sT[j] = 0.0;
    __syncthreads();
    lf_sommerfeld_table_block<GEN>(cp, rho, zz, levelh[l], 2 * P, sT, TS, Q, gt, gw, sJ, sA);
    double* out = tables + (size_t)k * TT;
    for (int j = threadIdx.x; j < TT; j += blockDim.x) {
        int N = j / TS, mu = j - N * TS;
        double v = (mu <= N) ? sT[j] : 0.0;
        if (cp.a == 2 && ((N + mu) & 1)) v = -v;
        out[j] = v;
    }
}

// ---------------------------------------------------------------------------
// Build-time preparation.
// ---------------------------------------------------------------------------
LfErr lf_prepare_m2r(lfmm_ctx* ctx, cudaStream_t st)
{
    ctx->m2r_nkeys = 0;
    ctx->m2r_nbatch = 0;
    ctx->m2r_ntab = 0;
    ctx->m2r_ops_prec = -1;
    ctx->m2r_dev_pending = 0;
    ctx->stats[LFMM_STAT_REACTION_KEYS] = 0;
    ctx->stats[LFMM_STAT_REACTION_TABLES] = 0;
    ctx->m2r_keyed_from = ctx->depth + 1;
    ctx->m2r_pending_ne = 0;
    ctx->m2r_nent = 0;
    // the keyed GEMM holds a whole operator in shared memory (p <= 10) or
    // stages it in chunks (p <= 15)
    if (ctx->m2l_rm == 0 || ctx->m2l_rm > 16 || ctx->m2r_total == 0) return LfErr();
    // every level with reaction entries is keyed; a level some of whose
    // entries fall outside the key's offset range stays per pair (found at
    // lf_prepare_m2r_finish)
    int la = ctx->depth + 1;
    for (int l = 0; l <= ctx->depth; ++l)
        if (ctx->levels[l].m2r_count > 0) {
            la = l;
            break;
        }
    if (la > ctx->depth) return LfErr();
    ctx->m2r_la = la;
    // per (component, level): the image's vertical offset in box units is
    // iz_t - s iz_s + g with g = (1 - s)/2 - K, K = (o + (s - 1) z0)/h; split
    // as an integer base (for the keys) and a fraction in [0, 1) (for the tables)
    {
        static_assert(LFMM_PIN_M2R + LFMM_MAXCOMP * 16 * (sizeof(double) + sizeof(int)) <= LFMM_PIN_BYTES,
                      "pinned regions");
        double* zf = lf_pin<double>(ctx, LFMM_PIN_M2R);
        int* zb = lf_pin<int>(ctx, LFMM_PIN_M2R + LFMM_MAXCOMP * 16 * sizeof(double));
        for (int c = 0; c < LFMM_MAXCOMP; ++c)
            for (int l = 0; l < 16; ++l) {
                double g = 0.0;
                if (c < ctx->ncomp && l <= ctx->depth) {
                    const LfmmComp& cp = ctx->comp[c];
                    const double K = (cp.o + (cp.s - 1.0) * ctx->origin[2]) / ctx->levels[l].h;
                    g = 0.5 * (1.0 - cp.s) - K;
                }
                const double b = std::floor(g + 1e-9);
                zb[c * 16 + l] = (int)b;
                zf[c * 16 + l] = std::max(0.0, g - b);
            }
        LF_TRY(lf_reserve(ctx->m2r_zfrac, LFMM_MAXCOMP * 16 * sizeof(double)));
        LF_TRY(lf_reserve(ctx->m2r_zbase, LFMM_MAXCOMP * 16 * sizeof(int)));
        LF_CHECK(cudaMemcpyAsync(ctx->m2r_zfrac.ptr, zf, LFMM_MAXCOMP * 16 * sizeof(double), cudaMemcpyHostToDevice, st));
        LF_CHECK(cudaMemcpyAsync(ctx->m2r_zbase.ptr, zb, LFMM_MAXCOMP * 16 * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    int64_t first = -1, last = -1;
    for (int l = la; l <= ctx->depth; ++l) {
        const LfmmLevel& lv = ctx->levels[l];
        if (lv.m2r_count == 0) continue;
        if (first < 0) first = lv.m2r_base;
        last = lv.m2r_base + lv.m2r_count;
    }
    if (first < 0) return LfErr();
    const int ne = (int)(last - first);
    LF_TRY(lf_reserve(ctx->m2r_keys, (size_t)ne * 4 + 16));
    LF_TRY(lf_reserve(ctx->m2r_order, (size_t)ne * 4 + 16));
    LF_TRY(lf_reserve(ctx->m2r_tgt, (size_t)ctx->m2r_total * 4 + 16));
    int* bad = reinterpret_cast<int*>(ctx->counts.as<char>() + 32768);  // [16 levels]
    LF_CHECK(cudaMemsetAsync(bad, 0, 16 * sizeof(int), st));
    // entries of levels la .. depth are contiguous: index them relative to `first`
    uint32_t* keys = ctx->m2r_keys.as<uint32_t>();
    uint32_t* vals = ctx->m2r_order.as<uint32_t>();
    for (int l = la; l <= ctx->depth; ++l) {
        const LfmmLevel& lv = ctx->levels[l];
        if (lv.nbox == 0 || lv.m2r_count == 0) continue;
        ++ctx->launches, k_m2r_keys<<<lf_blocks(lv.nbox, 4), 128, 0, st>>>(
            ctx->comp_dev.as<LfmmComp>(), lv.off, lv.nbox, ctx->box_grid.as<int4>(), ctx->m2r_zbase.as<int>(), ctx->m2r_off.as<int>(),
            ctx->m2r_off.as<int>() + ctx->nbox_total, ctx->m2r_ent.as<uint32_t>(), l, keys - first, vals - first,
            ctx->m2r_tgt.as<int>(), bad);
    }
    LF_TRY(lf_cuda(cudaGetLastError(), "m2r keys"));
    // vals hold absolute entry indices (e), keys sorted ascending
    // keys use bits 0..22 (level << 19 | component << 12 | offset): three digits
    LF_TRY(lf_radix_sort(ctx, keys, vals, ne, st, 0, 3, 1));
    LF_TRY(lf_reserve(ctx->flags, (size_t)ne * 4 + 16));
    LF_TRY(lf_reserve(ctx->idx, (size_t)ne * 4 + 16));
    int* fl = ctx->flags.as<int>();
    int* ix = ctx->idx.as<int>();
    ++ctx->launches, k_key_flags<<<lf_blocks(ne, 256), 256, 0, st>>>(keys, ne, fl);
    // the key count comes back with the last flag and scan value (pinned, no
    // wait here): the key arrays are sized for one key per entry
    int* klast = lf_pin<int>(ctx, LFMM_PIN_SCAN + 8);
    LF_CHECK(cudaMemcpyAsync(klast, fl + ne - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    LF_TRY(lf_scan_i32(ctx, fl, ix, ne, nullptr, st, 1));
    LF_CHECK(cudaMemcpyAsync(klast + 1, ix + ne - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    LF_TRY(lf_reserve(ctx->m2r_kstart, (size_t)(ne + 1) * 4));
    LF_TRY(lf_reserve(ctx->m2r_kval, (size_t)(ne + 1) * 4));
    ++ctx->launches, k_key_starts<<<lf_blocks(ne, 256), 256, 0, st>>>(keys, ne, fl, ix, ctx->m2r_kstart.as<int>(),
                                                                       ctx->m2r_kval.as<uint32_t>());
    LF_TRY(lf_cuda(cudaGetLastError(), "m2r key starts"));
    ctx->m2r_pending_ne = ne;  // the rest (key count, tables, batches) in lf_prepare_m2r_finish
    return LfErr();
}

// After lf_prepare_m2r: wait for its device part on st, read the keys back
// and set up the tables and batches.
LfErr lf_prepare_m2r_finish(lfmm_ctx* ctx, cudaStream_t st)
{
    const int ne = ctx->m2r_pending_ne;
    ctx->m2r_nent = ne;
    if (ne <= 0) return LfErr();
    ctx->m2r_pending_ne = 0;
    LF_CHECK(cudaStreamSynchronize(st));
    const int* klast = lf_pin<int>(ctx, LFMM_PIN_SCAN + 8);
    const int64_t nk = (int64_t)klast[0] + klast[1];
    int* bad = reinterpret_cast<int*>(ctx->counts.as<char>() + 32768);
    // key starts, key values and the per-level range counts come back into
    // the pinned buffer when they fit (one synchronisation), else into host
    // vectors (the pinned region's staged uploads are complete by now)
    const size_t pin_need = sizeof(int) * (2 * (size_t)nk + 17);
    const bool pinned = LFMM_PIN_M2R + pin_need <= LFMM_PIN_BYTES;
    std::vector<int>& kst_h = ctx->m2r_kstart_h;
    std::vector<uint32_t>& kv_h = ctx->m2r_kval_h;
    if (!pinned) {
        kst_h.resize(nk + 1);
        kv_h.resize(nk);
    }
    int* kstart = pinned ? lf_pin<int>(ctx, LFMM_PIN_M2R) : kst_h.data();
    uint32_t* kv = pinned ? lf_pin<uint32_t>(ctx, LFMM_PIN_M2R + sizeof(int) * (nk + 1)) : kv_h.data();
    int* hbad = pinned ? lf_pin<int>(ctx, LFMM_PIN_M2R + sizeof(int) * (2 * (size_t)nk + 1))
                       : lf_pin<int>(ctx, LFMM_PIN_SCAN + 16);
    LF_CHECK(cudaMemcpyAsync(kstart, ctx->m2r_kstart.ptr, sizeof(int) * nk, cudaMemcpyDeviceToHost, st));
    LF_CHECK(cudaMemcpyAsync(kv, ctx->m2r_kval.ptr, sizeof(uint32_t) * nk, cudaMemcpyDeviceToHost, st));
    LF_CHECK(cudaMemcpyAsync(hbad, bad, 16 * sizeof(int), cudaMemcpyDeviceToHost, st));
    LF_CHECK(cudaStreamSynchronize(st));
    kstart[nk] = ne;
    // levels from keyed_from on are keyed: below it, a level with an entry
    // outside the key range (and every coarser one) stays per pair.  Their
    // keys (sorted by level first) are a prefix, and the out-of-range ones
    // (KEY_NONE) the suffix
    int keyed_from = ctx->m2r_la;
    for (int l = ctx->m2r_la; l <= ctx->depth && l < 16; ++l)
        if (hbad[l] > 0) keyed_from = l + 1;
    ctx->m2r_keyed_from = keyed_from;
    int64_t k0 = 0, k1 = nk;
    while (k0 < nk && (int)(kv[k0] >> 19) < keyed_from) ++k0;  // (KEY_NONE >> 19 exceeds every level)
    while (k1 > k0 && kv[k1 - 1] == KEY_NONE) --k1;
    const int64_t nku = k1 - k0;
    ctx->m2r_kfirst = (int)k0;
    if (nku <= 0) return LfErr();
    // tables, one per distinct (component, level, rho^2, oz)
    std::vector<int4>& tdesc = ctx->m2r_tdesc_h;
    std::vector<int>& ktab = ctx->m2r_ktab_h;
    tdesc.clear();
    ktab.assign(nku, 0);
    {
        // keys arrive sorted by (component, level, offset): within one
        // (component, level) run a table is identified by (rho^2, oz), looked
        // up in a direct-indexed slot array (a generation stamp instead of
        // clearing it per run); tables are numbered in order of first use
        constexpr int NR2 = 2 * R_OR * R_OR + 1;
        std::vector<int>& slot = ctx->m2r_slot_h;
        std::vector<uint32_t>& stamp = ctx->m2r_stamp_h;
        slot.assign((size_t)NR2 * R_OW, 0);
        stamp.assign((size_t)NR2 * R_OW, 0u);
        uint32_t gen = 0, run = ~0u;
        for (int64_t k = k0; k < k1; ++k) {
            int c, l, ox, oy, oz;
            rkey_decode(kv[k], c, l, ox, oy, oz);
            if ((kv[k] >> 12) != run) {
                run = kv[k] >> 12;
                ++gen;
            }
            const int r2 = ox * ox + oy * oy;
            const size_t i = (size_t)r2 * R_OW + (oz + R_OR);
            if (stamp[i] != gen) {
                stamp[i] = gen;
                slot[i] = (int)tdesc.size();
                tdesc.push_back(make_int4(c, l, r2, oz));
            }
            ktab[k - k0] = slot[i];
        }
    }
    const int ntab = (int)tdesc.size();
    const int P = ctx->p, TS = 2 * P + 1, TT = TS * TS, Q = ctx->gl_q_m2l;
    LF_TRY(lf_reserve(ctx->m2r_tables, (size_t)ntab * TT * 8 + 16));
    LF_TRY(lf_reserve(ctx->m2r_tdesc, (size_t)ntab * sizeof(int4) + 16));
    LF_TRY(lf_reserve(ctx->m2r_ktab, (size_t)nku * sizeof(int) + 16));
    LF_CHECK(cudaMemcpyAsync(ctx->m2r_tdesc.ptr, tdesc.data(), ntab * sizeof(int4), cudaMemcpyHostToDevice, st));
    LF_CHECK(cudaMemcpyAsync(ctx->m2r_ktab.ptr, ktab.data(), nku * sizeof(int), cudaMemcpyHostToDevice, st));
    double* hl = ctx->m2r_levelh_h;
    for (int l = 0; l < 16; ++l) hl[l] = (l <= ctx->depth) ? ctx->levels[l].h : 0.0;
    LF_TRY(lf_reserve(ctx->m2r_levelh, sizeof(double) * 16));
    LF_CHECK(cudaMemcpyAsync(ctx->m2r_levelh.ptr, hl, sizeof(double) * 16, cudaMemcpyHostToDevice, st));
    (void)P;
    (void)Q;
    ctx->m2r_ntab = ntab;
    // batches of R_TB pairs of one key: key index, first sorted entry, count | key << 8, table
    std::vector<int4>& batches = ctx->m2r_batches_h;
    batches.clear();
    for (int64_t k = k0; k < k1; ++k)
        for (int s = kstart[k]; s < kstart[k + 1]; s += R_TB)
            batches.push_back(make_int4((int)(k - k0), s, std::min(R_TB, kstart[k + 1] - s) | (int)(kv[k] << 8),
                                        ktab[k - k0]));
    ctx->m2r_nkeys = (int)nku;
    ctx->m2r_nbatch = (int)batches.size();
    LF_TRY(lf_reserve(ctx->m2r_batches, batches.size() * sizeof(int4) + 16));
    LF_CHECK(cudaMemcpyAsync(ctx->m2r_batches.ptr, batches.data(), batches.size() * sizeof(int4),
                             cudaMemcpyHostToDevice, st));
    // (the host staging vectors live in the context; the build synchronises at its end)
    ctx->stats[LFMM_STAT_REACTION_KEYS] = nku;
    ctx->stats[LFMM_STAT_REACTION_TABLES] = ntab;
    // the tables and operators themselves are device work of the first
    // evaluation after this build (lf_m2r_device), beside its upward pass
    ctx->m2r_dev_pending = 1;
    return LfErr();
}

// Sommerfeld tables of the keys (FP64) and the keys' operators in the
// current precision, enqueued on `st` (the first evaluation after a build
// runs this on the near-field stream, so it overlaps the far field's upward
// pass and free M2L; the reaction M2L waits for it).
// (source box, target box) of every reaction M2L entry in key order
__global__ void k_m2r_pairs(const uint32_t* __restrict__ order, const uint32_t* __restrict__ ent,
                            const int* __restrict__ tgt, int ne, int2* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const uint32_t e = order[i];
    out[i] = make_int2((int)(ent[e] & LFMM_ENT_MASK), tgt[e]);
}

LfErr lf_m2r_device(lfmm_ctx* ctx, cudaStream_t st)
{
    if (ctx->m2r_nbatch == 0 || ctx->m2r_ntab == 0) {
        ctx->m2r_dev_pending = 0;
        return LfErr();
    }
    const int ntab = ctx->m2r_ntab;
    const int P = ctx->p, TS = 2 * P + 1, TT = TS * TS, Q = ctx->gl_q_m2l;
    size_t sm = sizeof(double) * ((size_t)TT + 2 * (size_t)Q * TS);
    auto tabk = (ctx->L >= 3) ? k_m2r_tables<true> : k_m2r_tables<false>;
    LF_CHECK(cudaFuncSetAttribute(tabk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    ++ctx->launches, tabk<<<ntab, 128, sm, st>>>(ctx->comp_dev.as<LfmmComp>(), ctx->m2r_tdesc.as<int4>(), ntab,
                                                 ctx->m2r_levelh.as<double>(), ctx->m2r_zfrac.as<double>(), P,
                                                 ctx->gl_t_m2l.as<double>(),
                                                 ctx->gl_w_m2l.as<double>(), Q, ctx->m2r_tables.as<double>());
    LF_TRY(lf_cuda(cudaGetLastError(), "m2r tables"));
    if (ctx->m2r_nent > 0) {
        LF_TRY(lf_reserve(ctx->m2r_pairs, (size_t)ctx->m2r_nent * sizeof(int2) + 16));
        ++ctx->launches, k_m2r_pairs<<<lf_blocks(ctx->m2r_nent, 256), 256, 0, st>>>(
            ctx->m2r_order.as<uint32_t>(), ctx->m2r_ent.as<uint32_t>(), ctx->m2r_tgt.as<int>(), ctx->m2r_nent,
            ctx->m2r_pairs.as<int2>());
        LF_TRY(lf_cuda(cudaGetLastError(), "m2r pairs"));
    }
    LF_TRY(lf_m2r_ops(ctx, st));
    ctx->m2r_dev_pending = 0;  // only once both are enqueued
    return LfErr();
}

// ---------------------------------------------------------------------------
// Evaluation: one operator per key (assembled once per build and precision),
// then batched GEMMs with atomic accumulation.
// ---------------------------------------------------------------------------
struct ROpArgs {
    int p, nc;
    const uint32_t* kval;
    const double* tables;   // one per (component, level, rho^2, oz)
    const int* ktab;        // table of each key
    const LfmmComp* comps;  // the context's components
    void* ops;              // [nkeys][RP][RP]: A_key[k_in][r_out], zero padded
};

// One block per key: A_key from its table, the lateral phases e^{i mu phi}
// and the signs (eq. coefintable with the reflection of the multipole).
template <typename R, int RP>
__global__ void __launch_bounds__(R_T) k_m2r_ops(ROpArgs g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = g.p, nc = g.nc, TS = 2 * p + 1;
    R* sT = reinterpret_cast<R*>(smem_raw);  // [TS*TS]
    R* sC = sT + TS * TS;                    // cos(m phi), m <= 2p
    R* sS = sC + TS;
    __shared__ unsigned char s_n[RP], s_m[RP], s_im[RP];  // (n, m, imaginary part) of each packed index
    const int tid = threadIdx.x;
    const int kidx = blockIdx.x;
    if (tid < RP) {
        int n = 0, m = 0, im = 0;
        if (tid < nc) lf_decode(p, tid, n, m, im);
        s_n[tid] = (unsigned char)n;
        s_m[tid] = (unsigned char)m;
        s_im[tid] = (unsigned char)im;
    }
    int c, lev, ox, oy, oz;
    rkey_decode(g.kval[kidx], c, lev, ox, oy, oz);
    (void)lev;
    (void)oz;
    const LfmmComp& cp = g.comps[c];
    const double phi = (ox == 0 && oy == 0) ? 0.0 : atan2((double)oy, (double)ox);
    if (tid < TS) {
        double sn, cs;
        sincos(tid * phi, &sn, &cs);
        sC[tid] = (R)cs;
        sS[tid] = (R)sn;
    }
    const double* Tk = g.tables + (size_t)g.ktab[kidx] * TS * TS;
    for (int j = tid; j < TS * TS; j += R_T) sT[j] = (R)Tk[j];
    __syncthreads();
    R* A = reinterpret_cast<R*>(g.ops) + (size_t)kidx * RP * RP;
    for (int idx = tid; idx < RP * RP; idx += R_T) {
        const int kin = idx / RP, rout = idx - kin * RP;
        R v = 0;
        if (kin < nc && rout < nc) {
            const int n = s_n[kin], mp = s_m[kin], bim = s_im[kin];
            const int k = s_n[rout], l = s_m[rout], aim = s_im[rout];
            // T_N^mu (complex) = e^{i mu phi} T(N, |mu|) with T_N^{-mu} = (-1)^mu conj
            const int N = n + k;
            const int mu1 = mp + l;
            const R c1 = sT[N * TS + mu1] * sC[mu1], d1 = sT[N * TS + mu1] * sS[mu1];
            R c2 = 0, d2 = 0, sg = 0;
            if (mp > 0) {
                const int mu2 = l - mp, a2 = mu2 < 0 ? -mu2 : mu2;
                const R tv = sT[N * TS + a2];
                c2 = tv * sC[a2];
                d2 = tv * sS[a2];
                if (mu2 < 0) {
                    if (a2 & 1) c2 = -c2; else d2 = -d2;
                }
                sg = (mp & 1) ? R(-1) : R(1);
            }
            const R sk = (k & 1) ? R(-1) : R(1);
            if (!aim && !bim) v = sk * (c1 + sg * c2);
            else if (!aim && bim) v = sk * (-d1 + sg * d2);
            else if (aim && !bim) v = sk * (d1 + sg * d2);
            else v = sk * (c1 - sg * c2);
            if (cp.refl && ((n + mp) & 1)) v = -v;
        }
        A[idx] = v;
    }
}

struct RGemmArgs {
    int p, nc;
    const int4* batches;    // key, first sorted entry, count
    const uint32_t* kval;
    const void* ops;        // [nkeys][RP][RP]
    const uint32_t* order;  // sorted entry indices
    const uint32_t* ent;    // m2r entries (component | source box)
    const int* tgt;         // target box per entry
    const double* levelh;
    const void* M;
    void* L;
    size_t stride;          // expansions per right-hand side, in elements
    int nr;                 // right-hand sides, applied in turn with the operator staged once
};

// Y = A X over the first 4 * CG columns (CG column groups of 4; the rest of
// the 256 threads split the RP rows), scaled by 1/h and added into the
// targets' local expansions.
template <typename R, int RP, int CG>
__device__ __forceinline__ void m2r_tile(const R* __restrict__ sA, const R* __restrict__ sX, int cnt,
                                         const int* s_tgt, R ih, R* __restrict__ L, int nc)
{
    constexpr int KP = RP, XS = KP + 1;
    constexpr int RG = R_T / CG;  // row groups
    constexpr int RM = RP / RG;   // rows per thread
    static_assert(RM >= 1 && RM * RG == RP, "tile shape");
    const int tid = threadIdx.x;
    const int cg = tid % CG, rg = tid / CG;
    R acc[RM][4];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = 0;
#pragma unroll 4
    for (int kk = 0; kk < KP; ++kk) {
        R a[RM];
#pragma unroll
        for (int r = 0; r < RM; ++r) a[r] = sA[kk * RP + rg * RM + r];
        R x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = sX[(4 * cg + q) * XS + kk];
#pragma unroll
        for (int r = 0; r < RM; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] += a[r] * x[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = 4 * cg + q;
        if (j >= cnt) continue;
        R* Lt = L + (size_t)s_tgt[j] * nc;
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            const int row = rg * RM + r;
            if (row < nc) atomicAdd(Lt + row, acc[r][q] * ih);
        }
    }
}

// One block per batch of up to R_TB pairs of one key.
template <typename R, int RP>
__global__ void __launch_bounds__(R_T) k_m2r_gemm(RGemmArgs g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int KP = RP;
    constexpr int XS = KP + 1;
    constexpr int CG_MIN = (R_T / RP) > 4 ? (R_T / RP) : 4;  // at least one row per thread
    const int nc = g.nc;
    R* sA = reinterpret_cast<R*>(smem_raw);  // [KP][RP]
    R* sX = sA + KP * RP;                    // [R_TB][XS]
    __shared__ int s_src[R_TB], s_tgt[R_TB];
    const int tid = threadIdx.x;
    const int4 b = g.batches[blockIdx.x];
    const int kidx = b.x, start = b.y, cnt = b.z & 255;
    int c, lev, ox, oy, oz;
    rkey_decode(g.kval[kidx], c, lev, ox, oy, oz);
    // the key's operator: a contiguous copy in 16-byte pieces
    {
        const float4* src = reinterpret_cast<const float4*>(reinterpret_cast<const R*>(g.ops) +
                                                            (size_t)kidx * KP * RP);
        float4* dst = reinterpret_cast<float4*>(sA);
        constexpr int NV = KP * RP * (int)sizeof(R) / 16;
        for (int i = tid; i < NV; i += R_T) dst[i] = src[i];
    }
    if (tid < R_TB) {
        if (tid < cnt) {
            const uint32_t e = g.order[start + tid];
            s_src[tid] = (int)(g.ent[e] & LFMM_ENT_MASK);
            s_tgt[tid] = g.tgt[e];
        } else {
            s_src[tid] = -1;
            s_tgt[tid] = -1;
        }
    }
    __syncthreads();
    // columns the tile shape below reads (block-uniform)
    const int cgs = cnt > 32 ? 16 : (cnt > 16 ? 8 : 4);
    const int ncol = 4 * (cgs > CG_MIN ? cgs : CG_MIN);
    const R ih = (R)(1.0 / g.levelh[lev]);
    const int tot = ncol * KP;
    for (int r = 0; r < g.nr; ++r) {
        if (r > 0) __syncthreads();  // the previous vector's products are read out of sX
        const R* M = reinterpret_cast<const R*>(g.M) + (size_t)r * g.stride;
        // eight loads in flight per thread before their stores
        for (int b0 = tid; b0 < tot; b0 += 8 * R_T) {
            R v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = b0 + u * R_T;
                v[u] = R(0);
                if (idx < tot) {
                    const int j = idx / KP, k = idx - j * KP;
                    const int s = s_src[j];
                    if (s >= 0 && k < nc) v[u] = M[(size_t)s * nc + k];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = b0 + u * R_T;
                if (idx < tot) {
                    const int j = idx / KP, k = idx - j * KP;
                    sX[j * XS + k] = v[u];
                }
            }
        }
        __syncthreads();
        R* L = reinterpret_cast<R*>(g.L) + (size_t)r * g.stride;
        if (cgs == 16 || CG_MIN >= 16)
            m2r_tile<R, RP, 16>(sA, sX, cnt, s_tgt, ih, L, nc);
        else if (cgs == 8 || CG_MIN >= 8)
            m2r_tile<R, RP, (CG_MIN > 8 ? CG_MIN : 8)>(sA, sX, cnt, s_tgt, ih, L, nc);
        else
            m2r_tile<R, RP, CG_MIN>(sA, sX, cnt, s_tgt, ih, L, nc);
    }
}

// Orders 11 .. 15 ((p+1)^2 up to 256): the key's operator is too large for
// shared memory, so it is staged in chunks of R_KC input rows while the
// gathered multipoles stay resident; the same tile shapes as m2r_tile.
#define R_KC 32

template <typename R, int RP, int CG>
__device__ __forceinline__ void m2r_tile_kc(const R* __restrict__ A, R* __restrict__ sA, const R* __restrict__ sX,
                                            int cnt, const int* s_tgt, R ih, R* __restrict__ L, int nc)
{
    constexpr int KP = RP, XS = KP + 1;
    constexpr int RG = R_T / CG;  // row groups
    constexpr int RM = RP / RG;   // rows per thread
    static_assert(RM >= 1 && RM * RG == RP, "tile shape");
    const int tid = threadIdx.x;
    const int cg = tid % CG, rg = tid / CG;
    R acc[RM][4];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = 0;
    for (int kc = 0; kc < KP; kc += R_KC) {
        __syncthreads();  // the previous chunk has been read
        {
            const float4* src = reinterpret_cast<const float4*>(A + (size_t)kc * RP);
            float4* dst = reinterpret_cast<float4*>(sA);
            constexpr int NV = R_KC * RP * (int)sizeof(R) / 16;
            for (int i = tid; i < NV; i += R_T) dst[i] = src[i];
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < R_KC; ++kk) {
            R a[RM];
#pragma unroll
            for (int r = 0; r < RM; ++r) a[r] = sA[kk * RP + rg * RM + r];
            R x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = sX[(4 * cg + q) * XS + kc + kk];
#pragma unroll
            for (int r = 0; r < RM; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] += a[r] * x[q];
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = 4 * cg + q;
        if (j >= cnt) continue;
        R* Lt = L + (size_t)s_tgt[j] * nc;
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            const int row = rg * RM + r;
            if (row < nc) atomicAdd(Lt + row, acc[r][q] * ih);
        }
    }
}

template <typename R, int RP>
__global__ void __launch_bounds__(R_T) k_m2r_gemm_kc(RGemmArgs g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int KP = RP;
    constexpr int XS = KP + 1;
    const int nc = g.nc;
    R* sA = reinterpret_cast<R*>(smem_raw);  // [R_KC][RP]
    R* sX = sA + R_KC * RP;                  // [R_TB][XS]
    __shared__ int s_src[R_TB], s_tgt[R_TB];
    const int tid = threadIdx.x;
    const int4 b = g.batches[blockIdx.x];
    const int kidx = b.x, start = b.y, cnt = b.z & 255;
    int c, lev, ox, oy, oz;
    rkey_decode(g.kval[kidx], c, lev, ox, oy, oz);
    const R* A = reinterpret_cast<const R*>(g.ops) + (size_t)kidx * KP * RP;
    if (tid < R_TB) {
        if (tid < cnt) {
            const uint32_t e = g.order[start + tid];
            s_src[tid] = (int)(g.ent[e] & LFMM_ENT_MASK);
            s_tgt[tid] = g.tgt[e];
        } else {
            s_src[tid] = -1;
            s_tgt[tid] = -1;
        }
    }
    __syncthreads();
    const int cgs = cnt > 32 ? 16 : (cnt > 16 ? 8 : 4);
    const int ncol = 4 * cgs;
    const R ih = (R)(1.0 / g.levelh[lev]);
    const int tot = ncol * KP;
    for (int r = 0; r < g.nr; ++r) {
        if (r > 0) __syncthreads();  // the previous vector's products are read out of sX
        const R* M = reinterpret_cast<const R*>(g.M) + (size_t)r * g.stride;
        for (int b0 = tid; b0 < tot; b0 += 8 * R_T) {
            R v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = b0 + u * R_T;
                v[u] = R(0);
                if (idx < tot) {
                    const int j = idx / KP, k = idx - j * KP;
                    const int s = s_src[j];
                    if (s >= 0 && k < nc) v[u] = M[(size_t)s * nc + k];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = b0 + u * R_T;
                if (idx < tot) {
                    const int j = idx / KP, k = idx - j * KP;
                    sX[j * XS + k] = v[u];
                }
            }
        }
        R* L = reinterpret_cast<R*>(g.L) + (size_t)r * g.stride;
        if (cgs == 16)
            m2r_tile_kc<R, RP, 16>(A, sA, sX, cnt, s_tgt, ih, L, nc);
        else if (cgs == 8)
            m2r_tile_kc<R, RP, 8>(A, sA, sX, cnt, s_tgt, ih, L, nc);
        else
            m2r_tile_kc<R, RP, 4>(A, sA, sX, cnt, s_tgt, ih, L, nc);
    }
}

// ---------------------------------------------------------------------------
// Tensor-core form (float32, (p+1)^2 <= 128): one CTA per batch of up to
// R_TB pairs of one key.  The key's operator is never stored: the CTA forms
// it in shared memory from the key's Sommerfeld table and the lateral phases
// (the same entries as k_m2r_ops), directly as two TF32 pieces a1 + a2 in the
// 64-byte-swizzled K-major layout of the MMA's A operand (M = 128 output
// coefficients, K = the input coefficients in chunks of 16).  The batch's
// source multipoles (B operand: N = the batch rounded up to 16 columns) are
// loaded into registers up front and split the same way.  K runs in rounds
// of RT_KQ chunks through two buffers: while the tensor cores take one round
// (3xTF32: a1 x1 + a1 x2 + a2 x1, issued by one thread into one accumulator
// of 64 tensor-memory columns), the threads form the next.  The operator
// entries come from a table of the reaction coefficient extended to negative
// orders, so each is two shared-memory loads and a fused multiply-add with
// signs and offsets precomputed per output row and input coefficient.  Each
// batch carries its key and table index, so one dependent load reaches the
// table, the phases and the batch's (source, target) pairs.  With 61 KB of
// shared memory the kernel shares its SMs with the near field that runs
// beside it.  The eight warps then read the accumulator back (warp w:
// lanes 32 (w mod 4) .., columns 32 (w / 4) ..), scale it by 1/h and add it
// into the targets' local expansions.  Several right-hand sides repeat the
// rounds per vector.  Every wait is bounded: on a timeout the CTA counts it
// in err and skips its read-backs.
// ---------------------------------------------------------------------------
#define RT_THREADS 256
#define RT_TS 21                        // table side 2p + 1 for p <= 10
#define RT_WS 41                        // 4p + 1: orders -2p .. 2p
// one K chunk per round and three CTAs per SM (61 KB of shared memory, 64
// registers each) measured 0.26 ms at N = 1M, p = 10, against 0.31 ms for
// rounds of two chunks at two CTAs per SM
#ifndef RT_KQ
#define RT_KQ 1                         // K chunks per round
#endif
#ifndef RT_MINB
#define RT_MINB 3                       // resident CTAs per SM
#endif
#define RT_A_CHUNK (128 * TC_ROWB)      // one K chunk of one operator piece: 128 rows x 64 B
#define RT_X_CHUNK (R_TB * TC_ROWB)     // one K chunk of one multipole piece: 64 rows x 64 B
#define RT_A_ROUND (RT_KQ * RT_A_CHUNK)
#define RT_X_ROUND (RT_KQ * RT_X_CHUNK)
#define RT_BUF (2 * RT_A_ROUND + 2 * RT_X_ROUND)  // a1, a2, x1, x2 of one round
#define RT_SMEM (2 * RT_BUF + 512)
#define RT_TMEM_COLS 64

struct RTcArgs {
    int p, nc, nkc;         // order, coefficients, K chunks of 16 that hold them
    const int4* batches;    // key index, first sorted entry, count | key << 8, table
    const double* tables;   // [table][TS][TS]
    const LfmmComp* comps;
    const float* phase;     // [225 lateral offsets][cos | sin][RT_TS] (k_m2r_phase)
    const int2* pairs;      // (source box, target box) per sorted entry (k_m2r_pairs)
    const double* levelh;
    const float* M;
    float* L;
    size_t stride;          // expansions per right-hand side, in floats
    int nr;
    int* err;               // [0]: timeouts
};

// e^{i m phi} of every lateral key offset (ox, oy) in [-7, 7]^2, m <= 2p:
// FP64 sincos rounded to float32, [offset][cos | sin][RT_TS]
__global__ void k_m2r_phase(int p, float* out)
{
    const int b = blockIdx.x, m = threadIdx.x;
    if (m > 2 * p) return;
    const int ox = b / R_OW - R_OR, oy = b % R_OW - R_OR;
    const double phi = (ox == 0 && oy == 0) ? 0.0 : atan2((double)oy, (double)ox);
    double sn, cs;
    sincos(m * phi, &sn, &cs);
    out[(size_t)b * 2 * RT_TS + m] = (float)cs;
    out[(size_t)b * 2 * RT_TS + RT_TS + m] = (float)sn;
}

__global__ void __launch_bounds__(RT_THREADS, RT_MINB) k_m2r_tc(RTcArgs g)
{
    extern __shared__ unsigned char smem_raw[];
    // 512-byte alignment: the period of the 64-byte swizzle
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 511) &
                                                         ~(uintptr_t)511);
    // W(N, mu) = T(N, |mu|) e^{i mu phi} for mu in [-2p, 2p], extended to
    // negative orders by W(N, -mu) = (-1)^mu conj W(N, mu); real parts, then
    // imaginary parts, each [N][mu + 2p] with rows of 4p + 1
    __shared__ float sW[2 * RT_TS * RT_WS];
    __shared__ float sPh[2 * RT_TS];
    __shared__ int2 s_off[2][128];   // per output parity aim and input: offsets of the two W terms
    __shared__ float2 s_cf[2][128];  // their signs (0: no second term, or no such input)
    __shared__ int s_roff[128];      // per output coefficient (k, l): k (4p + 1) + l + 2p
    __shared__ float s_sk[128];      // (-1)^k, 0 past the last coefficient
    __shared__ unsigned char s_aim[128];
    __shared__ int s_src[R_TB], s_tgt[R_TB];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ float s_ih;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p = g.p, nc = g.nc, nkc = g.nkc, TS = 2 * p + 1, WS = 4 * p + 1, TSZ = TS * WS;
    const int4 b = g.batches[blockIdx.x];
    // the batch carries its key and table: one dependent load to everything else
    const int start = b.y, cnt = b.z & 255, tab = b.w;
    if (cnt <= 0 || cnt > R_TB) return;
    const int N = (cnt + 15) & ~15;  // MMA columns
    const int nq = (nkc + RT_KQ - 1) / RT_KQ;
    int c, lev, ox, oy, oz;
    rkey_decode((uint32_t)b.z >> 8, c, lev, ox, oy, oz);
    const bool refl = g.comps[c].refl != 0;

    if (tid < 128) {
        // output coefficient tid as a row, input coefficient tid as a column
        int n = 0, m = 0, im = 0;
        const bool in = tid < nc;
        if (in) lf_decode(p, tid, n, m, im);
        s_roff[tid] = in ? n * WS + m + 2 * p : 0;
        s_sk[tid] = in ? ((n & 1) ? -1.f : 1.f) : 0.f;
        s_aim[tid] = (unsigned char)im;
        // the multipole's reflection sign (-1)^{n+m} for s = -1 maps
        const float rs = (refl && ((n + m) & 1)) ? -1.f : 1.f;
        const float sg = (m & 1) ? -1.f : 1.f;  // (-1)^m of the second term
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int t = (a ^ im) * TSZ;  // real parts where the parities agree, else imaginary
            s_off[a][tid] = in ? make_int2(t + n * WS + m, t + n * WS - m) : make_int2(0, 0);
            // (re,re): W1 + sg W2; (re out, im in): -W1 + sg W2; (im, re): W1 + sg W2; (im, im): W1 - sg W2
            const float c1 = (a == 0 && im == 1) ? -1.f : 1.f;
            const float c2 = m > 0 ? ((a == 1 && im == 1) ? -sg : sg) : 0.f;
            s_cf[a][tid] = in ? make_float2(rs * c1, rs * c2) : make_float2(0.f, 0.f);
        }
    }
    if (tid < R_TB) {
        const int2 pr = (tid < cnt) ? g.pairs[start + tid] : make_int2(-1, -1);
        s_src[tid] = pr.x;
        s_tgt[tid] = pr.y;
    }
    if (tid >= 128 && tid < 128 + 2 * RT_TS)
        sPh[tid - 128] = g.phase[(size_t)((ox + R_OR) * R_OW + (oy + R_OR)) * 2 * RT_TS + (tid - 128)];
    if (tid == 192) s_ih = (float)(1.0 / g.levelh[lev]);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(RT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    {
        const double* Tk = g.tables + (size_t)tab * TS * TS;
        for (int j = tid; j < TSZ; j += RT_THREADS) {
            const int Nn = j / WS, mu = j - Nn * WS - 2 * p, a = mu < 0 ? -mu : mu;
            const float t = (float)Tk[Nn * TS + a];
            float wr = t * sPh[a], wi = t * sPh[RT_TS + a];
            if (mu < 0) {
                if (a & 1) wr = -wr; else wi = -wi;
            }
            sW[j] = wr;
            sW[TSZ + j] = wi;
        }
    }
    const float ih = s_ih;
    // gather unit of every K chunk: column xj (rows >= N are not read), 16-byte
    // quarter xq; a warp covers 8 columns = 512 contiguous bytes of a chunk.
    // Operator units: rows xj and xj + 64, quarter xq.
    const int xj = tid >> 2, xq = tid & 3;
    const uint32_t idesc = tc_idesc(128, N);
    bool ok = true;
    for (int r = 0; r < g.nr && ok; ++r) {
        float xv[8][4];
        {
            const float* M = g.M + (size_t)r * g.stride;
            const int s = (xj < N) ? s_src[xj] : -1;
#pragma unroll
            for (int kc = 0; kc < 8; ++kc)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = kc * 16 + 4 * xq + e;
                    xv[kc][e] = (kc < nkc && s >= 0 && k < nc) ? M[(size_t)s * nc + k] : 0.f;
                }
        }
        if (r == 0) __syncthreads();  // W is in shared memory
#pragma unroll
        for (int i = 0; i < 8 / RT_KQ; ++i) {
            if (i >= nq) break;
            const int gr = r * nq + i, buf = gr & 1;  // round counter over the vectors
            if (gr >= 2 && !mbar_wait(&bar[buf], (uint32_t)(((gr - 2) >> 1) & 1))) s_abort = 1;
            unsigned char* sb = sm + (size_t)buf * RT_BUF;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = xj + 64 * h;
                const float* W = sW + s_roff[row];
                const float sk = s_sk[row];
                const int a = s_aim[row];
#pragma unroll
                for (int kl = 0; kl < RT_KQ; ++kl) {
                    const int kc = i * RT_KQ + kl;
                    if (kc >= nkc) break;
                    float hi[4], lo[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int kin = kc * 16 + 4 * xq + e;
                        const int2 o = s_off[a][kin];
                        const float2 cf = s_cf[a][kin];
                        const float v = sk * fmaf(cf.x, W[o.x], cf.y * W[o.y]);
                        hi[e] = __uint_as_float(to_tf32(v));
                        lo[e] = __uint_as_float(to_tf32(v - hi[e]));
                    }
                    const uint32_t off = (uint32_t)kl * RT_A_CHUNK + swz(row, 4 * xq);
                    *reinterpret_cast<float4*>(sb + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<float4*>(sb + RT_A_ROUND + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
            if (xj < N) {
#pragma unroll
                for (int kl = 0; kl < RT_KQ; ++kl) {
                    const int kc = i * RT_KQ + kl;
                    if (kc >= nkc) break;
                    float hi[4], lo[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        hi[e] = __uint_as_float(to_tf32(xv[kc][e]));
                        lo[e] = __uint_as_float(to_tf32(xv[kc][e] - hi[e]));
                    }
                    const uint32_t off = 2 * RT_A_ROUND + (uint32_t)kl * RT_X_CHUNK + swz(xj, 4 * xq);
                    *reinterpret_cast<float4*>(sb + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<float4*>(sb + RT_X_ROUND + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (*(volatile int*)&s_abort) break;  // block-uniform after the barrier
            if (tid == 0) {
                tc_fence_after();
                const uint32_t a0 = smem_u32(sb), x0 = a0 + 2 * RT_A_ROUND;
#pragma unroll
                for (int prod = 0; prod < 3; ++prod) {
                    const uint32_t a = a0 + (prod == 2 ? RT_A_ROUND : 0), x = x0 + (prod == 1 ? RT_X_ROUND : 0);
#pragma unroll
                    for (int kl = 0; kl < RT_KQ; ++kl) {
                        if (i * RT_KQ + kl >= nkc) break;
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks)
                            tc_mma(tmem, smem_desc(a + kl * RT_A_CHUNK + 32 * ks),
                                   smem_desc(x + kl * RT_X_CHUNK + 32 * ks), idesc,
                                   (i | prod | kl | ks) != 0 ? 1u : 0u);
                    }
                }
                tc_commit(&bar[buf]);
            }
            __syncwarp();
        }
        // the last round's commit covers every MMA before it
        bool got = false;
        if (!*(volatile int*)&s_abort) {
            const int gl = r * nq + nq - 1;
            got = mbar_wait(&bar[gl & 1], (uint32_t)((gl >> 1) & 1));
        }
        ok = __syncthreads_and(got) != 0;  // block-uniform
        tc_fence_after();
        if (ok) {
            const int q4 = warp & 3, half = warp >> 2;
            if (half * 32 < N) {
                float v[32];
                tc_ld32(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(half * 32), v);
                const int row = 32 * q4 + lane;
                if (row < nc) {
                    float* L = g.L + (size_t)r * g.stride;
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int j = half * 32 + i;
                        if (j < cnt) atomicAdd(L + (size_t)s_tgt[j] * nc + row, v[i] * ih);
                    }
                }
            }
        } else if (tid == 0) {
            atomicAdd(g.err, 1);
        }
        tc_fence_before();
        __syncthreads();  // the accumulator is free again
        tc_fence_after();
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(RT_TMEM_COLS)
                     : "memory");
}

template <typename R, int RP>
static LfErr m2r_build_ops(lfmm_ctx* ctx, cudaStream_t st)
{
    const int nk = ctx->m2r_nkeys;
    LF_TRY(lf_reserve(ctx->m2r_ops, (size_t)nk * RP * RP * sizeof(R) + 16));
    ROpArgs g;
    g.p = ctx->p;
    g.nc = lf_nc(ctx->p);
    g.kval = ctx->m2r_kval.as<uint32_t>() + ctx->m2r_kfirst;
    g.tables = ctx->m2r_tables.as<double>();
    g.ktab = ctx->m2r_ktab.as<int>();
    g.comps = ctx->comp_dev.as<LfmmComp>();
    g.ops = ctx->m2r_ops.ptr;
    const int TS = 2 * ctx->p + 1;
    const size_t sm = sizeof(R) * ((size_t)TS * TS + 2 * (size_t)TS) + 16;
    LF_CHECK(cudaFuncSetAttribute(k_m2r_ops<R, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    ++ctx->launches, k_m2r_ops<R, RP><<<nk, R_T, sm, st>>>(g);
    LF_TRY(lf_cuda(cudaGetLastError(), "m2r operators"));
    ctx->m2r_ops_prec = sizeof(R) == 4 ? 1 : 0;
    return LfErr();
}

template <typename R, int RP>
static LfErr m2r_apply_rp(lfmm_ctx* ctx, cudaStream_t st)
{
    if (ctx->m2r_ops_prec != (sizeof(R) == 4 ? 1 : 0)) LF_TRY((m2r_build_ops<R, RP>(ctx, st)));
    RGemmArgs g;
    g.p = ctx->p;
    g.nc = lf_nc(ctx->p);
    g.batches = ctx->m2r_batches.as<int4>();
    g.kval = ctx->m2r_kval.as<uint32_t>() + ctx->m2r_kfirst;
    g.ops = ctx->m2r_ops.ptr;
    g.order = ctx->m2r_order.as<uint32_t>();
    g.ent = ctx->m2r_ent.as<uint32_t>();
    g.tgt = ctx->m2r_tgt.as<int>();
    g.levelh = ctx->m2r_levelh.as<double>();
    g.M = ctx->Mexp.ptr;
    g.L = ctx->Lexp.ptr;
    g.stride = (size_t)ctx->nbox_total * g.nc;
    g.nr = ctx->nrhs_b;
    const size_t sm = sizeof(R) * ((size_t)RP * RP + (size_t)R_TB * (RP + 1)) + 16;
    LF_CHECK(cudaFuncSetAttribute(k_m2r_gemm<R, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    ++ctx->launches, k_m2r_gemm<R, RP><<<ctx->m2r_nbatch, R_T, sm, st>>>(g);
    return lf_cuda(cudaGetLastError(), "m2r gemm");
}

template <typename R, int RP>
static LfErr m2r_apply_kc(lfmm_ctx* ctx, cudaStream_t st)
{
    if (ctx->m2r_ops_prec != (sizeof(R) == 4 ? 1 : 0)) LF_TRY((m2r_build_ops<R, RP>(ctx, st)));
    RGemmArgs g;
    g.p = ctx->p;
    g.nc = lf_nc(ctx->p);
    g.batches = ctx->m2r_batches.as<int4>();
    g.kval = ctx->m2r_kval.as<uint32_t>() + ctx->m2r_kfirst;
    g.ops = ctx->m2r_ops.ptr;
    g.order = ctx->m2r_order.as<uint32_t>();
    g.ent = ctx->m2r_ent.as<uint32_t>();
    g.tgt = ctx->m2r_tgt.as<int>();
    g.levelh = ctx->m2r_levelh.as<double>();
    g.M = ctx->Mexp.ptr;
    g.L = ctx->Lexp.ptr;
    g.stride = (size_t)ctx->nbox_total * g.nc;
    g.nr = ctx->nrhs_b;
    const size_t sm = sizeof(R) * ((size_t)R_KC * RP + (size_t)R_TB * (RP + 1)) + 16;
    LF_CHECK(cudaFuncSetAttribute(k_m2r_gemm_kc<R, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    ++ctx->launches, k_m2r_gemm_kc<R, RP><<<ctx->m2r_nbatch, R_T, sm, st>>>(g);
    return lf_cuda(cudaGetLastError(), "m2r gemm (operator chunks)");
}

// the float32 form with (p+1)^2 <= 128 applies the keys on the tensor cores
// whenever the free M2L does (tensor-core option)
static bool m2r_tc_on(const lfmm_ctx* ctx) { return ctx->precision == 1 && ctx->p <= 10 && lf_tc_on(ctx); }

static LfErr m2r_apply_tc(lfmm_ctx* ctx, cudaStream_t st)
{
    RTcArgs g;
    g.p = ctx->p;
    g.nc = lf_nc(ctx->p);
    g.nkc = (g.nc + 15) / 16;
    g.batches = ctx->m2r_batches.as<int4>();
    g.tables = ctx->m2r_tables.as<double>();
    g.comps = ctx->comp_dev.as<LfmmComp>();
    g.pairs = ctx->m2r_pairs.as<int2>();
    g.levelh = ctx->m2r_levelh.as<double>();
    g.M = ctx->Mexp.as<float>();
    g.L = ctx->Lexp.as<float>();
    g.stride = (size_t)ctx->nbox_total * g.nc;
    g.nr = ctx->nrhs_b;
    g.err = reinterpret_cast<int*>(ctx->counts.as<char>() + LFMM_TIMEOUT_OFF);
    if (ctx->m2r_phase_p != ctx->p) {
        // once per context (the first evaluation; a captured batch graph never sees it)
        LF_TRY(lf_reserve(ctx->m2r_phase, (size_t)R_OW * R_OW * 2 * RT_TS * sizeof(float)));
        ++ctx->launches, k_m2r_phase<<<R_OW * R_OW, 32, 0, st>>>(ctx->p, ctx->m2r_phase.as<float>());
        LF_TRY(lf_cuda(cudaGetLastError(), "m2r phases"));
        ctx->m2r_phase_p = ctx->p;
    }
    g.phase = ctx->m2r_phase.as<float>();
    LF_CHECK(cudaFuncSetAttribute(k_m2r_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, RT_SMEM));
    ++ctx->launches, k_m2r_tc<<<ctx->m2r_nbatch, RT_THREADS, RT_SMEM, st>>>(g);
    return lf_cuda(cudaGetLastError(), "m2r tensor-core GEMM");
}

template <typename R>
static LfErr m2r_apply_t(lfmm_ctx* ctx, cudaStream_t st)
{
    if (sizeof(R) == 4 && m2r_tc_on(ctx)) return m2r_apply_tc(ctx, st);
    switch (ctx->m2l_rm) {
    case 2: return m2r_apply_rp<R, 32>(ctx, st);
    case 4: return m2r_apply_rp<R, 64>(ctx, st);
    case 8: return m2r_apply_rp<R, 128>(ctx, st);
    case 12: return m2r_apply_kc<R, 192>(ctx, st);
    case 16: return m2r_apply_kc<R, 256>(ctx, st);
    default: return "internal: reaction GEMM supports p <= 15";
    }
}

// assemble the operators of the keys for the current precision (build time)
LfErr lf_m2r_ops(lfmm_ctx* ctx, cudaStream_t st)
{
    // the tensor-core form assembles each operator where it is applied; the
    // CUDA-core GEMM builds them on first use if the option changes later
    if (ctx->m2r_nbatch == 0 || m2r_tc_on(ctx)) return LfErr();
    switch (ctx->m2l_rm) {
    case 2: return ctx->precision ? m2r_build_ops<float, 32>(ctx, st) : m2r_build_ops<double, 32>(ctx, st);
    case 4: return ctx->precision ? m2r_build_ops<float, 64>(ctx, st) : m2r_build_ops<double, 64>(ctx, st);
    case 8: return ctx->precision ? m2r_build_ops<float, 128>(ctx, st) : m2r_build_ops<double, 128>(ctx, st);
    case 12: return ctx->precision ? m2r_build_ops<float, 192>(ctx, st) : m2r_build_ops<double, 192>(ctx, st);
    case 16: return ctx->precision ? m2r_build_ops<float, 256>(ctx, st) : m2r_build_ops<double, 256>(ctx, st);
    default: return "internal: reaction GEMM supports p <= 15";
    }
}

LfErr lf_m2r_apply(lfmm_ctx* ctx, cudaStream_t st)
{
    if (ctx->m2r_nbatch == 0) return LfErr();
    return ctx->precision ? m2r_apply_t<float>(ctx, st) : m2r_apply_t<double>(ctx, st);
}
