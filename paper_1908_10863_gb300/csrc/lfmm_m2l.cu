// lfmm_m2l.cu -- free-space M2L (eq. metole) as dense per-offset GEMMs.
//
// In box units the free-space M2L between a target box and a source box at
// integer offset o = (t - s)/h is a fixed real-linear map A_o of the packed
// coefficients (Re of m >= 0, Im of m >= 1):
//   L_k^l = (-1)^k sum_{n,m} M_n^m T_{n+k}^{m+l}(o),
// the same at every level (the 1/h of the scaled expansions is applied when
// the result is stored).  A target box whose position inside its parent is
// the octant c interacts with the 189 offsets
//   o_x in [-3, 2] (c_x = 0) or [-2, 3] (c_x = 1), same for y, z, |o|_inf >= 2,
// so all targets of one octant share one offset list.  Targets are grouped by
// (level, octant) into tiles of 64; a block keeps the 64 local expansions of
// its tile in registers and, for each of the 189 offsets, gathers the 64
// source multipoles (zero where a target has no source at that offset) and
// multiplies them by A_o: 189 register-tiled GEMMs of (p+1)^2 x (p+1)^2 x 64.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <complex>
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

#define G_TB 64        // targets per tile
#define G_KC 32        // K chunk of the operator staged in shared memory
#define G_T 256        // threads per block: 16 row groups x 16 column groups
#define G_NOFF 189     // offsets per octant class
#define G_NALL 343     // offsets in [-3,3]^3

static inline int off_index(int ox, int oy, int oz) { return (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3); }

// rows per thread for expansion order p (rows covered = 16 * RM >= (p+1)^2)
static int gemm_rm(int p)
{
    int nc = lf_nc(p);
    const int opts[5] = {2, 4, 8, 12, 16};
    for (int r : opts)
        if (16 * r >= nc) return r;
    return 0;
}

// ---------------------------------------------------------------------------
// Host: operators and offset classes.
// ---------------------------------------------------------------------------
LfErr lf_setup_m2l_ops(lfmm_ctx* ctx)
{
    const int p = ctx->p;
    const int rm = gemm_rm(p);
    ctx->m2l_rm = rm;
    if (rm == 0) return LfErr();  // order too high for the GEMM path
    const int nc = lf_nc(p), nre = lf_nre(p), RP = 16 * rm, KP = RP;
    ctx->m2l_rp = RP;
    const int TS = 2 * p + 1;
    std::vector<double> A64((size_t)G_NALL * KP * RP, 0.0);
    std::vector<double> T(TS * TS);
    auto RE = [&](int n, int m) { return n * (n + 1) / 2 + m; };
    auto IM = [&](int n, int m) { return nre + n * (n - 1) / 2 + m - 1; };
    for (int ox = -3; ox <= 3; ++ox)
        for (int oy = -3; oy <= 3; ++oy)
            for (int oz = -3; oz <= 3; ++oz) {
                if (std::max(abs(ox), std::max(abs(oy), abs(oz))) < 2) continue;
                double rho = sqrt((double)(ox * ox + oy * oy));
                double phi = (ox == 0 && oy == 0) ? 0.0 : atan2((double)oy, (double)ox);
                for (int mu = 0; mu <= 2 * p; ++mu) lf_theta_column(rho, (double)oz, mu, 2 * p, 1.0, T.data(), TS);
                // complex T_N^mu = e^{i mu phi} T(N, mu); T_N^{-mu} = (-1)^mu conj(T_N^mu)
                auto Th = [&](int N, int mu, double& c, double& d) {
                    int a = mu < 0 ? -mu : mu;
                    double v = T[N * TS + a];
                    c = v * cos(a * phi);
                    d = v * sin(a * phi);
                    if (mu < 0) {
                        if (a & 1) c = -c; else d = -d;  // (-1)^a conj(c + i d)
                    }
                };
                double* Ao = &A64[(size_t)off_index(ox, oy, oz) * KP * RP];  // [k_in][r_out]
                for (int k = 0; k <= p; ++k)
                    for (int l = 0; l <= k; ++l) {
                        const double sk = (k & 1) ? -1.0 : 1.0;
                        for (int n = 0; n <= p; ++n)
                            for (int mp = 0; mp <= n; ++mp) {
                                double c1, d1, c2 = 0, d2 = 0, s = 0;
                                Th(n + k, mp + l, c1, d1);
                                if (mp > 0) {
                                    Th(n + k, l - mp, c2, d2);
                                    s = (mp & 1) ? -1.0 : 1.0;
                                }
                                Ao[(size_t)RE(n, mp) * RP + RE(k, l)] += sk * (c1 + s * c2);
                                if (mp > 0) Ao[(size_t)IM(n, mp) * RP + RE(k, l)] += sk * (-d1 + s * d2);
                                if (l > 0) {
                                    Ao[(size_t)RE(n, mp) * RP + IM(k, l)] += sk * (d1 + s * d2);
                                    if (mp > 0) Ao[(size_t)IM(n, mp) * RP + IM(k, l)] += sk * (c1 - s * c2);
                                }
                            }
                    }
            }
    (void)nc;
    LF_TRY(lf_setup_m2l_tc(ctx, A64.data(), KP, RP));
    std::vector<float> A32(A64.size());
    for (size_t i = 0; i < A64.size(); ++i) A32[i] = (float)A64[i];
    LF_TRY(lf_reserve(ctx->m2l_A64, A64.size() * 8));
    LF_TRY(lf_reserve(ctx->m2l_A32, A32.size() * 4));
    LF_CHECK(cudaMemcpy(ctx->m2l_A64.ptr, A64.data(), A64.size() * 8, cudaMemcpyHostToDevice));
    LF_CHECK(cudaMemcpy(ctx->m2l_A32.ptr, A32.data(), A32.size() * 4, cudaMemcpyHostToDevice));
    // offset classes: cls[c][i] = global offset index, inv[c][o] = i or -1
    std::vector<int> cls(8 * G_NOFF, -1), inv(8 * G_NALL, -1);
    for (int c = 0; c < 8; ++c) {
        int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        int i = 0;
        for (int ox = cx ? -2 : -3; ox <= (cx ? 3 : 2); ++ox)
            for (int oy = cy ? -2 : -3; oy <= (cy ? 3 : 2); ++oy)
                for (int oz = cz ? -2 : -3; oz <= (cz ? 3 : 2); ++oz) {
                    if (std::max(abs(ox), std::max(abs(oy), abs(oz))) < 2) continue;
                    cls[c * G_NOFF + i] = off_index(ox, oy, oz);
                    inv[c * G_NALL + off_index(ox, oy, oz)] = i;
                    ++i;
                }
        if (i != G_NOFF) return "internal: offset class size";
    }
    LF_TRY(lf_reserve(ctx->m2l_cls, sizeof(int) * cls.size()));
    LF_TRY(lf_reserve(ctx->m2l_inv, sizeof(int) * inv.size()));
    LF_CHECK(cudaMemcpy(ctx->m2l_cls.ptr, cls.data(), sizeof(int) * cls.size(), cudaMemcpyHostToDevice));
    LF_CHECK(cudaMemcpy(ctx->m2l_inv.ptr, inv.data(), sizeof(int) * inv.size(), cudaMemcpyHostToDevice));
    return LfErr();
}

// ---------------------------------------------------------------------------
// Build: slot table and tiles.
// ---------------------------------------------------------------------------
__global__ void k_fill_slots(int off, int nb, double h, const uint32_t* __restrict__ bkey,
                             const LfD4* __restrict__ cen, const int* __restrict__ mbeg,
                             const int* __restrict__ mend, const uint32_t* __restrict__ ment,
                             const int* __restrict__ inv, int* __restrict__ slots, int* __restrict__ err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int t = off + i;
    int c = (int)(bkey[t] & 7u);
    LfD4 ct = cen[t];
    double ih = 1.0 / h;
    for (int e = mbeg[t]; e < mend[t]; ++e) {
        int s = (int)(ment[e] & LFMM_ENT_MASK);
        LfD4 cs = cen[s];
        int ox = (int)lrint((ct.x - cs.x) * ih), oy = (int)lrint((ct.y - cs.y) * ih), oz = (int)lrint((ct.z - cs.z) * ih);
        int loc = -1;
        if (ox >= -3 && ox <= 3 && oy >= -3 && oy <= 3 && oz >= -3 && oz <= 3)
            loc = inv[c * G_NALL + (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3)];
        if (loc < 0) {
            atomicAdd(err, 1);
            continue;
        }
        slots[(size_t)t * G_NOFF + loc] = s;
    }
}

__global__ void k_class_keys(int off, int nb, int level, const uint32_t* __restrict__ bkey,
                             uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, int base,
                             int* __restrict__ counts)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int c = (int)(bkey[off + i] & 7u);
    keys[base + i] = ((uint32_t)level << 28) | ((uint32_t)c << 25) | (uint32_t)i;
    vals[base + i] = (uint32_t)(off + i);
    atomicAdd(&counts[level * 8 + c], 1);
}

LfErr lf_prepare_m2l(lfmm_ctx* ctx, cudaStream_t st)
{
    ctx->m2l_ntiles = 0;
    if (ctx->m2l_rm == 0) return LfErr();
    const int depth = ctx->depth;
    if (depth < 2) return LfErr();
    const size_t nb = (size_t)ctx->nbox_total;
    LF_TRY(lf_reserve(ctx->m2l_slots, nb * G_NOFF * sizeof(int)));
    LF_CHECK(cudaMemsetAsync(ctx->m2l_slots.ptr, 0xff, nb * G_NOFF * sizeof(int), st));
    int* err = reinterpret_cast<int*>(ctx->counts.as<char>() + 24576);
    int* cnt = err + 16;  // [16 levels][8]
    LF_CHECK(cudaMemsetAsync(err, 0, sizeof(int) * (16 + 16 * 8), st));
    int nsort = 0;
    for (int l = 2; l <= depth; ++l) nsort += ctx->levels[l].nbox;
    LF_TRY(lf_reserve(ctx->m2l_keys, (size_t)nsort * 4 + 16));
    LF_TRY(lf_reserve(ctx->m2l_sorted, (size_t)nsort * 4 + 16));
    int base = 0;
    for (int l = 2; l <= depth; ++l) {
        const LfmmLevel& lv = ctx->levels[l];
        if (lv.nbox == 0) continue;
        ++ctx->launches, k_fill_slots<<<lf_blocks(lv.nbox, 128), 128, 0, st>>>(
            lv.off, lv.nbox, lv.h, ctx->box_key.as<uint32_t>(), ctx->box_center.as<LfD4>(), ctx->m2l_off.as<int>(),
            ctx->m2l_off.as<int>() + ctx->nbox_total, ctx->m2l_ent.as<uint32_t>(), ctx->m2l_inv.as<int>(),
            ctx->m2l_slots.as<int>(), err);
        ++ctx->launches, k_class_keys<<<lf_blocks(lv.nbox, 256), 256, 0, st>>>(
            lv.off, lv.nbox, l, ctx->box_key.as<uint32_t>(), ctx->m2l_keys.as<uint32_t>(),
            ctx->m2l_sorted.as<uint32_t>(), base, cnt);
        base += lv.nbox;
    }
    LF_TRY(lf_cuda(cudaGetLastError(), "m2l slots"));
    LF_TRY(lf_radix_sort(ctx, ctx->m2l_keys.as<uint32_t>(), ctx->m2l_sorted.as<uint32_t>(), nsort, st));
    int hcnt[16 + 16 * 8];
    LF_CHECK(cudaMemcpyAsync(hcnt, err, sizeof(hcnt), cudaMemcpyDeviceToHost, st));
    LF_CHECK(cudaStreamSynchronize(st));
    if (hcnt[0] != 0) return "internal: free M2L entry outside its offset class";
    std::vector<int4> tiles;
    int start = 0;
    for (int l = 2; l <= depth; ++l)
        for (int c = 0; c < 8; ++c) {
            int n = hcnt[16 + l * 8 + c];
            for (int s = 0; s < n; s += G_TB) tiles.push_back(make_int4(l, c, start + s, std::min(G_TB, n - s)));
            start += n;
        }
    ctx->m2l_ntiles = (int)tiles.size();
    if (!tiles.empty()) {
        LF_TRY(lf_reserve(ctx->m2l_tiles, tiles.size() * sizeof(int4)));
        LF_CHECK(cudaMemcpyAsync(ctx->m2l_tiles.ptr, tiles.data(), tiles.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, st));
    }
    // wider tiles of the same (level, class) runs for the tensor-core kernel
    std::vector<int4> tct;
    ctx->m2l_tc_ntiles = 0;
    if (ctx->m2l_tc_ok) {
        const int TN = lf_m2l_tc_tile();
        int st0 = 0;
        for (int l = 2; l <= depth; ++l)
            for (int c = 0; c < 8; ++c) {
                int n = hcnt[16 + l * 8 + c];
                for (int s = 0; s < n; s += TN) tct.push_back(make_int4(l, c, st0 + s, std::min(TN, n - s)));
                st0 += n;
            }
        ctx->m2l_tc_ntiles = (int)tct.size();
        if (!tct.empty()) {
            LF_TRY(lf_reserve(ctx->m2l_tc_tiles, tct.size() * sizeof(int4)));
            LF_CHECK(cudaMemcpyAsync(ctx->m2l_tc_tiles.ptr, tct.data(), tct.size() * sizeof(int4),
                                     cudaMemcpyHostToDevice, st));
        }
    }
    double hl[16] = {0};
    for (int l = 0; l <= depth && l < 16; ++l) hl[l] = ctx->levels[l].h;
    LF_TRY(lf_reserve(ctx->m2l_levelh, sizeof(hl)));
    LF_CHECK(cudaMemcpyAsync(ctx->m2l_levelh.ptr, hl, sizeof(hl), cudaMemcpyHostToDevice, st));
    LF_CHECK(cudaStreamSynchronize(st));
    return LfErr();
}

// ---------------------------------------------------------------------------
// The GEMM kernel.  Thread (rg, cg): rows rg*RM .. rg*RM+RM-1 of the packed
// output, columns 4cg .. 4cg+3 of the tile.  X is stored column-major
// [j][k] with stride KP+1 (conflict-free gathers and reads).
// ---------------------------------------------------------------------------
struct GemmArgs {
    int p, nc, RP;
    const int4* tiles;
    const int* sorted;
    const int* slots;
    const int* cls;
    const double* levelh;
    const void* A;
    const void* M;
    void* L;
};

template <typename R, int RM>
__global__ void __launch_bounds__(G_T) k_m2l_gemm(GemmArgs g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int RP = 16 * RM;
    constexpr int KP = RP;
    constexpr int XS = KP + 1;
    R* sA = reinterpret_cast<R*>(smem_raw);  // [G_KC][RP]
    R* sX = sA + G_KC * RP;                  // [G_TB][XS]
    __shared__ int s_tb[G_TB];
    __shared__ int s_src[G_TB];
    const int tid = threadIdx.x;
    const int cg = tid & 15, rg = tid >> 4;
    const int4 tile = g.tiles[blockIdx.x];
    const int level = tile.x, cls = tile.y, start = tile.z, cnt = tile.w;
    const int nc = g.nc;
    const R* A = reinterpret_cast<const R*>(g.A);
    const R* M = reinterpret_cast<const R*>(g.M);
    R* L = reinterpret_cast<R*>(g.L);
    if (tid < G_TB) s_tb[tid] = (tid < cnt) ? g.sorted[start + tid] : -1;
    R acc[RM][4];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0;
    __syncthreads();
    for (int oi = 0; oi < G_NOFF; ++oi) {
        const int o = g.cls[cls * G_NOFF + oi];
        if (tid < G_TB) s_src[tid] = (tid < cnt) ? g.slots[(size_t)s_tb[tid] * G_NOFF + oi] : -1;
        __syncthreads();
        // gather the source multipoles: column j = source of target j (k fastest)
        for (int idx = tid; idx < G_TB * KP; idx += G_T) {
            int j = idx / KP, k = idx - j * KP;
            int s = s_src[j];
            R v = 0;
            if (s >= 0 && k < nc) v = M[(size_t)s * nc + k];
            sX[j * XS + k] = v;
        }
        const R* Ao = A + (size_t)o * KP * RP;
        for (int kc = 0; kc < KP; kc += G_KC) {
            __syncthreads();
            // stage A_o[kc .. kc+KC][0 .. RP) (contiguous)
            const R* src = Ao + (size_t)kc * RP;
            for (int idx = tid; idx < G_KC * RP; idx += G_T) sA[idx] = src[idx];
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < G_KC; ++kk) {
                R a[RM];
#pragma unroll
                for (int r = 0; r < RM; ++r) a[r] = sA[kk * RP + rg * RM + r];
                R x[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) x[c] = sX[(4 * cg + c) * XS + kc + kk];
#pragma unroll
                for (int r = 0; r < RM; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * x[c];
            }
        }
        __syncthreads();
    }
    const R ih = (R)(1.0 / g.levelh[level]);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int j = 4 * cg + c;
        if (j >= cnt) continue;
        R* Lt = L + (size_t)s_tb[j] * nc;
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            int row = rg * RM + r;
            if (row < nc) Lt[row] += acc[r][c] * ih;
        }
    }
}

template <typename R, int RM>
static LfErr launch_gemm(lfmm_ctx* ctx, cudaStream_t st, const GemmArgs& g)
{
    constexpr int RP = 16 * RM;
    size_t sm = sizeof(R) * ((size_t)G_KC * RP + (size_t)G_TB * (RP + 1));
    LF_CHECK(cudaFuncSetAttribute(k_m2l_gemm<R, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    ++ctx->launches, k_m2l_gemm<R, RM><<<ctx->m2l_ntiles, G_T, sm, st>>>(g);
    return lf_cuda(cudaGetLastError(), "m2l gemm");
}

template <typename R>
static LfErr m2l_gemm_t(lfmm_ctx* ctx, cudaStream_t st)
{
    GemmArgs g;
    g.p = ctx->p;
    g.nc = lf_nc(ctx->p);
    g.RP = ctx->m2l_rp;
    g.tiles = ctx->m2l_tiles.as<int4>();
    g.sorted = ctx->m2l_sorted.as<int>();
    g.slots = ctx->m2l_slots.as<int>();
    g.cls = ctx->m2l_cls.as<int>();
    g.levelh = ctx->m2l_levelh.as<double>();
    g.A = sizeof(R) == 8 ? ctx->m2l_A64.ptr : ctx->m2l_A32.ptr;
    g.M = ctx->Mexp.ptr;
    g.L = ctx->Lexp.ptr;
    switch (ctx->m2l_rm) {
    case 2: return launch_gemm<R, 2>(ctx, st, g);
    case 4: return launch_gemm<R, 4>(ctx, st, g);
    case 8: return launch_gemm<R, 8>(ctx, st, g);
    case 12: return launch_gemm<R, 12>(ctx, st, g);
    case 16: return launch_gemm<R, 16>(ctx, st, g);
    default: return "internal: unsupported GEMM tile";
    }
}

LfErr lf_m2l_gemm(lfmm_ctx* ctx, cudaStream_t st)
{
    if (ctx->m2l_ntiles == 0) return LfErr();
    return ctx->precision ? m2l_gemm_t<float>(ctx, st) : m2l_gemm_t<double>(ctx, st);
}
