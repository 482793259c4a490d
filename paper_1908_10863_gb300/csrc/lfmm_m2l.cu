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
//
// The same gathered GEMM runs the translations between levels: M2M (eq.
// metome) with the 8 child-octant maps (each parent gathers its children,
// one "offset" per octant) and L2L (eq. letole) with one map per child
// octant (children grouped by octant gather their parent).  Their matrices
// are the packed real forms of the complex shift formulas, built on the host
// by applying those formulas to unit coefficient vectors.
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
// complex coefficient (n, m) of a packed real vector; negative m by
// X_n^{-m} = (-1)^m conj(X_n^m)
static void h_get(const double* v, int p, int n, int m, double& re, double& im)
{
    const int a = m < 0 ? -m : m;
    re = v[lf_re(n, a)];
    im = a > 0 ? v[lf_im(p, n, a)] : 0.0;
    if (m < 0) {
        const double s = (a & 1) ? -1.0 : 1.0;
        re *= s;
        im *= -s;
    }
}
static void h_getU(const double* ur, const double* ui, int n, int m, double& re, double& im)
{
    const int a = m < 0 ? -m : m;
    re = ur[lf_re(n, a)];
    im = ui[lf_re(n, a)];
    if (m < 0) {
        const double s = (a & 1) ? -1.0 : 1.0;
        re *= s;
        im *= -s;
    }
}
// M2M: M_p(n, m) = sum_{k <= n, l} 2^{-k} M_c(k, l) conj(U_{n-k}^{m-l}(d))
static void h_m2m(int p, const double* ur, const double* ui, const double* in, double* out)
{
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m) {
            double ar = 0, ai = 0, sc = 1;
            for (int k = 0; k <= n; ++k, sc *= 0.5)
                for (int l = -k; l <= k; ++l) {
                    const int dm = m - l;
                    if (dm > n - k || dm < -(n - k)) continue;
                    double mr, mi, vr, vi;
                    h_get(in, p, k, l, mr, mi);
                    h_getU(ur, ui, n - k, dm, vr, vi);
                    ar += sc * (mr * vr + mi * vi);
                    ai += sc * (mi * vr - mr * vi);
                }
            out[lf_re(n, m)] = ar;
            if (m > 0) out[lf_im(p, n, m)] = ai;
        }
}
// L2L: L_c(j, i) = 2^{-j} sum_{k >= j, l} L_p(k, l) conj(U_{k-j}^{l-i}(d))
static void h_l2l(int p, const double* ur, const double* ui, const double* in, double* out)
{
    for (int j = 0; j <= p; ++j)
        for (int i = 0; i <= j; ++i) {
            double ar = 0, ai = 0;
            for (int k = j; k <= p; ++k)
                for (int l = -k; l <= k; ++l) {
                    const int dm = l - i;
                    if (dm > k - j || dm < -(k - j)) continue;
                    double lr, li, vr, vi;
                    h_get(in, p, k, l, lr, li);
                    h_getU(ur, ui, k - j, dm, vr, vi);
                    ar += lr * vr + li * vi;
                    ai += li * vr - lr * vi;
                }
            const double sc = std::ldexp(1.0, -j);
            out[lf_re(j, i)] = sc * ar;
            if (i > 0) out[lf_im(p, j, i)] = sc * ai;
        }
}

// the 8 octant matrices [k_in][r_out] of M2M (which = 0) or L2L (which = 1)
static void shift_ops(int p, int KP, int RP, int which, std::vector<double>& A)
{
    const int nc = lf_nc(p), nre = lf_nre(p);
    A.assign((size_t)8 * KP * RP, 0.0);
    std::vector<double> ur(nre), ui(nre), in(nc), out(nc);
    for (int o = 0; o < 8; ++o) {
        const double x = (o & 1) ? 0.25 : -0.25, y = (o & 2) ? 0.25 : -0.25, z = (o & 4) ? 0.25 : -0.25;
        lf_regular<double>(p, x, y, z, ur.data(), ui.data());
        for (int k = 0; k < nc; ++k) {
            std::fill(in.begin(), in.end(), 0.0);
            in[k] = 1.0;
            if (which == 0)
                h_m2m(p, ur.data(), ui.data(), in.data(), out.data());
            else
                h_l2l(p, ur.data(), ui.data(), in.data(), out.data());
            for (int r = 0; r < nc; ++r) A[((size_t)o * KP + k) * RP + r] = out[r];
        }
    }
}

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
    // M2M / L2L octant matrices: [which][o][k_in][r_out], and their class tables
    std::vector<double> S2[2];
    for (int which = 0; which < 2; ++which) {
        std::vector<double>& S = S2[which];
        shift_ops(p, KP, RP, which, S);
        std::vector<float> Sf(S.size());
        for (size_t i = 0; i < S.size(); ++i) Sf[i] = (float)S[i];
        DevBuf& b64 = which ? ctx->l2l_A64 : ctx->m2m_A64;
        DevBuf& b32 = which ? ctx->l2l_A32 : ctx->m2m_A32;
        LF_TRY(lf_reserve(b64, S.size() * 8));
        LF_TRY(lf_reserve(b32, Sf.size() * 4));
        LF_CHECK(cudaMemcpy(b64.ptr, S.data(), S.size() * 8, cudaMemcpyHostToDevice));
        LF_CHECK(cudaMemcpy(b32.ptr, Sf.data(), Sf.size() * 4, cudaMemcpyHostToDevice));
    }
    LF_TRY(lf_setup_m2l_tc(ctx, A64.data(), S2[0].data(), S2[1].data(), KP, RP));
    const int shift_cls[8] = {0, 1, 2, 3, 4, 5, 6, 7};  // M2M: one class of 8 offsets; L2L: 8 classes of 1
    LF_TRY(lf_reserve(ctx->shift_cls, sizeof(shift_cls)));
    LF_CHECK(cudaMemcpy(ctx->shift_cls.ptr, shift_cls, sizeof(shift_cls), cudaMemcpyHostToDevice));
    return LfErr();
}

// ---------------------------------------------------------------------------
// Build: slot table and tiles.
// ---------------------------------------------------------------------------
__global__ void k_child_slots(int off, int nb, const uint32_t* __restrict__ bkey, const int* __restrict__ parent,
                              int* __restrict__ slots)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    const int b = off + i, pb = parent[b];
    if (pb >= 0) slots[(size_t)pb * 8 + (bkey[b] & 7u)] = b;
}

// Levels 1 .. depth in one launch: sort position j belongs to level l when
// base[l] <= j < base[l] + nb[l] (levels in increasing order).
struct ClassLevels {
    int depth;
    int off[17], nb[17], base[17];
};

__global__ void k_class_keys(ClassLevels lv, int nsort, const uint32_t* __restrict__ bkey,
                             uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, int* __restrict__ counts)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nsort) return;
    int level = 1;
    while (level < lv.depth && j >= lv.base[level] + lv.nb[level]) ++level;
    const int i = j - lv.base[level];
    const int c = (int)(bkey[lv.off[level] + i] & 7u);
    keys[j] = ((uint32_t)level << 28) | ((uint32_t)c << 25) | (uint32_t)i;
    vals[j] = (uint32_t)(lv.off[level] + i);
    atomicAdd(&counts[level * 8 + c], 1);
}

// Free M2L tiles of levels 2 .. depth: the targets of a level are sorted by
// (octant class, Morton index) and cut into tiles of `tn` per class; the
// tiles go out with the classes interleaved (tile k of class 0, of class 1,
// ..., then tile k + 1), so that tiles running at the same time cover one
// region of the level and share its source multipoles in L2 (class after
// class, every class streams the whole level's multipoles).
static void m2l_tiles_interleaved(const int* hcnt, int depth, int tn, std::vector<int4>& out)
{
    out.clear();
    int start = 0;
    for (int l = 1; l <= depth; ++l) {
        int first[8], n[8], most = 0;
        for (int c = 0; c < 8; ++c) {
            n[c] = hcnt[16 + l * 8 + c];
            first[c] = start;
            start += n[c];
            most = std::max(most, n[c]);
        }
        if (l < 2) continue;
        for (int s = 0; s < most; s += tn)
            for (int c = 0; c < 8; ++c)
                if (s < n[c]) out.push_back(make_int4(l, c, first[c] + s, std::min(tn, n[c] - s)));
    }
}

// Tensor-core tiles: the full tiles of every (level, class) run, in the
// order of m2l_tiles_interleaved; the leftover of each run (fewer than tn
// targets: every run of a small level) joins the leftovers of its class on
// the other levels in merged tiles of up to tn targets and LFMM_TC_MSEG runs
// (tile.x = -1 - its index in segs, tile.z = its runs), after the full tiles.
// A tile streams the operators of its 189 offsets whatever its fill, so a
// small tree's coarse levels no longer pay that once per level and class.
static void m2l_tc_tiles(const int* hcnt, int depth, int tn, std::vector<int4>& out, std::vector<int4>& segs)
{
    out.clear();
    segs.clear();
    std::vector<int4> left[8];  // (level, start, count, 0)
    int start = 0;
    for (int l = 1; l <= depth; ++l) {
        int first[8], n[8], most = 0;
        for (int c = 0; c < 8; ++c) {
            n[c] = hcnt[16 + l * 8 + c];
            first[c] = start;
            start += n[c];
            most = std::max(most, n[c]);
        }
        if (l < 2) continue;
        for (int s = 0; s < most; s += tn)
            for (int c = 0; c < 8; ++c) {
                if (s + tn <= n[c])
                    out.push_back(make_int4(l, c, first[c] + s, tn));
                else if (s < n[c])
                    left[c].push_back(make_int4(l, first[c] + s, n[c] - s, 0));
            }
    }
    for (int c = 0; c < 8; ++c) {
        std::vector<int4> cur;
        int fill = 0;
        auto flush = [&]() {
            if (cur.empty()) return;
            if (cur.size() == 1) {
                out.push_back(make_int4(cur[0].x, c, cur[0].y, cur[0].z));
            } else {
                const int m = (int)(segs.size() / LFMM_TC_MSEG);
                segs.insert(segs.end(), cur.begin(), cur.end());
                segs.resize((size_t)(m + 1) * LFMM_TC_MSEG, make_int4(0, 0, 0, 0));
                out.push_back(make_int4(-1 - m, c, (int)cur.size(), fill));
            }
            cur.clear();
            fill = 0;
        };
        for (int4 r : left[c])
            while (r.z > 0) {
                if (fill == tn || (int)cur.size() == LFMM_TC_MSEG) flush();
                const int take = std::min(r.z, tn - fill);
                cur.push_back(make_int4(r.x, r.y, take, 0));
                fill += take;
                r.y += take;
                r.z -= take;
            }
        flush();
    }
}

LfErr lf_prepare_m2l(lfmm_ctx* ctx, cudaStream_t st)
{
    ctx->m2l_ntiles = 0;
    ctx->shift_ready = 0;
    if (ctx->m2l_rm == 0) return LfErr();
    const int depth = ctx->depth;
    if (depth < 2) return LfErr();
    const size_t nb = (size_t)ctx->nbox_total;
    // the slot table was filled with the lists; errors counted at `err`
    int* err = reinterpret_cast<int*>(ctx->counts.as<char>() + 24576);
    int* cnt = err + 16;  // [16 levels][8]
    LF_CHECK(cudaMemsetAsync(cnt, 0, sizeof(int) * 16 * 8, st));
    int nsort = 0;
    for (int l = 1; l <= depth; ++l) nsort += ctx->levels[l].nbox;
    LF_TRY(lf_reserve(ctx->m2l_keys, (size_t)nsort * 4 + 16));
    LF_TRY(lf_reserve(ctx->m2l_sorted, (size_t)nsort * 4 + 16));
    ClassLevels cl;
    cl.depth = depth;
    int base = 0;
    for (int l = 1; l <= depth; ++l) {
        cl.off[l] = ctx->levels[l].off;
        cl.nb[l] = ctx->levels[l].nbox;
        cl.base[l] = base;
        base += ctx->levels[l].nbox;
    }
    if (nsort > 0)
        ++ctx->launches, k_class_keys<<<lf_blocks(nsort, 256), 256, 0, st>>>(
            cl, nsort, ctx->box_key.as<uint32_t>(), ctx->m2l_keys.as<uint32_t>(), ctx->m2l_sorted.as<uint32_t>(), cnt);
    // M2M slots: children of each parent by octant (every box of levels
    // 1 .. depth, which hold the ids below the roots', in one launch)
    LF_TRY(lf_reserve(ctx->m2m_slots, nb * 8 * sizeof(int)));
    LF_CHECK(cudaMemsetAsync(ctx->m2m_slots.ptr, 0xff, nb * 8 * sizeof(int), st));
    if (ctx->levels[0].off > 0)
        ++ctx->launches, k_child_slots<<<lf_blocks(ctx->levels[0].off, 256), 256, 0, st>>>(
            0, ctx->levels[0].off, ctx->box_key.as<uint32_t>(), ctx->box_parent.as<int>(), ctx->m2m_slots.as<int>());
    LF_TRY(lf_cuda(cudaGetLastError(), "m2l slots"));
    // keys are level << 28 | class << 25 | index: with fewer than 2^24 boxes the
    // top byte alone orders them (stable within a level and class)
    if (nsort < (1 << 24))
        LF_TRY(lf_radix_sort(ctx, ctx->m2l_keys.as<uint32_t>(), ctx->m2l_sorted.as<uint32_t>(), nsort, st, 3, 1));
    else
        LF_TRY(lf_radix_sort(ctx, ctx->m2l_keys.as<uint32_t>(), ctx->m2l_sorted.as<uint32_t>(), nsort, st));
    static_assert(LFMM_PIN_M2L + (16 + 16 * 8) * sizeof(int) <= LFMM_PIN_ROOT, "pinned regions");
    const int* hcnt = lf_pin<int>(ctx, LFMM_PIN_M2L);
    LF_CHECK(cudaMemcpyAsync(lf_pin<int>(ctx, LFMM_PIN_M2L), err, (16 + 16 * 8) * sizeof(int), cudaMemcpyDeviceToHost,
                             st));
    LF_CHECK(cudaStreamSynchronize(st));
    if (hcnt[0] != 0) return "internal: free M2L entry outside its offset class";
    std::vector<int4>& tiles = ctx->m2l_tiles_h;
    std::vector<int4>& l2l_tiles = ctx->l2l_tiles_h;
    tiles.clear();
    l2l_tiles.clear();
    std::vector<int> l2l_first(depth + 2, 0);
    int start = 0;
    for (int l = 1; l <= depth; ++l) {
        l2l_first[l] = (int)l2l_tiles.size();
        for (int c = 0; c < 8; ++c) {
            int n = hcnt[16 + l * 8 + c];
            for (int s = 0; s < n; s += G_TB) l2l_tiles.push_back(make_int4(l, c, start + s, std::min(G_TB, n - s)));
            start += n;
        }
    }
    m2l_tiles_interleaved(hcnt, depth, G_TB, tiles);
    l2l_first[depth + 1] = (int)l2l_tiles.size();
    // M2M tiles: parents of levels 0 .. depth-1 in box order
    std::vector<int4>& m2m_tiles = ctx->m2m_tiles_h;
    m2m_tiles.clear();
    ctx->m2m_first.assign(depth + 1, 0);
    for (int l = 0; l < depth; ++l) {
        ctx->m2m_first[l] = (int)m2m_tiles.size();
        const LfmmLevel& lv = ctx->levels[l];
        for (int s = 0; s < lv.nbox; s += G_TB) m2m_tiles.push_back(make_int4(l, 0, lv.off + s, std::min(G_TB, lv.nbox - s)));
    }
    ctx->m2m_first[depth] = (int)m2m_tiles.size();
    ctx->l2l_first = l2l_first;
    LF_TRY(lf_reserve(ctx->shift_tiles, (m2m_tiles.size() + l2l_tiles.size()) * sizeof(int4) + 16));
    ctx->l2l_tile_base = (int)m2m_tiles.size();
    if (!m2m_tiles.empty())
        LF_CHECK(cudaMemcpyAsync(ctx->shift_tiles.ptr, m2m_tiles.data(), m2m_tiles.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, st));
    if (!l2l_tiles.empty())
        LF_CHECK(cudaMemcpyAsync(ctx->shift_tiles.as<int4>() + m2m_tiles.size(), l2l_tiles.data(),
                                 l2l_tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    ctx->m2l_ntiles = (int)tiles.size();
    if (!tiles.empty()) {
        LF_TRY(lf_reserve(ctx->m2l_tiles, tiles.size() * sizeof(int4)));
        LF_CHECK(cudaMemcpyAsync(ctx->m2l_tiles.ptr, tiles.data(), tiles.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, st));
    }
    // wider tiles of the same (level, class) runs for the tensor-core kernel
    std::vector<int4>& tct = ctx->tc_tiles_h;
    tct.clear();
    ctx->m2l_tc_ntiles = 0;
    if (ctx->m2l_tc_ok) {
        const int TN = lf_m2l_tc_tile(ctx);
        m2l_tc_tiles(hcnt, depth, TN, tct, ctx->tc_mseg_h);
        ctx->m2l_tc_ntiles = (int)tct.size();
        // translations: M2M tiles of parents (levels 0 .. depth-1, box order),
        // L2L tiles of children grouped by octant (levels 1 .. depth)
        std::vector<int4>& sht = ctx->tc_shift_h;
        sht.clear();
        ctx->tc_m2m_first.assign(depth + 2, 0);
        ctx->tc_l2l_first.assign(depth + 2, 0);
        for (int l = 0; l <= depth; ++l) {
            ctx->tc_m2m_first[l] = (int)sht.size();
            const LfmmLevel& lv = ctx->levels[l];
            if (l < depth)
                for (int s = 0; s < lv.nbox; s += TN) sht.push_back(make_int4(l, 0, lv.off + s, std::min(TN, lv.nbox - s)));
        }
        ctx->tc_m2m_first[depth + 1] = (int)sht.size();
        int st1 = 0;
        for (int l = 1; l <= depth; ++l) {
            ctx->tc_l2l_first[l] = (int)sht.size();
            for (int c = 0; c < 8; ++c) {
                const int n = hcnt[16 + l * 8 + c];
                for (int s = 0; s < n; s += TN) sht.push_back(make_int4(l, c, st1 + s, std::min(TN, n - s)));
                st1 += n;
            }
        }
        ctx->tc_l2l_first[0] = ctx->tc_l2l_first[1];
        ctx->tc_l2l_first[depth + 1] = (int)sht.size();
        if (!sht.empty()) {
            LF_TRY(lf_reserve(ctx->tc_shift_tiles, sht.size() * sizeof(int4)));
            LF_CHECK(cudaMemcpyAsync(ctx->tc_shift_tiles.ptr, sht.data(), sht.size() * sizeof(int4),
                                     cudaMemcpyHostToDevice, st));
        }
        if (!tct.empty()) {
            LF_TRY(lf_reserve(ctx->m2l_tc_tiles, tct.size() * sizeof(int4)));
            LF_CHECK(cudaMemcpyAsync(ctx->m2l_tc_tiles.ptr, tct.data(), tct.size() * sizeof(int4),
                                     cudaMemcpyHostToDevice, st));
        }
        const std::vector<int4>& segs = ctx->tc_mseg_h;
        LF_TRY(lf_reserve(ctx->tc_mseg, segs.size() * sizeof(int4) + 16));
        if (!segs.empty())
            LF_CHECK(cudaMemcpyAsync(ctx->tc_mseg.ptr, segs.data(), segs.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                     st));
    }
    double* hl = ctx->m2l_levelh_h;
    for (int l = 0; l < 16; ++l) hl[l] = (l <= depth) ? ctx->levels[l].h : 0.0;
    LF_TRY(lf_reserve(ctx->m2l_levelh, sizeof(double) * 16));
    LF_CHECK(cudaMemcpyAsync(ctx->m2l_levelh.ptr, hl, sizeof(double) * 16, cudaMemcpyHostToDevice, st));
    // (host staging lives in the context; the build synchronises at its end)
    ctx->shift_ready = 1;
    return LfErr();
}

// ---------------------------------------------------------------------------
// The GEMM kernel.  Thread (rg, cg): rows rg*RM .. rg*RM+RM-1 of the packed
// output, columns 4cg .. 4cg+3 of the tile.  X is stored column-major
// [j][k] with stride KP+1 (conflict-free gathers and reads).
// ---------------------------------------------------------------------------
struct GemmArgs {
    int p, nc, RP;
    int noff;           // offsets (gathered sources) per target: 189 (M2L), 8 (M2M), 1 (L2L)
    int mode;           // 0: L += D / h_level (M2L), 1: L = D, 2: L += D (L2L), 3: atomic L += D (M2M)
    int split;          // 1: one block per (tile, offset) instead of one per tile
    int tile_base;      // first tile of this launch
    const int4* tiles;  // level, class, start, count
    const int* sorted;  // targets grouped by class, or null: targets start .. start + count - 1
    const int* slots;   // [target][noff] source box, or -1
    const int* cls;     // [class][noff] operator index
    const double* levelh;
    const void* A;
    const void* M;
    void* L;
    size_t mstride, lstride;  // per right-hand side (blockIdx.y), in elements
};

template <typename R, int RM, bool COMPF = false>
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
    const int tix = g.split ? (int)blockIdx.x / g.noff : (int)blockIdx.x;
    const int4 tile = g.tiles[g.tile_base + tix];
    const int level = tile.x, cls = tile.y, start = tile.z, cnt = tile.w;
    const int nc = g.nc;
    const R* A = reinterpret_cast<const R*>(g.A);
    const R* M = reinterpret_cast<const R*>(g.M) + (size_t)blockIdx.y * g.mstride;
    R* L = reinterpret_cast<R*>(g.L) + (size_t)blockIdx.y * g.lstride;
    if (tid < G_TB) s_tb[tid] = (tid < cnt) ? (g.sorted ? g.sorted[start + tid] : start + tid) : -1;
    // float32 free M2L (COMPF): each offset's products are summed into a
    // fresh partial, which is then added into the total with compensation
    // (Kahan), so that the rounding of the (p+1)^2 x 189 additions per output
    // does not pile up in one float.  FP64, and the translations between
    // levels (at most 8 offsets), sum directly.
    constexpr bool COMP = COMPF && sizeof(R) == 4;
    constexpr int RC = COMP ? RM : 1;
    R acc[RM][4], part[RC][4], cmp[RC][4];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0;
#pragma unroll
    for (int r = 0; r < RC; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) part[r][c] = cmp[r][c] = 0;
    __syncthreads();
    const int noff = g.noff;
    const int oi0 = g.split ? (int)blockIdx.x % noff : 0, oi1 = g.split ? oi0 + 1 : noff;
    for (int oi = oi0; oi < oi1; ++oi) {
        const int o = g.cls[cls * noff + oi];
        const int sj = (tid < cnt) ? g.slots[(size_t)s_tb[tid] * noff + oi] : -1;
        if (tid < G_TB) s_src[tid] = sj;
        // block-uniform: skip offsets where no target of the tile has a source
        if (!__syncthreads_or(sj >= 0)) continue;
        // gather the source multipoles: column j = source of target j (k fastest)
        // eight loads in flight per thread before their stores
        for (int b0 = tid; b0 < G_TB * KP; b0 += 8 * G_T) {
            R v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = b0 + u * G_T;
                v[u] = R(0);
                if (idx < G_TB * KP) {
                    const int j = idx / KP, k = idx - j * KP;
                    const int s = s_src[j];
                    if (s >= 0 && k < nc) v[u] = M[(size_t)s * nc + k];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = b0 + u * G_T;
                if (idx < G_TB * KP) {
                    const int j = idx / KP, k = idx - j * KP;
                    sX[j * XS + k] = v[u];
                }
            }
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
                    for (int c = 0; c < 4; ++c) {
                        if constexpr (COMP)
                            part[r][c] += a[r] * x[c];
                        else
                            acc[r][c] += a[r] * x[c];
                    }
            }
        }
        __syncthreads();
        if constexpr (COMP) {
#pragma unroll
            for (int r = 0; r < RM; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const R y = part[r][c] - cmp[r][c];
                    const R t = acc[r][c] + y;
                    cmp[r][c] = (t - acc[r][c]) - y;
                    acc[r][c] = t;
                    part[r][c] = 0;
                }
        }
    }
    if constexpr (COMP) {
#pragma unroll
        for (int r = 0; r < RM; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] -= cmp[r][c];
    }
    const R ih = (g.mode == 0) ? (R)(1.0 / g.levelh[level]) : R(1);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int j = 4 * cg + c;
        if (j >= cnt) continue;
        R* Lt = L + (size_t)s_tb[j] * nc;
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            int row = rg * RM + r;
            if (row < nc) {
                if (g.mode == 1)
                    Lt[row] = acc[r][c];
                else if (g.mode == 3)
                    atomicAdd(Lt + row, acc[r][c]);
                else if (g.split)
                    atomicAdd(Lt + row, acc[r][c] * ih);
                else
                    Lt[row] += acc[r][c] * ih;
            }
        }
    }
}

template <typename R, int RM>
static LfErr launch_gemm(lfmm_ctx* ctx, cudaStream_t st, const GemmArgs& g, int ntiles)
{
    if (ntiles <= 0) return LfErr();
    constexpr int RP = 16 * RM;
    size_t sm = sizeof(R) * ((size_t)G_KC * RP + (size_t)G_TB * (RP + 1));
    const int nblk = g.split ? ntiles * g.noff : ntiles;
    // compensated sums where one block adds many offsets into one output
    if constexpr (sizeof(R) == 4) {
        if (g.noff == G_NOFF && !g.split) {
            LF_CHECK(cudaFuncSetAttribute(k_m2l_gemm<R, RM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm));
            ++ctx->launches, k_m2l_gemm<R, RM, true><<<dim3(nblk, ctx->nrhs_b), G_T, sm, st>>>(g);
            return lf_cuda(cudaGetLastError(), "gathered gemm");
        }
    }
    {
        LF_CHECK(cudaFuncSetAttribute(k_m2l_gemm<R, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        ++ctx->launches, k_m2l_gemm<R, RM><<<dim3(nblk, ctx->nrhs_b), G_T, sm, st>>>(g);
    }
    return lf_cuda(cudaGetLastError(), "gathered gemm");
}

template <typename R>
static LfErr launch_gemm_rm(lfmm_ctx* ctx, cudaStream_t st, const GemmArgs& g, int ntiles)
{
    switch (ctx->m2l_rm) {
    case 2: return launch_gemm<R, 2>(ctx, st, g, ntiles);
    case 4: return launch_gemm<R, 4>(ctx, st, g, ntiles);
    case 8: return launch_gemm<R, 8>(ctx, st, g, ntiles);
    case 12: return launch_gemm<R, 12>(ctx, st, g, ntiles);
    case 16: return launch_gemm<R, 16>(ctx, st, g, ntiles);
    default: return "internal: unsupported GEMM tile";
    }
}

template <typename R>
static LfErr m2l_gemm_t(lfmm_ctx* ctx, cudaStream_t st)
{
    GemmArgs g;
    g.p = ctx->p;
    g.nc = lf_nc(ctx->p);
    g.RP = ctx->m2l_rp;
    g.noff = G_NOFF;
    g.mode = 0;
    g.split = 0;
    g.tile_base = 0;
    g.tiles = ctx->m2l_tiles.as<int4>();
    g.sorted = ctx->m2l_sorted.as<int>();
    g.slots = ctx->m2l_slots.as<int>();
    g.cls = ctx->m2l_cls.as<int>();
    g.levelh = ctx->m2l_levelh.as<double>();
    g.A = sizeof(R) == 8 ? ctx->m2l_A64.ptr : ctx->m2l_A32.ptr;
    g.M = ctx->Mexp.ptr;
    g.L = ctx->Lexp.ptr;
    g.mstride = g.lstride = (size_t)ctx->nbox_total * g.nc;
    // too few tiles to fill the SMs (small trees): one block per (tile, offset), summed by atomics
    g.split = (int64_t)ctx->m2l_ntiles * ctx->nrhs_b < 4 * 152;
    return launch_gemm_rm<R>(ctx, st, g, ctx->m2l_ntiles);
}

// M2M into the parents of `level` (mode store) or L2L into the boxes of `level`
template <typename R>
static LfErr shift_gemm_t(lfmm_ctx* ctx, int level, bool l2l, cudaStream_t st)
{
    // The L2L into the leaves runs on the tensor cores in the float32 form
    // (the CUDA-core gather of parent locals is latency-bound there).  The
    // other translations stay on the CUDA cores: at N = 1M, p = 10 the
    // tensor-core M2M saved 0.05 ms, and chaining 3xTF32 L2L over every level
    // raised Err2(phi) from 2.0e-6 to 3.2e-6.
    if (sizeof(R) == 4 && l2l && level == ctx->depth && lf_tc_on(ctx) && !ctx->m2l_tc_wide)
        return lf_shift_tc(ctx, level, l2l, st);
    GemmArgs g;
    g.p = ctx->p;
    g.nc = lf_nc(ctx->p);
    g.RP = ctx->m2l_rp;
    g.levelh = ctx->m2l_levelh.as<double>();
    g.cls = ctx->shift_cls.as<int>();
    g.tiles = ctx->shift_tiles.as<int4>();
    g.mstride = g.lstride = (size_t)ctx->nbox_total * g.nc;
    int first, ntiles;
    g.split = 0;
    if (!l2l) {
        // one block per (tile of parents, child octant), summed by atomics
        g.noff = 8;
        g.mode = 3;
        g.split = 1;
        g.sorted = nullptr;
        g.slots = ctx->m2m_slots.as<int>();
        g.A = sizeof(R) == 8 ? ctx->m2m_A64.ptr : ctx->m2m_A32.ptr;
        g.M = ctx->Mexp.ptr;
        g.L = ctx->Mexp.ptr;
        first = ctx->m2m_first[level];
        ntiles = ctx->m2m_first[level + 1] - first;
        const LfmmLevel& lv = ctx->levels[level];
        LF_CHECK(cudaMemset2DAsync(reinterpret_cast<R*>(ctx->Mexp.ptr) + (size_t)lv.off * g.nc, g.mstride * sizeof(R), 0,
                                   sizeof(R) * (size_t)lv.nbox * g.nc, ctx->nrhs_b, st));
    } else {
        g.noff = 1;
        g.mode = 2;
        g.sorted = ctx->m2l_sorted.as<int>();
        g.slots = ctx->box_parent.as<int>();
        g.A = sizeof(R) == 8 ? ctx->l2l_A64.ptr : ctx->l2l_A32.ptr;
        g.M = ctx->Lexp.ptr;
        g.L = ctx->Lexp.ptr;
        first = ctx->l2l_tile_base + ctx->l2l_first[level];
        ntiles = ctx->l2l_first[level + 1] - ctx->l2l_first[level];
    }
    g.tile_base = first;
    return launch_gemm_rm<R>(ctx, st, g, ntiles);
}

LfErr lf_shift_gemm(lfmm_ctx* ctx, int level, bool l2l, cudaStream_t st)
{
    return ctx->precision ? shift_gemm_t<float>(ctx, level, l2l, st) : shift_gemm_t<double>(ctx, level, l2l, st);
}

LfErr lf_m2l_gemm(lfmm_ctx* ctx, cudaStream_t st)
{
    if (ctx->m2l_ntiles == 0) return LfErr();
    return ctx->precision ? m2l_gemm_t<float>(ctx, st) : m2l_gemm_t<double>(ctx, st);
}
