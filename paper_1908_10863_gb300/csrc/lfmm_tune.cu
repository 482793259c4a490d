// lfmm_tune.cu -- run-time choice of the launch settings of one geometry.
//
// The settings trade stages against each other: a deeper tree (smaller leaf
// capacity) moves work from the near field (P2P) to the translations, the
// free M2L can run on the tensor cores or the CUDA cores, and small problems
// need each leaf's near list shared by several warps to fill the SMs.  Each
// candidate is timed with CUDA events on the context's stream.
#include <algorithm>
#include <cmath>

#include "lfmm_ctx.h"

namespace {

struct Setting {
    int leaf_cap, tc, split;
};

struct Tuner {
    lfmm_ctx* ctx;
    int64_t n;
    const double* xyz;
    const int32_t* layer;
    int mode, reps;
    double* q;  // device, one charge vector
    double* phi;
    double* fld;
    cudaEvent_t a = nullptr, b = nullptr;
    std::vector<double> rows;  // LFMM_TUNE_COLS per timed setting
    int built_cap = -1;

    void apply(const Setting& s)
    {
        ctx->leaf_cap = s.leaf_cap;
        ctx->use_tc = s.tc;
        ctx->p2p_split = s.split;
        ++ctx->serial;
    }

    // build the tree of the setting (mode 0 reuses a tree of the same leaf capacity)
    lfmm_status build(const Setting& s)
    {
        apply(s);
        if (built_cap == s.leaf_cap && mode == 0) return LFMM_OK;
        lfmm_status st = lf_build_dev(ctx, n, xyz, layer);
        built_cap = st == LFMM_OK ? s.leaf_cap : -1;
        return st;
    }

    lfmm_status once()
    {
        if (mode == 1) {
            lfmm_status st = lf_build_dev(ctx, n, xyz, layer);
            if (st != LFMM_OK) return st;
        }
        return lf_eval_enqueue(ctx, 1, q, phi, fld);
    }

    // median milliseconds of `reps` runs of the setting, after one untimed run
    lfmm_status time(const Setting& s, double* ms)
    {
        lfmm_status st = build(s);
        if (st == LFMM_OK) st = once();
        if (st != LFMM_OK) return st;
        std::vector<float> t;
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(a, ctx->s_main);
            st = once();
            if (st != LFMM_OK) return st;
            cudaEventRecord(b, ctx->s_main);
            cudaError_t ce = cudaEventSynchronize(b);
            if (ce != cudaSuccess) {
                ctx->err = lf_cuda(ce, "tuning run");
                return LFMM_ECUDA;
            }
            float v = 0.f;
            cudaEventElapsedTime(&v, a, b);
            t.push_back(v);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        const double row[LFMM_TUNE_COLS] = {(double)s.leaf_cap, (double)s.tc, (double)s.split, (double)ctx->depth,
                                            *ms, 0.0};
        rows.insert(rows.end(), row, row + LFMM_TUNE_COLS);
        return LFMM_OK;
    }
};

}  // namespace

extern "C" lfmm_status lfmm_autotune(lfmm_ctx* ctx, int64_t n, const double* xyz, const int32_t* layer, int mode,
                                     int reps, double* report, int max_rows, int* nrows)
{
    if (!ctx) return LFMM_EINVAL;
    ctx->err.clear();
    if (nrows) *nrows = 0;
    if (n < 1 || !xyz || !layer || (mode != 0 && mode != 1) || reps < 1 || (report && max_rows < 0)) {
        ctx->err = "EINVAL: need n >= 1, host arrays, mode 0 or 1, reps >= 1";
        return LFMM_EINVAL;
    }
    if (ctx->profile) {
        ctx->err = "ESTATE: turn profiling off while tuning";
        return LFMM_ESTATE;
    }
    // one validating host build puts the inputs on the device (ctx->xyz_in, ctx->layer_in)
    lfmm_status st = lfmm_build(ctx, n, xyz, layer);
    if (st != LFMM_OK) return st;
    LfErr e = lf_reserve(ctx->q_stage, (size_t)n * 8);
    if (e.empty()) e = lf_reserve(ctx->phi_stage, (size_t)n * 8);
    if (e.empty()) e = lf_reserve(ctx->fld_stage, (size_t)n * 24);
    if (e.empty()) {
        // the timing does not depend on the charge values
        std::vector<double> ones((size_t)n, 1.0);
        e = lf_cuda(cudaMemcpyAsync(ctx->q_stage.ptr, ones.data(), (size_t)n * 8, cudaMemcpyHostToDevice,
                                    ctx->s_main), "tuning charges");
        if (e.empty()) e = lf_cuda(cudaStreamSynchronize(ctx->s_main), "tuning charges");
    }
    if (!e.empty()) {
        ctx->err = e;
        return LFMM_ENOMEM;
    }
    Tuner T;
    T.ctx = ctx;
    T.n = n;
    T.xyz = ctx->xyz_in.as<double>();
    T.layer = ctx->layer_in.as<int32_t>();
    T.mode = mode;
    T.reps = reps;
    T.q = ctx->q_stage.as<double>();
    T.phi = ctx->phi_stage.as<double>();
    T.fld = ctx->fld_stage.as<double>();
    if (cudaEventCreate(&T.a) != cudaSuccess || cudaEventCreate(&T.b) != cudaSuccess) {
        if (T.a) cudaEventDestroy(T.a);
        ctx->err = "ECUDA: tuning events";
        return LFMM_ECUDA;
    }
    const Setting start{ctx->leaf_cap, ctx->use_tc, ctx->p2p_split};
    Setting best = start;
    double best_ms = INFINITY;
    auto consider = [&](const Setting& s) -> lfmm_status {
        double ms = 0.0;
        lfmm_status r = T.time(s, &ms);
        if (r == LFMM_OK && ms < best_ms) {
            best_ms = ms;
            best = s;
        }
        return r;
    };
    // 1. leaf capacity with the current settings (capacities that repeat a depth are skipped)
    std::vector<int> depths;
    const int caps[] = {10, 20, 40, 80, 160};
    for (int cap : caps) {
        if (st != LFMM_OK) break;
        Setting s{cap, start.tc, start.split};
        st = T.build(s);
        if (st != LFMM_OK) break;
        if (std::find(depths.begin(), depths.end(), ctx->depth) != depths.end()) continue;
        depths.push_back(ctx->depth);
        st = consider(s);
    }
    // 2. free M2L engine
    if (st == LFMM_OK && ctx->precision == 1 && ctx->m2l_tc_ok) {
        Setting s = best;
        // the other engine: off where the tensor cores run, on (at any order) where not
        const int saved = ctx->use_tc;
        ctx->use_tc = best.tc;
        s.tc = lf_tc_on(ctx) ? 0 : 1;
        ctx->use_tc = saved;
        st = consider(s);
    }
    // 3. near-list split (the automatic rule included)
    const int splits[] = {0, 1, 2, 4, 8, 16};
    const Setting base = best;
    for (int k : splits) {
        if (st != LFMM_OK) break;
        if (k == base.split) continue;
        Setting s = base;
        s.split = k;
        st = consider(s);
    }
    cudaEventDestroy(T.a);
    cudaEventDestroy(T.b);
    if (st != LFMM_OK) {
        T.apply(start);
        return st;
    }
    // keep the winner, built
    T.built_cap = -1;
    st = T.build(best);
    if (st != LFMM_OK) return st;
    const int nr = (int)(T.rows.size() / LFMM_TUNE_COLS);
    for (int r = 0; r < nr; ++r) {
        double* row = &T.rows[(size_t)r * LFMM_TUNE_COLS];
        if ((int)row[0] == best.leaf_cap && (int)row[1] == best.tc && (int)row[2] == best.split &&
            row[4] == best_ms)
            row[5] = 1.0;
    }
    if (report) {
        const int w = std::min(nr, max_rows);
        std::copy(T.rows.begin(), T.rows.begin() + (size_t)w * LFMM_TUNE_COLS, report);
        if (nrows) *nrows = w;
    } else if (nrows) {
        *nrows = nr;
    }
    return LFMM_OK;
}
