// lfmm_batch.cu -- many independent problems evaluated as one CUDA graph.
//
// Each problem is a built context (its own geometry and tree, any medium).
// One evaluation of the batch forks every context's stream from a root
// event, enqueues that context's whole evaluation (Algorithm 2: upward pass,
// M2L, downward pass, near field) on it and joins all of them back.  The first
// evaluation runs these launches directly (which also grows every context's
// buffers to their final size); it is then captured once into a graph, so the
// following evaluations are a single cudaGraphLaunch in which the problems'
// kernels run as concurrent branches.  No allocation and no host
// synchronisation happen inside the captured region.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lfmm_ctx.h"

struct lfmm_batch {
    std::vector<lfmm_ctx*> ctx;
    std::vector<int> nrhs;
    std::vector<int64_t> off;  // charges before problem i (concatenated [problem][nrhs_i][n_i])
    int use_graph = 1;
    std::string err;
    cudaStream_t s = nullptr;
    cudaEvent_t ev_root = nullptr, ev_in = nullptr, ev_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // what the graph was captured for
    const double* cq = nullptr;
    double* cphi = nullptr;
    double* cfld = nullptr;
    std::vector<uint64_t> serial;
    std::vector<uint64_t> launch_delta;  // kernels per problem in one evaluation
    DevBuf q_stage, phi_stage, fld_stage, flags;
    int64_t nodes = 0, kernel_nodes = 0, captures = 0, graph_launches = 0, direct_runs = 0;
};

static lfmm_status bfail(lfmm_batch* b, const std::string& e, lfmm_status s)
{
    b->err = e;
    return s;
}

static void drop_graph(lfmm_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Enqueue every problem on its own context stream, forked from and joined to b->s.
static lfmm_status enqueue_all(lfmm_batch* b, const double* q, double* phi, double* fld)
{
    cudaError_t ce = cudaEventRecord(b->ev_root, b->s);
    if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "batch fork"), LFMM_ECUDA);
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        lfmm_ctx* c = b->ctx[i];
        const int64_t o = b->off[i];
        ce = cudaStreamWaitEvent(c->s_main, b->ev_root, 0);
        if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "batch fork"), LFMM_ECUDA);
        const uint64_t l0 = c->launches;
        lfmm_status st = lf_eval_enqueue(c, b->nrhs[i], q + o, phi + o, fld ? fld + 3 * o : nullptr);
        if (st != LFMM_OK) return bfail(b, "problem " + std::to_string(i) + ": " + c->err, st);
        b->launch_delta[i] = c->launches - l0;
        // this problem's count of device waits that ran out
        ce = cudaMemcpyAsync(b->flags.as<int>() + i, c->counts.as<char>() + LFMM_TIMEOUT_OFF, sizeof(int),
                             cudaMemcpyDeviceToDevice, c->s_main);
        if (ce == cudaSuccess) ce = cudaEventRecord(c->ev_join, c->s_main);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->s, c->ev_join, 0);
        if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "batch join"), LFMM_ECUDA);
    }
    return LFMM_OK;
}

static lfmm_status capture(lfmm_batch* b, const double* q, double* phi, double* fld)
{
    drop_graph(b);
    // relaxed: calls that are not stream work (function attributes, buffer
    // checks) stay legal while the problems' streams are being captured
    cudaError_t ce = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeRelaxed);
    if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "begin capture"), LFMM_ECUDA);
    lfmm_status st = enqueue_all(b, q, phi, fld);
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(b->s, &g);
    if (st != LFMM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "end capture"), LFMM_ECUDA);
    b->graph = g;
    ce = cudaGraphInstantiate(&b->exec, g, 0);
    if (ce != cudaSuccess) {
        drop_graph(b);
        return bfail(b, lf_cuda(ce, "instantiate graph"), LFMM_ECUDA);
    }
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    int64_t nk = 0;
    for (cudaGraphNode_t n : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(n, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
    }
    b->nodes = (int64_t)nn;
    b->kernel_nodes = nk;
    b->cq = q;
    b->cphi = phi;
    b->cfld = fld;
    ++b->captures;
    return LFMM_OK;
}

// Evaluate on b->s (the caller orders b->s against its own stream).
static lfmm_status run(lfmm_batch* b, const double* q, double* phi, double* fld)
{
    bool fresh = true;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        lfmm_ctx* c = b->ctx[i];
        if (!c->built) return bfail(b, "ESTATE: problem " + std::to_string(i) + " is not built", LFMM_ESTATE);
        if (c->profile) return bfail(b, "ESTATE: problem " + std::to_string(i) + " has profiling on", LFMM_ESTATE);
        if (c->serial != b->serial[i]) fresh = false;
    }
    if (!fresh || !b->use_graph) {
        // direct launches: the result of this call, and every buffer at its final size
        drop_graph(b);
        lfmm_status st = enqueue_all(b, q, phi, fld);
        if (st != LFMM_OK) return st;
        ++b->direct_runs;
        for (size_t i = 0; i < b->ctx.size(); ++i) b->serial[i] = b->ctx[i]->serial;
        if (!b->use_graph) return LFMM_OK;
        cudaError_t ce = cudaStreamSynchronize(b->s);
        if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "batch"), LFMM_ECUDA);
        return capture(b, q, phi, fld);  // captured, not launched: this call's result is already there
    }
    if (!b->exec || b->cq != q || b->cphi != phi || b->cfld != fld) {
        lfmm_status st = capture(b, q, phi, fld);
        if (st != LFMM_OK) return st;
    }
    cudaError_t ce = cudaGraphLaunch(b->exec, b->s);
    if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "graph launch"), LFMM_ECUDA);
    ++b->graph_launches;
    for (size_t i = 0; i < b->ctx.size(); ++i) b->ctx[i]->launches += b->launch_delta[i];
    return LFMM_OK;
}

extern "C" {

lfmm_status lfmm_batch_create(lfmm_ctx* const* ctxs, int k, const int* nrhs, int use_graph, lfmm_batch** out)
{
    if (!out) return LFMM_EINVAL;
    *out = nullptr;
    if (!ctxs || k < 1) return LFMM_EINVAL;
    for (int i = 0; i < k; ++i) {
        if (!ctxs[i]) return LFMM_EINVAL;
        if (nrhs && nrhs[i] < 1) return LFMM_EINVAL;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return LFMM_EINVAL;  // one context appears once
        if (!ctxs[i]->built) return LFMM_ESTATE;
    }
    lfmm_batch* b = new lfmm_batch();
    b->use_graph = use_graph != 0;
    b->off.assign(k + 1, 0);
    for (int i = 0; i < k; ++i) {
        b->ctx.push_back(ctxs[i]);
        b->nrhs.push_back(nrhs ? nrhs[i] : 1);
        b->off[i + 1] = b->off[i] + ctxs[i]->n * b->nrhs[i];
    }
    b->serial.assign(k, ~0ull);  // nothing captured yet
    b->launch_delta.assign(k, 0);
    int pr_lo = 0, pr_hi = 0;
    cudaError_t ce = cudaDeviceGetStreamPriorityRange(&pr_lo, &pr_hi);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&b->s, cudaStreamNonBlocking, pr_hi);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ev_root, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    LfErr e = ce == cudaSuccess ? LfErr() : lf_cuda(ce, "batch streams");
    if (e.empty()) e = lf_reserve(b->flags, sizeof(int) * (size_t)k);
    if (!e.empty()) {
        lfmm_batch_destroy(b);
        return LFMM_ECUDA;
    }
    *out = b;
    return LFMM_OK;
}

lfmm_status lfmm_batch_offsets(const lfmm_batch* b, int64_t* off)
{
    if (!b || !off) return LFMM_EINVAL;
    for (size_t i = 0; i < b->off.size(); ++i) off[i] = b->off[i];
    return LFMM_OK;
}

lfmm_status lfmm_batch_evaluate_device(lfmm_batch* b, const double* q_dev, double* phi_dev, double* field_dev,
                                       void* cuda_stream)
{
    if (!b) return LFMM_EINVAL;
    b->err.clear();
    if (!q_dev || !phi_dev) return bfail(b, "EINVAL: need q and phi", LFMM_EINVAL);
    cudaStream_t us = (cudaStream_t)cuda_stream;
    cudaError_t ce = cudaEventRecord(b->ev_in, us);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->s, b->ev_in, 0);
    if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "stream order"), LFMM_ECUDA);
    lfmm_status st = run(b, q_dev, phi_dev, field_dev);
    if (st != LFMM_OK) {
        cudaStreamSynchronize(b->s);
        return st;
    }
    ce = cudaEventRecord(b->ev_out, b->s);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(us, b->ev_out, 0);
    if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "stream order"), LFMM_ECUDA);
    return LFMM_OK;
}

lfmm_status lfmm_batch_evaluate(lfmm_batch* b, const double* q, double* phi, double* field)
{
    if (!b) return LFMM_EINVAL;
    b->err.clear();
    if (!q || !phi) return bfail(b, "EINVAL: need q and phi", LFMM_EINVAL);
    const int64_t n = b->off.back();
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(q[i])) return bfail(b, "ENUMERIC: non-finite charge", LFMM_ENUMERIC);
    LfErr e = lf_reserve(b->q_stage, (size_t)n * 8);
    if (e.empty()) e = lf_reserve(b->phi_stage, (size_t)n * 8);
    if (e.empty() && field) e = lf_reserve(b->fld_stage, (size_t)n * 24);
    if (!e.empty()) return bfail(b, e, LFMM_ENOMEM);
    cudaError_t ce = cudaMemcpyAsync(b->q_stage.ptr, q, (size_t)n * 8, cudaMemcpyHostToDevice, b->s);
    if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "copy charges"), LFMM_ECUDA);
    lfmm_status st = run(b, b->q_stage.as<double>(), b->phi_stage.as<double>(),
                         field ? b->fld_stage.as<double>() : nullptr);
    if (st != LFMM_OK) {
        cudaStreamSynchronize(b->s);
        return st;
    }
    std::vector<int> tmo(b->ctx.size(), 0);
    ce = cudaMemcpyAsync(phi, b->phi_stage.ptr, (size_t)n * 8, cudaMemcpyDeviceToHost, b->s);
    if (ce == cudaSuccess && field)
        ce = cudaMemcpyAsync(field, b->fld_stage.ptr, (size_t)n * 24, cudaMemcpyDeviceToHost, b->s);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(tmo.data(), b->flags.ptr, sizeof(int) * tmo.size(), cudaMemcpyDeviceToHost, b->s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->s);
    if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "batch evaluate"), LFMM_ECUDA);
    for (size_t i = 0; i < tmo.size(); ++i)
        if (tmo[i])
            return bfail(b, "ETIMEOUT: a device wait of problem " + std::to_string(i) + " ran out", LFMM_ETIMEOUT);
    return LFMM_OK;
}

// One candidate setting applied to every member: tensor-core free M2L for the
// members with at least tc_min charges (float32 form), near-list split, and
// the pre-computed near-field tables for members whose near lists hold
// reaction pairs.
struct BatchSetting {
    int64_t tc_min;
    int split;
    int tables;
};

static lfmm_status apply_setting(lfmm_batch* b, const BatchSetting& s)
{
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        lfmm_ctx* c = b->ctx[i];
        lfmm_status st = lfmm_set_option(c, LFMM_OPT_TENSOR_CORES, c->n >= s.tc_min ? 1.0 : 0.0);
        if (st == LFMM_OK) st = lfmm_set_option(c, LFMM_OPT_P2P_SPLIT, (double)s.split);
        const bool tab = s.tables && c->near_reaction_entries > 0;
        if (st == LFMM_OK) st = lfmm_set_option(c, LFMM_OPT_NEAR_TABLES, tab ? 1.0 : 0.0);
        if (st != LFMM_OK) return bfail(b, "problem " + std::to_string(i) + ": " + c->err, st);
    }
    return LFMM_OK;
}

// Median milliseconds of `reps` graph replays of the whole batch (after the
// direct run and capture that a changed setting brings).
static lfmm_status time_batch(lfmm_batch* b, int reps, double* ms)
{
    double* q = b->q_stage.as<double>();
    double* phi = b->phi_stage.as<double>();
    double* fld = b->fld_stage.as<double>();
    lfmm_status st = run(b, q, phi, fld);  // direct run + capture
    if (st == LFMM_OK) st = run(b, q, phi, fld);  // one replay
    if (st != LFMM_OK) return st;
    std::vector<float> t;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    for (int r = 0; r < reps && ce == cudaSuccess; ++r) {
        ce = cudaEventRecord(e0, b->s);
        if (ce == cudaSuccess && (st = run(b, q, phi, fld)) != LFMM_OK) break;
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, b->s);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float v = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&v, e0, e1);
        t.push_back(v);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != LFMM_OK) return st;
    if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "batch timing"), LFMM_ECUDA);
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return LFMM_OK;
}

lfmm_status lfmm_batch_autotune(lfmm_batch* b, int reps, double* report, int max_rows, int* nrows)
{
    if (!b) return LFMM_EINVAL;
    b->err.clear();
    if (nrows) *nrows = 0;
    if (reps < 1 || (report && max_rows < 0)) return bfail(b, "EINVAL: reps >= 1", LFMM_EINVAL);
    if (!b->use_graph) return bfail(b, "ESTATE: the tuner times graph replays (use_graph = 1)", LFMM_ESTATE);
    const int64_t n = b->off.back();
    // unit charges (timing does not depend on the values) in the batch's staging buffers
    LfErr e = lf_reserve(b->q_stage, (size_t)n * 8);
    if (e.empty()) e = lf_reserve(b->phi_stage, (size_t)n * 8);
    if (e.empty()) e = lf_reserve(b->fld_stage, (size_t)n * 24);
    if (!e.empty()) return bfail(b, e, LFMM_ENOMEM);
    {
        std::vector<double> ones((size_t)n, 1.0);
        cudaError_t ce = cudaMemcpyAsync(b->q_stage.ptr, ones.data(), (size_t)n * 8, cudaMemcpyHostToDevice, b->s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->s);
        if (ce != cudaSuccess) return bfail(b, lf_cuda(ce, "tuning charges"), LFMM_ECUDA);
    }
    int64_t nmax = 0;
    for (lfmm_ctx* c : b->ctx) nmax = std::max<int64_t>(nmax, c->n);
    std::vector<double> rows;
    auto timed = [&](const BatchSetting& s, double* ms) -> lfmm_status {
        lfmm_status st = apply_setting(b, s);
        if (st == LFMM_OK) st = time_batch(b, reps, ms);
        if (st == LFMM_OK) {
            const double r[LFMM_BATCH_TUNE_COLS] = {(double)std::min<int64_t>(s.tc_min, nmax + 1), (double)s.split,
                                                    (double)s.tables, *ms, 0.0};
            rows.insert(rows.end(), r, r + LFMM_BATCH_TUNE_COLS);
        }
        return st;
    };
    BatchSetting best{0, 0, 0};
    double best_ms = 0.0;
    lfmm_status st = timed(best, &best_ms);
    size_t best_row = 0;
    // 1. which members take the tensor-core free M2L (all, none, the larger ones)
    const int64_t tcs[3] = {nmax + 1, 20000, 60000};
    for (int i = 0; i < 3 && st == LFMM_OK; ++i) {
        BatchSetting s = best;
        s.tc_min = tcs[i];
        double ms = 0.0;
        st = timed(s, &ms);
        if (st == LFMM_OK && ms < best_ms) best = s, best_ms = ms, best_row = rows.size() / LFMM_BATCH_TUNE_COLS - 1;
    }
    // 2. near-list split
    const int splits[4] = {1, 2, 4, 8};
    for (int i = 0; i < 4 && st == LFMM_OK; ++i) {
        BatchSetting s = best;
        s.split = splits[i];
        double ms = 0.0;
        st = timed(s, &ms);
        if (st == LFMM_OK && ms < best_ms) best = s, best_ms = ms, best_row = rows.size() / LFMM_BATCH_TUNE_COLS - 1;
    }
    // 3. near-field reaction kernels from the pre-computed tables
    if (st == LFMM_OK) {
        BatchSetting s = best;
        s.tables = 1;
        double ms = 0.0;
        st = timed(s, &ms);
        if (st == LFMM_OK && ms < best_ms) best = s, best_ms = ms, best_row = rows.size() / LFMM_BATCH_TUNE_COLS - 1;
    }
    if (st == LFMM_OK) st = apply_setting(b, best);
    if (st != LFMM_OK) return st;
    rows[best_row * LFMM_BATCH_TUNE_COLS + 4] = 1.0;
    const int nr = (int)(rows.size() / LFMM_BATCH_TUNE_COLS);
    if (report) {
        const int w = std::min(nr, max_rows);
        std::copy(rows.begin(), rows.begin() + (size_t)w * LFMM_BATCH_TUNE_COLS, report);
        if (nrows) *nrows = w;
    } else if (nrows) {
        *nrows = nr;
    }
    return LFMM_OK;
}

lfmm_status lfmm_batch_info(lfmm_batch* b, int64_t* out, int nout)
{
    if (!b || !out || nout < 1) return LFMM_EINVAL;
    int64_t tmo = 0;
    std::vector<int> f(b->ctx.size(), 0);
    if (lf_d2h(f.data(), b->flags.ptr, sizeof(int) * f.size(), b->s) == cudaSuccess)
        for (int v : f) tmo += v;
    const int64_t v[LFMM_BATCH_INFO_COUNT] = {(int64_t)b->ctx.size(), b->off.back(), b->nodes, b->kernel_nodes,
                                              b->captures, b->graph_launches, b->direct_runs, tmo};
    for (int i = 0; i < nout && i < LFMM_BATCH_INFO_COUNT; ++i) out[i] = v[i];
    return LFMM_OK;
}

const char* lfmm_batch_last_error(const lfmm_batch* b) { return b ? b->err.c_str() : "null batch"; }

void lfmm_batch_destroy(lfmm_batch* b)
{
    if (!b) return;
    if (b->s) cudaStreamSynchronize(b->s);
    drop_graph(b);
    DevBuf* bufs[] = {&b->q_stage, &b->phi_stage, &b->fld_stage, &b->flags};
    for (DevBuf* d : bufs)
        if (d->ptr) cudaFree(d->ptr);
    if (b->ev_root) cudaEventDestroy(b->ev_root);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->s) cudaStreamDestroy(b->s);
    delete b;
}

}  // extern "C"
