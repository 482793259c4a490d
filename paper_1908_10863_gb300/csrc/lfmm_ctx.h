// lfmm_ctx.h -- host-side context of the layered-media FMM library and the
// launcher functions each translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lfmm.h"
#include "lfmm_internal.cuh"

// Grow-only device buffer owned by the context.
struct DevBuf {
    void* ptr = nullptr;
    size_t cap = 0;
    template <typename T>
    T* as() const { return reinterpret_cast<T*>(ptr); }
};

// Status from a launcher: empty string = fine, else the error message.
using LfErr = std::string;

struct LfmmLevel {
    int nbox = 0;
    int off = 0;      // first global box id
    double h = 0.0;   // box size
    // list CSR offsets into the global near / m2l entry arrays
    int64_t near_base = 0, m2l_base = 0, m2r_base = 0;
    int64_t near_count = 0, m2l_count = 0, m2r_count = 0;  // near, free M2L, reaction M2L
};

struct lfmm_ctx {
    // medium and order
    int L = 0;
    double d[LFMM_MAXL] = {0};
    double eps[LFMM_MAXL + 1] = {1, 1, 1, 1, 1};
    int p = 0;
    // options
    int precision = 0;
    int leaf_cap = 40;
    int profile = 0;
    int quad_nodes = 64;
    int quad_nodes_near = 32;
    int near_pole = 0;  // the interface problem has a pole just left of k = 0 (x = e^{-kD} in (1, 1.5])
    std::string err;
    // bumped by every successful build, option change and surrogate update:
    // a captured evaluation is valid only for the serial it was captured at
    uint64_t serial = 0;
    int p2p_split = 0;  // near-list sharing of the P2P kernels (0: by occupancy)

    // components
    int ncomp = 0;
    LfmmComp comp[LFMM_MAXCOMP];

    // device and streams
    int device = 0;
    cudaStream_t s_main = nullptr, s_near = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<cudaEvent_t> prof_ev;

    // quadrature tables (device): [Qm2l] then [Qnear] nodes/weights
    DevBuf gl_t_m2l, gl_w_m2l, gl_t_near, gl_w_near;
    int gl_q_m2l = 0, gl_q_near = 0;

    // free-space M2L tables per offset (box units), [343][(2p+1)^2] (FP64 and FP32)
    DevBuf free_T64, free_T32;
    // regular harmonics of the 8 child offsets (+-1/4)^3, [8][2*NRE] (re, im)
    DevBuf oct_U64, oct_U32;
    DevBuf comp_dev;  // LfmmComp[ncomp]

    // geometry of the grid
    bool built = false;
    int64_t n = 0;
    int nrhs_b = 1;
    // wider separation for high orders: far-field pairs also need a centre
    // distance of at least sqrt(6) boxes (set at create for p >= LFMM_SEP_EXT_P)
    int sep_ext = 0;  // right-hand sides of the evaluation in flight (expansions [nrhs_b][boxes][nc])
    int depth = 0;
    double H = 1.0;
    double origin[3] = {0, 0, 0};
    int nlayer_used[LFMM_MAXL + 1] = {0};
    std::vector<LfmmLevel> levels;  // index = level 0..depth
    int nbox_total = 0;

    // particle data (sorted order)
    DevBuf perm;          // int32 [n]: sorted index -> caller index
    DevBuf xs, ys, zs;    // double [n]
    DevBuf keys, keys_tmp, vals_tmp, scan_tmp, hist;
    DevBuf keys_tmp2, vals_tmp2, scan_tmp2, hist2;  // the same scratch for the build's second stream
    DevBuf xyz_in, layer_in;  // staging of host inputs
    DevBuf err_flag;          // int [4]
    DevBuf counts;            // misc small counters

    // boxes (global ids)
    DevBuf box_key;     // uint32
    DevBuf box_pbeg;    // int32
    DevBuf box_pend;    // int32
    DevBuf box_parent;  // int32
    DevBuf box_cbeg;    // int32 (first child id, -1 for leaves)
    DevBuf box_cend;    // int32
    DevBuf box_center;  // LfD4 (x, y, z, layer)
    DevBuf box_grid;    // int4 (ix, iy, iz, layer): grid cell of the box at its level
    DevBuf pos_rel;  // float4 per sorted charge: offset from its leaf centre
    DevBuf leaf_of;  // leaf (global box id) of each sorted charge
    DevBuf level_consts;  // float4 [LFMM_MAXCOMP][16]: (K, F, G, Z) of the list tests, in box units
    DevBuf p2p_consts;    // float4 [LFMM_MAXCOMP]: (s, K, is_free, 0) at the leaf level, for the float32 near field
    int tc_persistent = 0;     // free M2L on the tensor cores: persistent kernel (1) or one CTA per work unit (0)
    int num_sms = 152;
    int p2p_staged = 1;        // float32 free-space near field: staged-list kernel (1) or per-box staging (0)
    int serial_near = 0;       // 1: near field on the calling stream before the far field (no overlap)
    int leaf_int_offsets = 0;  // 1: every polarization image of a leaf box is a leaf grid cell (K integral)
    DevBuf flags, idx;  // temporaries

    // lists: offsets per level box (near_off[level_box] relative to level base) and entries
    DevBuf near_off, near_ent, m2l_off, m2l_ent, m2r_off, m2r_ent;
    int64_t near_total = 0, m2l_total = 0, m2r_total = 0;
    int64_t list_cap[3] = {0, 0, 0};  // near, free M2L, reaction M2L entry capacities (grow-only)

    // free-space M2L as per-offset GEMMs (p <= 15)
    DevBuf m2l_A64, m2l_A32, m2l_cls, m2l_inv, m2l_slots, m2l_keys, m2l_sorted, m2l_tiles, m2l_levelh;
    int m2l_rm = 0, m2l_rp = 0, m2l_ntiles = 0;
    // tensor-core free M2L (float32 form, (p+1)^2 <= 128)
    DevBuf m2l_Atc, m2l_tc_tiles, m2l_Ms;
    DevBuf tc_mseg;  // runs of the merged tensor-core tiles, [merged tile][LFMM_TC_MSEG] int4 (level, start, count, 0)
    DevBuf m2m_Atc, l2l_Atc, tc_shift_tiles;        // tensor-core M2M / L2L operators and tiles
    std::vector<int> tc_m2m_first, tc_l2l_first;    // first tensor-core translation tile of each level
    std::vector<int4> tc_shift_h;
    // M2M / L2L as gathered GEMMs (the same kernel as the free M2L)
    DevBuf m2m_A64, m2m_A32, l2l_A64, l2l_A32, shift_cls, m2m_slots, shift_tiles;
    std::vector<int> m2m_first, l2l_first;  // first tile of each level
    int l2l_tile_base = 0, shift_ready = 0;
    std::vector<int4> m2l_tiles_h, l2l_tiles_h, m2m_tiles_h, tc_tiles_h, tc_mseg_h;  // host staging of asynchronous uploads
    std::vector<float4> level_consts_h;
    std::vector<float4> p2p_consts_h;
    void* host_pin = nullptr;  // small pinned host buffer for readbacks that must not wait
    DevBuf near_tab;            // remainder tables of the near-field reaction kernels
    DevBuf near_tab4;           // their float32 copy, one float4 per grid point (float32 kernels)
    int near_tab_ready = 0;
    int use_near_tab = 2;       // 0 quadrature, 1 tables, 2 tables in the float32 form (default)
    double near_tab_err = -1.0;  // largest relative deviation from the quadrature at the check points
    double m2l_levelh_h[16] = {0};
    // use_tc: 2 automatic (tensor cores where (p+1)^2 <= 128), 1 at every order, 0 never
    int m2l_tc_ok = 0, m2l_tc_ntiles = 0, use_tc = 2, tc_groups = 0;  // tc_groups 0: automatic
    int m2l_tc_wide = 0;  // tensor-core free M2L in its wide form ((p+1)^2 > 128): no tensor-core M2M / L2L
    // reaction M2L grouped by geometry key on interface-aligned levels
    DevBuf m2r_keys, m2r_order, m2r_tgt, m2r_kstart, m2r_kval, m2r_tables, m2r_levelh, m2r_batches;
    DevBuf m2r_tdesc, m2r_ktab;  // table descriptors (component, level, rho^2, oz); table of each key
    std::vector<int4> m2r_tdesc_h, m2r_batches_h;  // host staging of asynchronous uploads
    int m2r_pending_ne = 0;             // reaction M2L entries whose key grouping awaits lf_prepare_m2r_finish
    int m2r_la = 0;                     // first level with reaction M2L entries (keyed from there if in range)
    int m2r_kfirst = 0;                 // first key of the keyed levels among the sorted keys
    DevBuf m2r_zfrac, m2r_zbase;        // per (component, level): image offset fraction and integer base
    int64_t near_reaction_entries = 0;  // leaf-level near entries of reaction components (last build)
    int p2p_stats_stale = 0;            // the particle-pair statistics wait for lf_p2p_pair_stats
    std::vector<int> m2r_slot_h;                   // reaction table lookup: slot per (rho^2, oz)
    std::vector<int> m2r_kstart_h;                 // key starts and values read back (when the
    std::vector<uint32_t> m2r_kval_h;              // pinned buffer is too small for them)
    std::vector<uint32_t> m2r_stamp_h;             // and the generation that filled it
    std::vector<int> m2r_ktab_h;
    double m2r_levelh_h[16] = {0};
    int m2r_nkeys = 0, m2r_nbatch = 0, m2r_keyed_from = 0, m2r_ntab = 0;
    DevBuf m2r_ops;         // assembled operator per key, [nkeys][RP][RP] in the precision below
    DevBuf m2r_phase;       // float32 e^{i m phi} of the 225 lateral key offsets, m <= 2p (tensor-core form)
    int m2r_phase_p = -1;   // order the phase table holds
    DevBuf m2r_pairs;       // int2 (source box, target box) per sorted reaction entry
    int m2r_nent = 0;       // sorted reaction entries
    int m2r_ops_prec = -1;  // 0 FP64, 1 FP32, -1 not assembled for this build
    int m2r_dev_pending = 0;  // 1: the keys' tables and operators are still to be computed (first evaluation)
    cudaEvent_t ev_m2r = nullptr;  // recorded after them on the stream that computed them
    int m2r_wait = 0;              // 1: the far field must wait for ev_m2r before the reaction M2L

    // learned surrogate of the near-field reaction kernels
    DevBuf surr_theta, surr_grad, surr_m1, surr_m2, surr_w, surr_b, surr_meta, surr_err, surr_comps, surr_xoff,
        surr_counters;
    int surr_ready = 0, use_surr = 0;
    double surr_tol = 1e-6;
    float surr_info[LFMM_MAXCOMP][8] = {{0}};
    LfmmSurrMeta surr_meta_h[LFMM_MAXCOMP] = {};

    // evaluation buffers
    DevBuf q_sorted;            // R [n]
    DevBuf Mexp, Lexp;          // R [nbox][(p+1)^2]
    DevBuf phi_far, phi_near;   // double [n]
    DevBuf fld_far, fld_near;   // double [n*3]
    DevBuf q_stage, phi_stage, fld_stage;  // host<->device staging for lfmm_evaluate

    // statistics
    int64_t launches = 0;  // kernels launched by this context since creation
    int64_t stats[16] = {0};
    double timings[12] = {0};
    // profiling: (slot, start, stop) event triples recorded during an evaluation
    struct ProfRec { int slot; cudaEvent_t a, b; };
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
    size_t prof_used = 0;
};

// ---- allocation helpers (lfmm_api.cu) ----
LfErr lf_reserve(DevBuf& b, size_t bytes);
LfErr lf_cuda(cudaError_t e, const char* what);
// The context's pinned host buffer, in regions for the build's read-backs:
// copies into pinned memory are queued without waiting, so each build phase
// synchronises once for all of its read-backs.
#define LFMM_PIN_BYTES (256 * 1024)
#define LFMM_PIN_ERR 0          // input check flags (4 ints)
#define LFMM_PIN_LEVELS 256     // boxes per level (16 ints)
#define LFMM_PIN_SCAN 512       // a scan's last input and output (2 ints)
#define LFMM_PIN_LIST 1024      // list statistics, overflow, counters, per-level snapshots (< 1 KB)
#define LFMM_PIN_M2L 2048       // free M2L class counts (144 ints)
#define LFMM_PIN_ROOT 2688      // root box keys (up to 128)
#define LFMM_PIN_BOUNDS 4096    // bounding-box partials (256 blocks x 6 doubles)
#define LFMM_PIN_UP 4096        // later in the build: root lists and list counters to upload (12 KB)
#define LFMM_PIN_M2R 16384      // reaction M2L key starts and values (the rest)
template <typename T>
inline T* lf_pin(const lfmm_ctx* ctx, size_t off)
{
    return reinterpret_cast<T*>(static_cast<char*>(ctx->host_pin) + off);
}
// device-to-host copy ordered after the work queued on st, complete on return
inline cudaError_t lf_d2h(void* dst, const void* src, size_t bytes, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
}

// ---- tree construction (lfmm_tree.cu) ----
LfErr lf_build_tree(lfmm_ctx* ctx, const double* xyz_dev, const int32_t* layer_dev, int64_t n, cudaStream_t st);
LfErr lf_p2p_pair_stats(lfmm_ctx* ctx);
// whether the float32 free M2L runs on the tensor cores: the automatic setting
// keeps the compensated CUDA-core sums for the wide form ((p+1)^2 > 128),
// where they are the more accurate choice
inline bool lf_tc_on(const lfmm_ctx* ctx)
{
    return ctx->m2l_tc_ok && (ctx->use_tc == 1 || (ctx->use_tc == 2 && !ctx->m2l_tc_wide));
}

// ---- free-space M2L GEMM (lfmm_m2l.cu) ----
LfErr lf_setup_m2l_ops(lfmm_ctx* ctx);
LfErr lf_prepare_m2l(lfmm_ctx* ctx, cudaStream_t st);
LfErr lf_m2l_gemm(lfmm_ctx* ctx, cudaStream_t st);
// ---- reaction M2L by geometry key (lfmm_m2r.cu) ----
LfErr lf_prepare_m2r(lfmm_ctx* ctx, cudaStream_t st);         // enqueue (no synchronisation)
LfErr lf_prepare_m2r_finish(lfmm_ctx* ctx, cudaStream_t st);  // synchronise st, host part
LfErr lf_m2r_apply(lfmm_ctx* ctx, cudaStream_t st);
LfErr lf_m2r_ops(lfmm_ctx* ctx, cudaStream_t st);
LfErr lf_m2r_device(lfmm_ctx* ctx, cudaStream_t st);
// stable LSD radix sort of uint32 (key, value) pairs (lfmm_tree.cu); uses keys_tmp, vals_tmp, hist
// (set 1: keys_tmp2, vals_tmp2, hist2)
LfErr lf_radix_sort(lfmm_ctx* ctx, uint32_t* keys, uint32_t* vals, int64_t n, cudaStream_t st, int first_pass = 0,
                    int npass = 4, int set = 0);

// ---- evaluation (lfmm_fmm.cu, lfmm_near.cu) ----
LfErr lf_evaluate_sorted(lfmm_ctx* ctx, int nrhs, const double* q_dev, double* phi_dev, double* field_dev,
                         cudaStream_t st);
// enqueue nrhs evaluations on ctx->s_main (no host synchronisation, no
// allocation once the buffers have grown to this size: capturable)
lfmm_status lf_eval_enqueue(lfmm_ctx* ctx, int nrhs, const double* q_dev, double* phi_dev, double* fld_dev);
// build from device inputs on ctx->s_main (synchronises it)
lfmm_status lf_build_dev(lfmm_ctx* ctx, int64_t n, const double* xyz_dev, const int32_t* layer_dev);
#define LFMM_P2P_SPLIT_MAX 16
// right-hand sides evaluated in one pass (larger requests are split)
#define LFMM_RHS_BATCH 64
#define LFMM_SEP_EXT_P 18
LfErr lf_near_field(lfmm_ctx* ctx, cudaStream_t st);
LfErr lf_near_prepare(lfmm_ctx* ctx, cudaStream_t st);
LfErr lf_near_tables(lfmm_ctx* ctx, double* max_err);

// ---- surrogate (lfmm_surrogate.cu) ----
LfErr lf_surrogate_train(lfmm_ctx* ctx, int64_t nsamples, int epochs, uint64_t seed);
LfErr lf_surrogate_eval_dev(lfmm_ctx* ctx, int comp, int n, const double* rho, const double* ht, const double* hs,
                            double* out);
LfErr lf_surrogate_grad_dev(lfmm_ctx* ctx, int comp, int n, const float* x, const float* ystd, double* loss,
                            float* grad);
LfErr lf_surrogate_device_view(lfmm_ctx* ctx, LfmmSurrView* v);

LfErr lf_shift_gemm(lfmm_ctx* ctx, int level, bool l2l, cudaStream_t st);

// ---- tensor-core free M2L (lfmm_m2l_tc.cu) ----
// byte offset in ctx->counts of the int counting device waits that ran out
#define LFMM_TIMEOUT_OFF 40960
#define LFMM_TC_MSEG 16  // runs per merged tensor-core M2L tile (one leftover run per level and class)
LfErr lf_setup_m2l_tc(lfmm_ctx* ctx, const double* A64, const double* M2M64, const double* L2L64, int KP, int RP);
LfErr lf_shift_tc(lfmm_ctx* ctx, int level, bool l2l, cudaStream_t st);
LfErr lf_wait_probe(lfmm_ctx* ctx, double limit_ms, int* timed_out);
LfErr lf_m2l_tc(lfmm_ctx* ctx, cudaStream_t st);
int lf_m2l_tc_tile(const lfmm_ctx* ctx);
LfErr lf_surrogate_alloc(lfmm_ctx* ctx);
LfErr lf_surrogate_pack(lfmm_ctx* ctx, int comp);
LfErr lf_surrogate_forward_dev(lfmm_ctx* ctx, int comp, int n, const float* x, float* y);

// ---- debug / parity kernels (lfmm_near.cu) ----
LfErr lf_sommerfeld_tables_dev(lfmm_ctx* ctx, int comp, int npts, const double* rho, const double* z, double S,
                               int P, double* out);
LfErr lf_reaction_kernel_dev(lfmm_ctx* ctx, int comp, int npts, const double* rho, const double* h, double* out);

// index of the reaction component (l, lp, a, b), or -1 (lfmm_api.cu)
int lf_find_comp(const lfmm_ctx* ctx, int l, int lp, int a, int b);

// exclusive scan of int32 (lfmm_tree.cu); returns the total through *total (host) if non-null
// set: scratch buffers 0 (the build's main stream) or 1 (its second stream)
LfErr lf_scan_i32(lfmm_ctx* ctx, const int* in, int* out, int64_t n, int64_t* total, cudaStream_t st, int set = 0);

// profile helpers: lf_prof_start returns a handle for lf_prof_stop (or -1 when off)
int lf_prof_start(lfmm_ctx* ctx, int slot, cudaStream_t st);
void lf_prof_stop(lfmm_ctx* ctx, int handle, cudaStream_t st);
