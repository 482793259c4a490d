/*
 * lfmm.h -- C ABI of the layered-media Laplace FMM for one GB300 (sm_103a).
 *
 * The library evaluates, for N point charges Q_j at r_j in a medium of L+1
 * horizontal layers (interfaces z = d_0 > d_1 > ... > d_{L-1}, permittivity
 * eps_l in layer l, layer 0 on top), the potential and field at every charge
 *
 *   Phi(r_i) = sum_{j != i, l_j = l_i} Q_j / (4 pi |r_i - r_j|)
 *            + sum_j Q_j u^r_{l_i l_j}(r_i, r_j),          E = -grad Phi,
 *
 * (Section 3.1, eqs. potential1, totalinteraction, freereactioncomponents of
 * Wang, Zhang & Cai, arXiv 1908.10863), where u^r is the reaction part of the
 * layered Green's function (eqs. reactioncomponent, generalcomponents,
 * zexponential).  The free-space part is computed by a classic FMM and each
 * reaction component by the FMM of Algorithm 1 on equivalent polarization
 * sources (eq. eqpolarizedsource), summed as in Algorithm 2.
 *
 * Conventions for every call:
 *   - All pointers are plain host or device pointers as stated per argument;
 *     the caller owns every array it passes and keeps ownership.  The library
 *     copies what it needs; no pointer is retained after a call returns.
 *   - Arrays of points are row-major [n][3] float64.
 *   - Results are written in the caller's order of the charges.
 *   - A context is not thread-safe: one host thread at a time.
 *   - No exception crosses the ABI.  A failing call returns a status other
 *     than LFMM_OK, leaves the context usable (or, for lfmm_create, sets *out
 *     to NULL) and stores a message readable with lfmm_last_error.
 *   - The library needs a CUDA device; it never computes on the host.
 */
#ifndef LFMM_H
#define LFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lfmm_ctx lfmm_ctx;

typedef enum {
    LFMM_OK = 0,
    LFMM_EINVAL = 1,   /* invalid argument (sizes, layer ids, points on an interface, ...) */
    LFMM_ENOMEM = 2,   /* device or host allocation failed */
    LFMM_ECUDA = 3,    /* a CUDA runtime call failed (message holds the CUDA error) */
    LFMM_ESTATE = 4,   /* call out of order (e.g. evaluate before build) */
    LFMM_ETIMEOUT = 5, /* reserved: bounded device-side wait expired */
    LFMM_ENUMERIC = 6  /* non-finite input or result */
} lfmm_status;

/* Options for lfmm_set_option. */
enum {
    LFMM_OPT_PRECISION = 1, /* 0 = plain FP64 (default); 1 = FP32 P2P/M2L/L2P with
                               compensated far-field sums, FP64 Sommerfeld tables */
    LFMM_OPT_LEAF_CAP = 2,  /* octree leaf capacity (default 40) */
    LFMM_OPT_PROFILE = 3,   /* 1 = time every stage with CUDA events (lfmm_get_timings) */
    LFMM_OPT_QUAD_NODES = 4, /* Gauss-Laguerre nodes of the M2L remainder integrals (16..128, default 64) */
    LFMM_OPT_SURROGATE = 5,  /* 1 = near-field reaction kernels by the trained network (default 0) */
    LFMM_OPT_SURROGATE_TOL = 6, /* error estimate above which a pair falls back to quadrature (default 1e-6) */
    LFMM_OPT_TENSOR_CORES = 7,  /* float32 free M2L engine: 2 = automatic (default): tensor cores (3xTF32)
                                   where (p+1)^2 <= 128, the compensated CUDA-core sums above; 1 = tensor
                                   cores at every order (for 11 <= p <= 14 the wide form: Err2 of the
                                   potential ~8e-7 at p = 14 against ~4e-7 on the CUDA cores, in a sixth
                                   of the time); 0 = CUDA cores.  Where (p+1)^2 <= 128 the tensor cores
                                   also take the L2L into the leaves and the keyed reaction M2L (each
                                   key's operator formed in shared memory from its Sommerfeld table,
                                   eqs. metoleimage1, coefintable); 0 puts both on the CUDA cores. */
    LFMM_OPT_P2P_SPLIT = 8,     /* near list of a leaf shared by this many warps/blocks of the P2P kernels:
                                   0 = chosen from the leaf count (default), else 1, 2, 4, 8 or 16 */
    LFMM_OPT_TC_GROUPS = 9,     /* tensor-core free M2L: CTAs per tile of targets (256, or 128 in the wide
                                   form), each summing 189/groups offsets in its tensor-memory accumulator
                                   before a float atomic add; a divisor of 189, or 0 = automatic (default:
                                   27, i.e. 7 offsets per accumulation; 63 in the wide form) */
    LFMM_OPT_NEAR_TABLES = 10,  /* near-field reaction kernels: 2 = automatic (default): the float32 form
                                   takes the remainder from pre-computed tables (deviation from the
                                   quadrature ~2e-8, see lfmm_near_tables) once a build's near lists hold
                                   reaction pairs, building them at the end of that build (once per
                                   context), the FP64 form keeps the quadrature; 1 = tables in both forms
                                   (built on first use); 0 = quadrature */
    LFMM_OPT_TC_PERSISTENT = 11, /* tensor-core free M2L: 1 = one persistent CTA per SM walking the
                                   (tile, offset group) units with a double-buffered accumulator, for
                                   launches of at least 4 units per SM; 0 = one CTA per unit, two CTAs per
                                   SM (default; measured as fast at N = 1M).  Same arithmetic and result. */
    LFMM_OPT_P2P_STAGED = 12,   /* float32 near field with one charge vector and no reaction pairs in the near
                                   lists: 1 = each warp stages its leaf's whole near list once (default);
                                   0 = staging per source box.  Same pairs either way. */
    LFMM_OPT_SERIAL_NEAR = 13   /* 1 = run the near field on the calling stream before the far field instead
                                   of beside it (then its stage time in lfmm_get_timings is the near-field
                                   kernels' own duration); 0 = concurrent (default).  Same result. */
};

/* Create a context for the medium.
 *   d   : host, L interface heights, strictly decreasing (Section 3.1).
 *   L   : number of interfaces, 0 <= L <= 4 (one to five layers).  With
 *         three or four interfaces the reaction densities are evaluated by
 *         solving the interface problem of Appendix A at each quadrature node
 *         (the learned near-field kernels stay limited to three layers); when
 *         the interface gaps share a unit, grid planes contain the interfaces
 *         and the reaction M2L uses its keyed tables on the aligned levels.
 *         Five layers take three bits of a box key for the layer id, so their
 *         trees stop at level 9.
 *   eps : host, L+1 permittivities > 0, layer 0 on top.
 *   p   : truncation order of all expansions, 1 <= p <= 20 (FP64) and
 *         p <= 14 in the FP32 form.
 *   out : receives the context, or NULL on failure.
 * Selects CUDA device 0 unless a device is already current. */
lfmm_status lfmm_create(const double* d, int L, const double* eps, int p, lfmm_ctx** out);

/* Set one option (see LFMM_OPT_*). Takes effect at the next build/evaluate. */
lfmm_status lfmm_set_option(lfmm_ctx* ctx, int opt, double value);

/* Build the octree and interaction lists for n charges (Algorithm 1, first
 * two steps; Section 3.3 for the interface-aligned boxes).
 *   xyz   : host, [n][3] positions.
 *   layer : host, [n] layer ids, with d_l < z < d_{l-1} (eq. Laplaceeqlayer).
 * Points on or outside their layer's slab are rejected with LFMM_EINVAL.
 * n >= 1.  Replaces any previous build. */
lfmm_status lfmm_build(lfmm_ctx* ctx, int64_t n, const double* xyz, const int32_t* layer);

/* Same as lfmm_build with device-resident inputs, ordered on cuda_stream
 * (a cudaStream_t, or NULL for the legacy default stream).  Inputs must stay
 * valid until the call returns (it synchronises the stream). */
lfmm_status lfmm_build_device(lfmm_ctx* ctx, int64_t n, const double* xyz_dev, const int32_t* layer_dev,
                              void* cuda_stream);

/* Evaluate potentials and fields for nrhs charge vectors over the built
 * geometry (Algorithm 2).
 *   q     : host, [nrhs][n] charges in the caller's order.
 *   phi   : host, [nrhs][n] output potentials (1/(4 pi) included).
 *   field : host, [nrhs][n][3] output E = -grad Phi, or NULL to skip.
 * Returns LFMM_ESTATE before a successful build. */
lfmm_status lfmm_evaluate(lfmm_ctx* ctx, int nrhs, const double* q, double* phi, double* field);

/* Same with device arrays (float64), ordered on cuda_stream; returns once the
 * work is enqueued on that stream (no host synchronisation). */
lfmm_status lfmm_evaluate_device(lfmm_ctx* ctx, int nrhs, const double* q_dev, double* phi_dev, double* field_dev,
                                 void* cuda_stream);

/* Pre-computed tables for the near-field reaction kernels (Section 4's
 * "pre-computed tables" variant, here for I_00, I_10, I_11 of each reaction
 * component): the closed-form leading image stays exact; the remainder,
 * scaled as T_N = Z^{N+1} r_N with Z = h + zeta_r, is tabulated over
 * s = rho / Z in [0, 4] and w = zeta_r / Z in [0, 1] (257 x 129 points,
 * FP64, the M2L quadrature rule) and read by fourth-order Lagrange
 * interpolation; pairs beyond the table keep the quadrature.  Builds the
 * tables if needed (once per context) and writes the largest deviation of the
 * interpolated kernels from the quadrature at 2048 seeded points per
 * component, relative to |I_00| (field kernels times the distance), to
 * *max_rel_err (may be NULL).  Does not change LFMM_OPT_NEAR_TABLES: with its
 * automatic default the float32 form uses built tables wherever the near
 * lists hold reaction pairs; the float32 kernels read a float32 copy. */
lfmm_status lfmm_near_tables(lfmm_ctx* ctx, double* max_rel_err);

/* Self-check of failure detection (the paper has no counterpart).  Every
 * wait of the device pipelines is bounded: when one runs out, the kernel
 * counts a timeout, releases what it holds and returns, and the evaluate
 * reports LFMM_ETIMEOUT.  This call exercises that path on purpose: one
 * thread waits on a barrier that will never complete, with a budget of
 * limit_ms milliseconds (0 < limit_ms <= 2000).  Returns LFMM_ETIMEOUT when
 * the wait ran out and was reported (the expected outcome); the context
 * stays usable and its timeout counter is cleared. */
lfmm_status lfmm_check_bounded_wait(lfmm_ctx* ctx, double limit_ms);

/* Message of the last failed call on ctx ("" if none); valid until the next call. */
const char* lfmm_last_error(const lfmm_ctx* ctx);

/* Release every resource of ctx.  NULL is allowed. */
void lfmm_destroy(lfmm_ctx* ctx);

/* ---- tuning ------------------------------------------------------------- */

/* Pick the launch settings of this geometry by timing them on the device
 * (CUDA events on the context's stream); the paper tunes nothing at run time,
 * this is a library facility.  Coordinate search, in this order:
 *   1. leaf capacity (tree depth) in {10, 20, 40, 80, 160};
 *   2. float32 form: free M2L on the other engine (CUDA cores where the
 *      tensor cores run, tensor cores at any order where not);
 *   3. near-list split of the P2P kernels in {automatic, 1, 2, 4, 8, 16}.
 * Each setting is timed as the median of `reps` (>= 1) evaluations of one
 * charge vector (mode 0) or builds plus evaluations (mode 1), after one
 * untimed run.  Afterwards the options hold the winner and ctx is built
 * with it.
 *   xyz, layer : host arrays as for lfmm_build.
 *   report     : host [max_rows][LFMM_TUNE_COLS] or NULL: leaf capacity,
 *                tensor cores, split, tree depth, milliseconds, 1 for the winner.
 *   nrows      : rows written (may be NULL). */
#define LFMM_TUNE_COLS 6
lfmm_status lfmm_autotune(lfmm_ctx* ctx, int64_t n, const double* xyz, const int32_t* layer, int mode, int reps,
                          double* report, int max_rows, int* nrows);

/* ---- many independent problems in one launch --------------------------- */

/* A batch of k built contexts (independent problems: own geometry, own
 * medium), evaluated together.  The paper evaluates one problem at a time;
 * batching is a library interface for workloads of many uneven problems.
 *   ctxs      : k distinct built contexts; they must outlive the batch.
 *   nrhs      : charge vectors per problem (NULL: one each).
 *   use_graph : 1 = capture the batch's launches once into a CUDA graph and
 *               replay it (one cudaGraphLaunch per evaluation, the problems'
 *               kernels as concurrent graph branches); 0 = launch them
 *               directly every time, on the same concurrent streams.
 * Charges, potentials and fields are concatenated over the problems:
 * problem i occupies [off_i, off_{i+1}) of q and phi ([nrhs_i][n_i] inside,
 * charges in that context's input order) and [3 off_i, 3 off_{i+1}) of the
 * field (lfmm_batch_offsets gives off).
 * Rebuilding a member or changing one of its options is allowed: the next
 * evaluation sees the changed serial of that context, runs directly once and
 * captures again.  Members must not be evaluated on their own while a batch
 * evaluation is in flight, and must not have profiling on (LFMM_ESTATE). */
typedef struct lfmm_batch lfmm_batch;
lfmm_status lfmm_batch_create(lfmm_ctx* const* ctxs, int k, const int* nrhs, int use_graph, lfmm_batch** out);

/* off[0..k]: prefix sums of n_i * nrhs_i (host array of k + 1 entries). */
lfmm_status lfmm_batch_offsets(const lfmm_batch* b, int64_t* off);

/* Evaluate every problem from device arrays (float64, layout above), ordered
 * on cuda_stream.  Returns once the work is enqueued, except on the first
 * call and after a member changed: that call launches directly, waits for it
 * (these launches size every buffer) and captures the graph for the next
 * calls.  Different array addresses than at capture time trigger a new
 * capture (no direct run).  field_dev may be NULL. */
lfmm_status lfmm_batch_evaluate_device(lfmm_batch* b, const double* q_dev, double* phi_dev, double* field_dev,
                                       void* cuda_stream);

/* Same with host arrays: copies in, evaluates, copies out and checks every
 * problem's bounded device waits (LFMM_ETIMEOUT if one ran out). */
lfmm_status lfmm_batch_evaluate(lfmm_batch* b, const double* q, double* phi, double* field);

/* Counters (host array of up to LFMM_BATCH_INFO_COUNT int64). */
enum {
    LFMM_BATCH_PROBLEMS = 0,
    LFMM_BATCH_CHARGES = 1,        /* sum of n_i * nrhs_i */
    LFMM_BATCH_GRAPH_NODES = 2,    /* nodes of the captured graph (0 if none) */
    LFMM_BATCH_KERNEL_NODES = 3,   /* of which kernel launches */
    LFMM_BATCH_CAPTURES = 4,
    LFMM_BATCH_GRAPH_LAUNCHES = 5,
    LFMM_BATCH_DIRECT_RUNS = 6,
    LFMM_BATCH_TIMEOUTS = 7,       /* device waits that ran out in the last evaluation (synchronises) */
    LFMM_BATCH_INFO_COUNT = 8
};
lfmm_status lfmm_batch_info(lfmm_batch* b, int64_t* out, int nout);

/* Tune the batch as a whole: a coordinate search over settings applied to
 * every member, each timed as the median of `reps` (>= 1) graph replays of
 * the whole batch (CUDA events on the batch's stream, after the direct run
 * and capture a changed setting brings), with unit charges:
 *   1. tensor-core free M2L (float32 form) for every member, for none, or for
 *      the members of at least 20,000 / 60,000 charges;
 *   2. near-list split of the P2P kernels: automatic, 1, 2, 4, 8;
 *   3. near-field reaction kernels by quadrature (0) or from the pre-computed
 *      tables (1; members whose near lists hold reaction pairs; see
 *      lfmm_near_tables).  The members' automatic default already takes the
 *      tables in the float32 form.
 * A member tuned alone picks the settings that fill the GPU with its own
 * work; in a batch the members fill it together, which is what this times.
 * Afterwards every member holds the winner.  Needs use_graph = 1.
 *   report : host [max_rows][LFMM_BATCH_TUNE_COLS] or NULL: smallest member
 *            size on the tensor cores (> every size: none), split, tables,
 *            milliseconds, 1 for the winner.
 *   nrows  : rows written (may be NULL). */
#define LFMM_BATCH_TUNE_COLS 5
lfmm_status lfmm_batch_autotune(lfmm_batch* b, int reps, double* report, int max_rows, int* nrows);

/* Message of the last failed batch call ("" if none). */
const char* lfmm_batch_last_error(const lfmm_batch* b);

/* Release the batch (not its contexts).  NULL is allowed. */
void lfmm_batch_destroy(lfmm_batch* b);

/* ---- inspection and measurement --------------------------------------- */

/* Counters of the current build (host array of at least LFMM_STAT_COUNT
 * int64 entries, see LFMM_STAT_*). */
enum {
    LFMM_STAT_N = 0,
    LFMM_STAT_DEPTH = 1,
    LFMM_STAT_BOXES = 2,          /* all levels, all layers */
    LFMM_STAT_LEAVES = 3,
    LFMM_STAT_M2L_FREE = 4,       /* free-space M2L box pairs, all levels */
    LFMM_STAT_M2L_REACTION = 5,   /* reaction M2L box pairs, all levels and components */
    LFMM_STAT_P2P_FREE = 6,       /* free-space near-field particle pairs (incl. i == j slots) */
    LFMM_STAT_P2P_REACTION = 7,   /* reaction near-field particle pairs */
    LFMM_STAT_COMPONENTS = 8,     /* free + reaction components of the medium */
    LFMM_STAT_M2M_EDGES = 9,      /* parent-child edges (also the L2L count) */
    LFMM_STAT_LAUNCHES = 10,      /* kernels launched by this context since lfmm_create (cumulative) */
    LFMM_STAT_REACTION_KEYS = 11, /* distinct (component, level, offset) reaction M2L operators */
    LFMM_STAT_SURR_NET = 12,      /* near-field reaction pairs of the last evaluate done by the network */
    LFMM_STAT_SURR_QUAD = 13,     /* ... and by the quadrature */
    LFMM_STAT_TIMEOUTS = 14,      /* bounded device waits of the last evaluate that ran out (0 expected) */
    LFMM_STAT_REACTION_TABLES = 15, /* Sommerfeld tables behind the reaction M2L keys (one per component,
                                       level, lateral distance and vertical offset) */
    LFMM_STAT_COUNT = 16
};
lfmm_status lfmm_get_stats(const lfmm_ctx* ctx, int64_t* out, int nout);

/* Stage timings of the last evaluate in milliseconds (needs
 * LFMM_OPT_PROFILE = 1), host array of LFMM_TIME_COUNT doubles. */
enum {
    LFMM_TIME_P2M = 0,
    LFMM_TIME_M2M = 1,
    LFMM_TIME_M2L_FREE = 2,
    LFMM_TIME_M2L_REACTION = 3,
    LFMM_TIME_L2L = 4,
    LFMM_TIME_L2P = 5,
    LFMM_TIME_P2P = 6,
    LFMM_TIME_TOTAL = 7,
    LFMM_TIME_BUILD = 8,
    LFMM_TIME_COUNT = 12
};
lfmm_status lfmm_get_timings(const lfmm_ctx* ctx, double* out, int nout);

/* Sommerfeld-type integral tables of one reaction component, as used by the
 * reaction M2L (eqs. uniformintegral, scaledsommerfeldint; Section 3.4), for
 * npts geometries on the device:
 *   comp : (l, lp, a, b) of the component (a, b in {1, 2}).
 *   rho, z : host, [npts] horizontal distance and vertical separation
 *            (z > 0: |z_c^t - z_c^{ab}|) in physical units.
 *   S    : box size used for scaling (eq. scaledsommerfeldint).
 *   out  : host, [npts][2P+1][2P+1] row-major (N, mu), the unnormalised,
 *          scaled integral S^{N+1} int_0^inf J_mu(k rho) k^N e^{-kz}
 *          sigma(k) dk for 0 <= mu <= N <= 2P (other entries 0).
 *   P    : expansion order (tables cover N <= 2P).
 * Computed by the same device routine as the M2L kernel. */
lfmm_status lfmm_sommerfeld_tables(lfmm_ctx* ctx, int l, int lp, int a, int b, int npts, const double* rho,
                                   const double* z, double S, int P, double* out);

/* Reaction kernel values of one component for npts (rho, h) pairs on the
 * device: out[i][0..2] = (int J0 e^{-kh} sigma dk, int k J0 e^{-kh} sigma dk,
 * int k J1 e^{-kh} sigma dk), the quantities of the near-field interactions
 * of Algorithm 1 (I_00 and its derivatives).  Host arrays. */
lfmm_status lfmm_reaction_kernel(lfmm_ctx* ctx, int l, int lp, int a, int b, int npts, const double* rho,
                                 const double* h, double* out);

/* ---- learned surrogate of the near-field reaction kernels --------------
 * Not in the paper: a small network per reaction component (4 inputs, three
 * hidden layers of 64 with SiLU, 3 outputs; bfloat16 weights, float32
 * accumulation) replaces the quadrature of the near-field integrals I_00,
 * I_10, I_11 (Algorithm 1, local direct interactions) where its validated
 * error is below LFMM_OPT_SURROGATE_TOL; elsewhere the quadrature is kept. */

/* Train the networks of every reaction component of a three-layer medium on
 * the device: nsamples (rho, h_t, h_s) samples per component (1000 .. 2^26),
 * rho log-uniform in [1e-3, 3], the depths below/above the interfaces
 * uniform in [0, d0 - d1] for half the samples and log-uniform in
 * [1e-4, d0 - d1] for the rest, labelled by the FP64 quadrature; epochs
 * passes of Adam over them; a tenth as many held-out samples (at least
 * 4096) fill the per-cell error table (32 x 32 cells of log10 rho by
 * log10 h).  Deterministic for a given seed.  Replaces earlier networks. */
lfmm_status lfmm_surrogate_train(lfmm_ctx* ctx, int64_t nsamples, int epochs, uint64_t seed);

/* Training summary of component (l, lp, a, b): out[0] trained (0/1), out[1]
 * maximum validation error (relative to the kernel scale below), out[2] fraction of
 * error-table cells at or below the tolerance, out[3] final training loss,
 * out[4] training samples, out[5] validation samples, out[6] fraction of the
 * validation samples that fall in accepted cells.  Errors are measured
 * against the pair's kernel scale |C| / R + |c_r| / R_r (I_00; squared
 * distances for I_10, I_11), C e^{-k zeta} the density's leading image and
 * c_r e^{-k zeta_r} its remainder's.  Host array of 8. */
lfmm_status lfmm_surrogate_info(const lfmm_ctx* ctx, int l, int lp, int a, int b, double* out);

/* Network values for npts pairs (host arrays): rho, target depth ht and
 * source depth hs (h = ht + hs); out[i][0..3] = (I_00, I_10, I_11 by the
 * network, 1 if the error table accepts the pair else 0). */
lfmm_status lfmm_surrogate_eval(lfmm_ctx* ctx, int l, int lp, int a, int b, int npts, const double* rho,
                                const double* ht, const double* hs, double* out);

/* Master (float32) parameters of one component's network, LFMM_SURR_NPARAM
 * floats in the order W1[64][4], b1[64], W2[64][64], b2[64], W3[64][64],
 * b3[64], W4[3][64], b4[3].  get reads them, set replaces them and re-derives
 * that network's bfloat16 inference weights (allocating the network state on
 * first use; the error table and standardisation are left as they are). */
#define LFMM_SURR_NPARAM 8835
lfmm_status lfmm_surrogate_get_params(const lfmm_ctx* ctx, int l, int lp, int a, int b, float* theta);
lfmm_status lfmm_surrogate_set_params(lfmm_ctx* ctx, int l, int lp, int a, int b, const float* theta);

/* Raw network outputs y[n][3] (standardised remainders) for features
 * x[n][4] (host arrays), by the same warp-level bfloat16 tensor-core kernel
 * the near field uses. */
lfmm_status lfmm_surrogate_forward(lfmm_ctx* ctx, int l, int lp, int a, int b, int n, const float* x, float* y);

/* Loss (1/n) sum (out - y)^2 and its gradient with respect to the master
 * parameters for n samples (host arrays x[n][4], y[n][3]; n a multiple of
 * 64), computed by the training kernels with the current parameters
 * (forward with bfloat16-rounded weights). */
lfmm_status lfmm_surrogate_loss_grad(lfmm_ctx* ctx, int l, int lp, int a, int b, int n, const float* x,
                                     const float* y, double* loss, float* grad);

/* Allocation-free variant of lfmm_reaction_kernel, for callers that may not
 * allocate device memory during the call: real-time or embedded loops whose
 * rules forbid allocator calls after start-up, and hosts on which another
 * runtime owns the device-memory budget.  The paper has no counterpart; this
 * is a library interface only.
 * Same arguments and results as lfmm_reaction_kernel (host arrays, copied in
 * and out; the call waits for the context's stream).  Inputs and outputs are
 * staged through one static device array shared by all calls
 * (LFMM_NOALLOC_MAX_POINTS points, 2.6 MB per GPU that loads the library, held
 * until process exit); the call makes no cudaMalloc / cudaFree.
 *   npts : 1 <= npts <= LFMM_NOALLOC_MAX_POINTS, else LFMM_EINVAL.
 * The context's device must be the current device (else LFMM_EINVAL).  The
 * first call on a device resolves the array's device address, so that first
 * call should come before any stream capture.  Calls that overlap on the GPU
 * race on the shared array: serialise them. */
#define LFMM_NOALLOC_MAX_POINTS 65536
lfmm_status lfmm_reaction_kernel_noalloc(lfmm_ctx* ctx, int l, int lp, int a, int b, int npts, const double* rho,
                                         const double* h, double* out);

/* Host-only helper (no device needed): Gauss-Laguerre nodes and weights of
 * order Q (weight e^{-t} on [0, inf)) as used by the quadratures. */
lfmm_status lfmm_gauss_laguerre(int Q, double* nodes, double* weights);

/* Host-only helper (no device needed): the components a context for this
 * medium would evaluate (Section 3.3, eqs. generalcomponents, zexponential,
 * eqpolarizedsource), the free-space ones first.
 *   d, L, eps : as for lfmm_create (EINVAL under the same conditions).
 *   out       : host, max_rows x LFMM_MEDIUM_COLS doubles, row-major, or NULL;
 *               per component (l, lp, a, b, is_free, s, o, iface, C, zeta,
 *               zeta_r): target layer l, source layer lp, the polarization
 *               map z'' = s z' + o, the interface between targets and
 *               polarization sources, the density's leading term
 *               C exp(-k zeta), and the decay rate zeta_r of the remainder
 *               sigma - C exp(-k zeta) (-1 where there is none).  a = b = 0
 *               for free-space components.
 *   nrows     : receives the component count (also when out is too small).
 * With out given and max_rows below the component count nothing is written
 * and the call returns LFMM_EINVAL: call with out = NULL first to learn the
 * count.  The caller owns out. */
#define LFMM_MEDIUM_COLS 11
lfmm_status lfmm_medium_components(const double* d, int L, const double* eps, double* out, int max_rows,
                                   int* nrows);

#ifdef __cplusplus
}
#endif
#endif /* LFMM_H */
