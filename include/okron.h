/*
 * okron.h -- C ABI of libokron: exhaustive Kron-based reduction of unbalanced
 * three-phase radial distribution feeders on a GB300 (sm_103a) GPU.
 *
 * The method is Algorithm 1 ("Exhaustive Network Reduction") of Sec. IV of
 * "Optimal Kron-based reduction of three-phase distribution feeders"
 * (arXiv 2510.19608).  Starting from every bus being its own super-node, each
 * iteration evaluates every feasible assignment of one super-node's cluster to
 * an adjacent super-node (Sec. II-C rules: connectivity, phase availability,
 * uniqueness), solves the network with the aggregated injections -- which gives
 * the Kron-reduced super-node voltages of Sec. II-B -- scores the per-phase
 * voltage-magnitude error against the full network (MICE / SMICE, Sec. III),
 * rejects candidates whose error exceeds the margin, and commits the argmin.
 *
 * Conventions shared by every call
 *   - Buses are numbered 0..n_bus-1 by the caller; bus 0 is the substation
 *     (slack, fixed voltage) and parent[i] < i for i >= 1.  phases[i] is a bit
 *     mask (a = 1, b = 2, c = 4), non-empty, a subset of phases[parent[i]].
 *   - Complex numbers are two doubles (re, im).  Per-unit throughout.
 *   - Three-phase arrays are padded: x[..][bus][3][2]; entries of absent phases
 *     are ignored on input and written as 0 on output.
 *   - Every call returns an okr_status; no call aborts or throws.  On error the
 *     context keeps a message (okr_last_error) and the previous results are
 *     invalid.
 *   - A context owns one CUDA stream and its device memory; it is not thread
 *     safe.  Calls that run GPU work return after that work has finished.
 *   - Input arrays are caller-owned and only read during the call.  Output
 *     buffers are caller-owned and sized as documented per call.
 *
 * Readings of the paper taken by the library (where the text leaves a choice):
 *   the slack bus keeps its voltage and is never reduced (it may absorb a
 *   neighbour); a candidate moves the whole cluster of r into s and every member
 *   takes the super-node's voltage; the error is per phase,
 *   e = | |Vhat| - |V^c| |; MICE is the largest error in a cluster and SMICE
 *   sums it over clusters and scenarios; ties: every feasible candidate whose
 *   score is within tie_tol of the minimum is tied and the smallest (r, s) pair
 *   of caller bus ids wins; the scenario injections are Ihat = Y Vhat.
 */
#ifndef OKRON_H
#define OKRON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum okr_status {
    OKR_OK = 0,
    OKR_EINVAL = 1,     /* bad argument: null pointer, size, tree or phase rule broken */
    OKR_ENOMEM = 2,     /* host or device allocation failed */
    OKR_ECUDA = 3,      /* a CUDA runtime call failed (message in okr_last_error) */
    OKR_EPF = 4,        /* load flow did not converge */
    OKR_ETIMEOUT = 5,   /* a device-side wait gave up after its spin limit */
    OKR_ENOTREADY = 6,  /* no result is available yet */
    OKR_ESINGULAR = 7,  /* a line impedance block is singular */
    OKR_EINTERNAL = 8   /* internal bound exceeded (should not happen) */
} okr_status;

typedef struct okr_ctx okr_ctx;

/* A feeder (Sec. II-A network model).  Which memory the pointers refer to is
 * stated by each entry point. */
typedef struct okr_feeder {
    int32_t n_bus;              /* 2 .. 32768 */
    int32_t n_scen;             /* scenarios L, 1 .. 4 */
    const int32_t *parent;      /* [n_bus]; parent[0] = -1 */
    const uint8_t *phases;      /* [n_bus] */
    const double *z_line;       /* [n_bus][3][3][2] series impedance of line parent(i) -> i
                                   (row 0 unused); the block on phases[i] must be invertible */
    const double *s_load;       /* [n_scen][n_bus][3][2] constant-power load per phase
                                   (consumption positive) */
    double v_slack[3][2];       /* slack voltage per phase */
} okr_feeder;

/* Search parameters (Algorithm 1 inputs and the stop rule). */
typedef struct okr_params {
    double margin;              /* voltage-error bound E_bar (eq. v_abs), p.u., > 0 */
    double target_reduction;    /* stop after ceil(target * n_bus) merges (capped at
                                   n_bus - 1); 1.0 = run until no candidate is feasible */
    double tie_tol;             /* tie band tau on the score, >= 0 (default 1e-9) */
    int32_t objective;          /* 0 = SMICE (Algorithm 1); 1 = the largest per-phase error of the
                                   candidate network (the iteration objective of Sec. IV); other
                                   values are rejected */
    int32_t precision;          /* 0 = every candidate scored in FP64;
                                   1 = FP32 screen with a rigorous error bound, FP64 rescoring of
                                   the candidates the bound cannot separate, FP64 merges.  Both
                                   select the same candidate as an all-FP64 search. */
    int32_t record_iters;       /* keep every candidate's score for the first K iterations */
    int32_t max_merges;         /* >= 0 overrides the target; -1 = use target_reduction */
    int32_t profile;            /* 1 = count the search's arithmetic and time its sweep phase */
    int32_t scorer_topk;        /* 0 = exhaustive; k > 0 = evaluate exactly only the k candidates the
                                   learned scorer ranks best in each iteration (okr_scorer_init with
                                   OKR_SCORER_FEATURES inputs first).  An iteration whose k candidates
                                   are all infeasible is re-evaluated exhaustively.  The committed
                                   candidate is always exactly evaluated; it may differ from the
                                   exhaustive choice. */
    int32_t engine;             /* how the candidates are scored (all give the same decisions):
                                   OKR_ENGINE_AUTO (0): incremental when objective = 0 and
                                     scorer_topk = 0, otherwise the sweep;
                                   OKR_ENGINE_SWEEP (1): every iteration evaluates every candidate
                                     afresh (one persistent launch over all SMs);
                                   OKR_ENGINE_INCREMENTAL (2): every candidate's score is carried
                                     from one iteration to the next and only the terms whose inputs
                                     the last merge changed are evaluated again (exact: a carried
                                     score is a fixed-point sum of its terms; precision 0 carries FP64
                                     terms, precision 1 FP32 terms with a carried error bound and an
                                     FP64 rescoring where the bound cannot decide); one CTA per feeder.
                                     Needs objective 0 and scorer_topk 0 (else OKR_EINVAL);
                                     record_iters records scores but not scorer features;
                                   OKR_ENGINE_VERIFY (3): as 2, and after every merge every candidate
                                     is also evaluated afresh and compared bit for bit with its
                                     carried score (okr_summary.inc_mismatches; for tests). */
    int64_t max_spins;          /* polls before a device-side wait gives up with OKR_ETIMEOUT: the grid
                                   barriers of the load flow and of the sweep engine (0 = default,
                                   1,000,000: one L2 round trip each, under a second) */
    int32_t prune_exact;        /* 1 = certified pruning with the learned ordering (scorer_topk > 0,
                                   objective 0, precision 0, the sweep engine; else OKR_EINVAL): each
                                   iteration scores the scorer's top-k candidates exactly, then every
                                   other candidate whose certified lower bound on its score does not
                                   exclude it from the tie band; the decisions are the exhaustive
                                   search's.  The bound: a cluster evaluated at one voltage magnitude
                                   has MICE >= half the spread of its members' |Vhat|, so a merged
                                   cluster adds at least that half spread less the two MICE it
                                   replaces, and every other cluster at least its own half spread less
                                   its MICE.  okr_summary.pruned counts the candidates it excluded. */
    int32_t reserved;           /* 0 */
} okr_params;

#define OKR_ENGINE_AUTO 0
#define OKR_ENGINE_SWEEP 1
#define OKR_ENGINE_INCREMENTAL 2
#define OKR_ENGINE_VERIFY 3

typedef struct okr_summary {
    int32_t n_bus, n_scen;
    int32_t n_iter;             /* merges committed */
    int32_t stop_reason;        /* 0 target reached, 1 no feasible candidate */
    int32_t pf_sweeps;          /* load-flow sweeps (largest over scenarios; 0 if given) */
    int32_t n_kept;             /* super-nodes left */
    int64_t candidates;         /* candidates evaluated over the run */
    double smice;               /* SMICE of the final reduction */
    double max_error;           /* largest per-phase magnitude error of the final reduction */
    int64_t launches;           /* kernels launched by the last call */
    double search_ms;           /* duration of the search kernel (CUDA events on the
                                   library stream; the search runs as one persistent launch) */
    int64_t sweeps;             /* candidate sweeps run (one per iteration) */
    /* filled when params.profile = 1 (zero otherwise): */
    double sweep_ms;            /* time inside the sweep phase (device timer of CTA 0) */
    double flops;               /* algorithmic floating-point operations of the search */
    int32_t rechecks;           /* precision 1: iterations that rescored candidates in FP64 */
    int32_t recheck_cands;      /* precision 1: candidates rescored in FP64 over the run */
    double phase_ms[16];        /* profile mode: time of CTA 0 per step of an iteration.  Sweep engine:
                                   selection, FP64 recheck, merge, candidate setup, barrier, merge
                                   bookkeeping, list update, offsets, compaction, chunk map, barrier,
                                   sweep.  Incremental engine: selection, changed set, merge with the
                                   rebuilt candidates beside it, the terms that change (before and
                                   after the merge, one pass, with the write-back) */
    double kron_ms;             /* device time of the last okr_kron since the reduction (0 if none) */
    int32_t scorer_fallbacks;   /* learned pruning: iterations re-evaluated exhaustively because the
                                   scorer's k candidates were all infeasible */
    int32_t inc_mismatches;     /* OKR_ENGINE_VERIFY: carried scores that differed from a fresh
                                   evaluation, summed over the merges (0 when correct) */
    int32_t engine;             /* engine that ran: OKR_ENGINE_SWEEP or OKR_ENGINE_INCREMENTAL */
    int32_t pad;
    int64_t terms;              /* incremental engine, profile mode: (candidate, phase-node, scenario)
                                   items evaluated over the run, the initial evaluation, the merges'
                                   own evaluations and FP64 rescorings included (0 otherwise) */
    /* incremental engine: the launch shape that ran (okr_inc_shape's meaning; 0 for the sweep) */
    int32_t inc_threads, inc_eval_warps, inc_shared_entries, inc_records;
    int64_t pruned;             /* prune_exact: candidates excluded by the certified bound over the run */
} okr_summary;

/* Launch shape of the incremental engine (one CTA runs one feeder's search).
 * Every shape gives the same results; only the time differs.  Set per
 * context (okr_set_inc_shape), used by the later okr_reduce* and
 * okr_reduce_batch calls on it.  A field of 0 takes its default. */
typedef struct okr_inc_shape {
    int32_t threads;            /* threads of the CTA: 256, 384 or 512 (0 = 384) */
    int32_t eval_warps;         /* warps that evaluate the merge's own new values while the others
                                   find the changed candidates: 1 .. threads/32 - 1 (0 = 2, or 4
                                   with 512 threads) */
    int32_t shared_entries;     /* work entries of one merge kept in shared memory, 1 .. 256
                                   (0 = 256); the rest live in device memory */
    int32_t records;            /* where the per-candidate selection records live: 0 automatic
                                   (shared memory when it fits), 1 device memory, 2 shared memory,
                                   3 shared memory with the largest MICE per super-node (single-
                                   feeder searches only).  A forced placement that does not fit
                                   makes the reduction fail with OKR_EINVAL. */
} okr_inc_shape;

/* Sets the context's incremental-engine shape (NULL = every field default).
 * OKR_EINVAL for a value outside the ranges above. */
okr_status okr_set_inc_shape(okr_ctx *ctx, const okr_inc_shape *shape);
/* The context's shape with the defaults filled in (records 0 stays automatic). */
okr_status okr_get_inc_shape(const okr_ctx *ctx, okr_inc_shape *shape);

/* Autotuner of the incremental engine's shape: times the search kernel under
 * each of a fixed list of shapes (CTA sizes 256/384/512, evaluation-warp
 * splits, a smaller shared tile, records in device memory) on the caller's
 * workload -- one feeder through okr_reduce when n_feeders = 1, else the
 * batch through okr_reduce_batch -- two runs each, the faster counted, and
 * keeps the fastest shape on the context for later calls.  feeders: HOST,
 * as okr_reduce / okr_reduce_batch; params: [n_params], n_params = 1 or
 * n_feeders, selecting the incremental engine (else OKR_EINVAL).
 * best (may be NULL): the shape kept.  shapes, search_ms (may be NULL): the
 * first `cap` shapes tried and their search times in ms (infinity for a
 * shape whose record placement does not fit the workload); *n_tried (may be
 * NULL): how many shapes the list holds.  The results of the runs are those
 * of the last run (every shape gives the same results). */
okr_status okr_inc_autotune(okr_ctx *ctx, int32_t n_feeders, const okr_feeder *feeders, const okr_params *params,
                            int32_t n_params, okr_inc_shape *best, okr_inc_shape *shapes, double *search_ms,
                            int32_t cap, int32_t *n_tried);

/* Fills *p with the defaults: margin 0.005, target 1.0, tie_tol 1e-9,
 * objective 0, precision 0, record_iters 0, max_merges -1, profile 0, scorer_topk 0,
 * engine OKR_ENGINE_AUTO, max_spins 0, prune_exact 0. */
void okr_default_params(okr_params *p);

/* Creates a context on CUDA device `device`.  stream: a cudaStream_t to run
 * on, or NULL for a stream owned by the context.  *ctx is library-owned until
 * okr_destroy.  Device memory is allocated lazily by the first reduction and
 * grown when a larger feeder arrives. */
okr_status okr_create(okr_ctx **ctx, int device, void *stream);
okr_status okr_destroy(okr_ctx *ctx);
const char *okr_status_str(okr_status s);
const char *okr_last_error(const okr_ctx *ctx);

/* Device memory from the caller's allocator (e.g. a framework's caching
 * allocator, so that the library's workspace is accounted for and reused
 * there).  Every device allocation of the context -- its workspace, batch
 * arenas, batch plans, Y_Kron and scorer buffers -- then calls
 * alloc(user, bytes, device, stream) and later free(user, ptr, device,
 * stream), with the context's device and stream; pinned host staging is
 * unaffected.  alloc returns NULL on failure (the call then returns
 * OKR_ENOMEM) and must return memory usable by work on `stream` at once.
 * The library frees a block only after the work on its stream that used it
 * has finished.  Without a registered allocator the context uses
 * cudaMalloc / cudaFree.  Must be called before the context's first device
 * allocation (right after okr_create), else OKR_EINVAL; alloc = free = NULL
 * restores cudaMalloc / cudaFree under the same condition. */
typedef void *(*okr_alloc_fn)(void *user, size_t bytes, int device, void *stream);
typedef void (*okr_free_fn)(void *user, void *ptr, int device, void *stream);
okr_status okr_set_allocator(okr_ctx *ctx, okr_alloc_fn alloc, okr_free_fn free_fn, void *user);

/* Full path (Sec. III operating points, then Algorithm 1): load flow of every
 * scenario by backward/forward sweep, Ihat = Y Vhat, then the search.  Feeder
 * arrays in HOST memory (copied to the device inside the call). */
okr_status okr_reduce(okr_ctx *ctx, const okr_feeder *f, const okr_params *p);

/* Same as okr_reduce with the feeder arrays (parent, phases, z_line, s_load)
 * already in DEVICE memory of the context's device; v_slack is read from *f. */
okr_status okr_reduce_device(okr_ctx *ctx, const okr_feeder *f, const okr_params *p);

/* Algorithm 1 with a caller-supplied scenario library (its inputs Vhat, Ihat
 * with Y Vhat = Ihat), HOST memory, [n_scen][n_bus][3][2] each; s_load unused. */
okr_status okr_reduce_ops(okr_ctx *ctx, const okr_feeder *f, const double *vhat,
                          const double *ihat, const okr_params *p);

/* Load flow only (HOST feeder).  vhat_out: [n_scen][n_bus][3][2], ihat_out
 * (may be NULL): Y Vhat, same layout; *sweeps (may be NULL): sweeps used. */
okr_status okr_power_flow(okr_ctx *ctx, const okr_feeder *f, double *vhat_out, double *ihat_out,
                          int32_t *sweeps);

/* Y_Kron (Sec. II-B, eqs. (Y-partitioned) and (Y_kron)): the Kron-reduced
 * admittance matrix Y_KK - Y_KR Y_RR^-1 Y_RK of the feeder of the last
 * okr_reduce* / okr_power_flow call onto a kept bus set, over the kept
 * phase-nodes, the slack bus included.
 *
 * kept: HOST [n_bus] flags in caller numbering (bus 0 must be kept), or NULL
 *   for the super-nodes of the last reduction (the network the search chose).
 * *k_phi (required): number of kept phase-nodes.  Pass y_out = phase_node =
 *   NULL to query it alone.
 * y_out (HOST, may be NULL): [k_phi][k_phi][2] complex, row-major, rows and
 *   columns in phase_node order; needs cap >= k_phi.
 * phase_node (HOST, may be NULL): [k_phi], caller bus * 3 + phase, ordered by
 *   bus then phase.
 * Computed in FP64 on the device: one small dense elimination per connected
 * component of reduced buses.  Errors: OKR_ENOTREADY without a feeder (or
 * without a reduction when kept is NULL); OKR_EINVAL if bus 0 is not kept,
 * cap < k_phi, or a reduced component borders more than 1024 kept
 * phase-nodes; OKR_ESINGULAR for a singular block. */
okr_status okr_kron(okr_ctx *ctx, const uint8_t *kept, int32_t cap, double *y_out,
                    int32_t *phase_node, int32_t *k_phi);

/* ---- many feeders in one launch ----------------------------------------
 * Result of one feeder of okr_reduce_batch. */
typedef struct okr_batch_item {
    int32_t status;             /* okr_status of this feeder */
    int32_t n_iter;             /* merges committed */
    int32_t stop_reason;        /* 0 target reached, 1 no feasible candidate */
    int32_t n_kept;             /* super-nodes left */
    int64_t candidates;         /* candidates evaluated */
    double smice;               /* SMICE of the final reduction */
    double max_error;           /* largest per-phase error of the final reduction */
} okr_batch_item;

typedef struct okr_batch_stats {
    double setup_ms;            /* device time of the setup of every feeder (load flows included) */
    double search_ms;           /* device time of the batched search launch(es) */
    int64_t candidates;         /* over all feeders */
    int32_t config;             /* team shape: 0/1/2/3 = 1/2/4/8 CTAs (512 threads each) per feeder */
    int32_t ctas;               /* CTAs of the batched search launch */
    int32_t fallbacks;          /* feeders re-run alone because their work buffer was too small */
    int32_t reserved;
} okr_batch_stats;

/* Algorithm 1 for many independent feeders (Sec. IV; the candidates of one
 * feeder are independent, and so are feeders): one batched setup of every
 * feeder (load flows included), then ONE persistent cooperative launch in
 * which each team of CTAs takes the next feeder from a queue ordered
 * largest-first and runs that feeder's whole search (teams of 1, 2, 4 or 8
 * CTAs, chosen by okr_batch_autotune; default 2).  Each feeder's result is the one okr_reduce
 * gives for it alone.
 *
 * feeders: [n_feeders] HOST feeders.  params: [n_params] with n_params = 1
 * (shared) or n_feeders; record_iters must be 0.  items: [n_feeders] HOST,
 * written.  super_of (HOST, may be NULL): the assignments, concatenated in
 * feeder order (sum of n_bus entries).  stats (HOST, may be NULL).
 * Returns a non-OK status only for bad arguments or a CUDA failure of the
 * batch; each feeder's own outcome is in items[f].status. */
okr_status okr_reduce_batch(okr_ctx *ctx, int32_t n_feeders, const okr_feeder *feeders, const okr_params *params,
                            int32_t n_params, okr_batch_item *items, int32_t *super_of, okr_batch_stats *stats);

/* Times the batched search with each team shape on this batch (two runs
 * each), keeps the fastest for later okr_reduce_batch calls on this context,
 * and returns it in *config (search_ms: [4] times in ms, may be NULL). */
okr_status okr_batch_autotune(okr_ctx *ctx, int32_t n_feeders, const okr_feeder *feeders, const okr_params *params,
                              int32_t n_params, int32_t *config, double *search_ms);

/* ---- a batch reduced again and again: one CUDA graph --------------------
 * okr_batch_plan_create checks and stages a batch (the feeders are copied into
 * the plan's pinned host block), allocates the plan's own device memory and
 * captures the whole device sequence of one okr_reduce_batch -- input copy,
 * setup launches, search launch(es), result copies -- as one CUDA graph on the
 * context's stream.  okr_batch_plan_run replays it with one graph launch and
 * returns what okr_reduce_batch returns for the same batch (items, super_of,
 * stats; each pointer as there).  okr_batch_plan_set_loads replaces feeder f's
 * s_load (HOST, [n_scen][n_bus][3][2]) for the following runs, e.g. another
 * loading scenario of the same feeders.  The plan uses the context's stream and
 * the team shape current at creation; it must be destroyed before its context.
 * Errors as okr_reduce_batch; OKR_ECUDA when the capture fails. */
typedef struct okr_batch_plan okr_batch_plan;
okr_status okr_batch_plan_create(okr_ctx *ctx, int32_t n_feeders, const okr_feeder *feeders, const okr_params *params,
                                 int32_t n_params, okr_batch_plan **plan);
okr_status okr_batch_plan_run(okr_batch_plan *plan, okr_batch_item *items, int32_t *super_of,
                              okr_batch_stats *stats);
okr_status okr_batch_plan_set_loads(okr_batch_plan *plan, int32_t feeder, const double *s_load);
void okr_batch_plan_destroy(okr_batch_plan *plan);

/* Sets the team shape of later okr_reduce_batch calls on this context
 * (0/1/2/3 = 1/2/4/8 CTAs per feeder); OKR_EINVAL outside that range. */
okr_status okr_set_batch_config(okr_ctx *ctx, int32_t config);

/* Three-phase radialization (Sec. V): the critical buses that make the
 * Kron-reduced network radial.  For every maximal clique of Y_Kron's bus
 * graph (one per connected component of reduced buses and its boundary),
 * the reduced buses of degree >= 3 in the sub-tree spanning the clique.  The
 * radial network keeps kept + critical buses (okr_kron with that set gives
 * its Y_Kron); with no injection moved to the critical buses, the super-node
 * voltages are those of the unradialized network.
 *
 * kept: HOST [n_bus] flags (bus 0 kept) or NULL for the last reduction's
 * super-nodes.  critical: HOST [n_bus] flags, written (caller numbering).
 * *n_critical (may be NULL): their number.  Errors as okr_kron. */
okr_status okr_radialize(okr_ctx *ctx, const uint8_t *kept, uint8_t *critical, int32_t *n_critical);

/* ---- learned candidate scorer -----------------------------------------
 * A small network (three hidden layers of 128 ReLU units; weights kept in
 * FP32, used as bfloat16 in every product with FP32 accumulation) that
 * predicts a candidate's score change from local features.  It is trained on
 * the scores the exhaustive search itself produces (record_iters, precision 0)
 * and is used to rank candidates; the exhaustive search remains the reference
 * that measures how often the ranking misses the optimum.  It is an addition
 * to the method, which has no learned part.
 *
 * Features of candidate (s, r), OKR_SCORER_FEATURES floats: log10 of the path
 * impedance between r and the common ancestor a, same for s; log10 of the
 * injections of r and of s (sum over scenarios and phases of |re| + |im|);
 * phase counts of r and s / 3; current MICE of r and of s / margin; direction
 * (1: the cluster above joins the one below); log10(1 + affected clusters);
 * voltage spread (max hi - lo) of r and of s / margin; the merged cluster's
 * error at s's present voltage magnitude / margin, and that error less the
 * MICE of r and s / margin. */
#define OKR_SCORER_FEATURES 14

/* Features of every candidate of recorded iteration `iter` of the last
 * reduction (same order as okr_get_recorded).  features: HOST
 * [cap][OKR_SCORER_FEATURES] floats, caller-owned, written for the first
 * min(cap, count) candidates; NULL with cap = 0 queries *count alone. */
okr_status okr_get_recorded_features(const okr_ctx *ctx, int32_t iter, int32_t cap, float *features,
                                     int32_t *count);

/* (Re)creates the scorer for n_features (1..16) inputs with parameters theta
 * (HOST, okr_scorer_params order; NULL = zeros) and clears the Adam state.
 * Parameter order: W1 (n_features x 128, row-major), b1 (128), W2 (128 x 128),
 * b2, W3 (128 x 128), b3, w4 (128), b4 (1). */
okr_status okr_scorer_init(okr_ctx *ctx, int32_t n_features, const float *theta);
/* Current parameters (theta may be NULL to query *n_params). */
okr_status okr_scorer_params(okr_ctx *ctx, float *theta, int32_t *n_params);
/* Gradient of the mean squared error (1/n) sum (y_i - t_i)^2 at the current
 * parameters over n samples x (HOST [n][n_features]), t (HOST [n]); grad:
 * HOST [n_params] (may be NULL); *loss (may be NULL). */
okr_status okr_scorer_gradient(okr_ctx *ctx, const float *x, const float *t, int32_t n, float *grad, double *loss);
/* Adam (lr, beta 0.9 / 0.999) over `epochs` passes of consecutive minibatches
 * of `batch` samples (the caller shuffles); epoch_loss: HOST [epochs], the
 * mean squared error over each pass (may be NULL). */
okr_status okr_scorer_train(okr_ctx *ctx, const float *x, const float *t, int64_t n, int32_t batch, int32_t epochs,
                            float lr, double *epoch_loss);
/* Predictions y (HOST [n]) for x (HOST [n][n_features]). */
okr_status okr_scorer_predict(okr_ctx *ctx, const float *x, int64_t n, float *y);
/* The same network on the tensor cores (tcgen05, 128 samples per product):
 * the features and the hidden activations enter each product as bfloat16
 * (both operands of a bfloat16 tensor-core product are bfloat16), products and
 * sums are FP32.  For ranking many candidates; training keeps FP32 activations
 * (okr_scorer_predict).  OKR_ETIMEOUT if a wait for the products gave up. */
okr_status okr_scorer_predict_tc(okr_ctx *ctx, const float *x, int64_t n, float *y);

/* The reduced network of a given assignment, evaluated on the feeder's own
 * scenarios (HOST feeder; its load flows are solved first): super-nodes take
 * the aggregated injections of their members, the network is solved with the
 * slack fixed, every bus takes its super-node's voltage (Algorithm 1's
 * voltage model), and max_error[l] (HOST [n_scen]) receives the largest
 * per-phase magnitude error against the full network.  Used to test a
 * reduction on operating points other than the ones it was built from.
 * super_of: HOST [n_bus] caller ids; every super_of[i] must be a super-node
 * (super_of[super_of[i]] == super_of[i]) and super_of[0] == 0.
 * vred (HOST [n_scen][n_bus][3][2], may be NULL): the reduced voltages.
 * Invalidates the last reduction's results. */
okr_status okr_evaluate(okr_ctx *ctx, const okr_feeder *f, const int32_t *super_of, double *max_error, double *vred);

/* Largest feeder okr_power_flow_static accepts (buses; scenarios up to 4). */
#define OKR_STATIC_MAX_BUS 4096

/* The load flow of okr_power_flow for callers that cannot allocate device
 * memory: code inside a host framework whose allocator owns the GPU's memory
 * (a cudaMalloc there fails or escapes its accounting), and loops that cannot
 * take the device-wide synchronisation of cudaMalloc/cudaFree.  The paper has
 * no counterpart: this is an interface variant, not a step of the method.
 *
 * Needs no context and allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine.  Its scratch is one static device array of
 * 5,396,480 bytes (sized for OKR_STATIC_MAX_BUS buses and 4 scenarios) that
 * every GPU which loads the library holds until the process exits.  Runs on the CURRENT device and on `stream` (a cudaStream_t,
 * NULL = the default stream); returns after the stream has finished the work.
 *
 * f: feeder arrays (parent, phases, z_line, s_load) in DEVICE memory of the
 * current device, caller-owned, read only; v_slack is read from *f.
 * vhat_out (required), ihat_out (may be NULL): DEVICE buffers
 * [n_scen][n_bus][3][2], caller-owned, written (0 on absent phases);
 * *sweeps (HOST, may be NULL): sweeps of the slowest scenario.
 * Errors: OKR_EINVAL for NULL arrays, n_bus outside [2, OKR_STATIC_MAX_BUS],
 * n_scen outside [1, 4] or an invalid tree; OKR_ESINGULAR, OKR_EPF as
 * okr_power_flow; OKR_ECUDA for a CUDA failure.  No message string is kept.
 *
 * The first call on a device also looks up the device address of the static
 * array (once per device, with that device current): make that first call
 * before any stream capture.  Every call shares the one array, which keeps
 * the previous call's contents; calls that overlap on the GPU (other streams,
 * other host threads on the same device) race on it and must be serialised
 * by the caller. */
okr_status okr_power_flow_static(const okr_feeder *f, double *vhat_out, double *ihat_out,
                                 int32_t *sweeps, void *stream);

/* ---- results as library-owned objects ----------------------------------
 * The problem statement's outputs (Sec. III-IV: the kept set and clusters,
 * the reduced network's voltages and errors; Sec. II-B: Y_Kron) of one
 * reduction, copied out of the context so that later calls on the context
 * do not touch them.  The object holds host memory only and is owned by the
 * library until okr_result_free; its getters copy into caller buffers and
 * never fail on a valid object.  Any output pointer may be NULL; a call with
 * every array pointer NULL returns the sizes alone. */
typedef struct okr_result okr_result;

/* Takes the results of the context's last okr_reduce / okr_reduce_device /
 * okr_reduce_ops: the summary, the decision sequence, the assignment, the
 * voltages of the full and of the reduced network and, with with_ykron = 1,
 * Y_Kron of the chosen network (computed on the device as by okr_kron).
 * Errors: OKR_ENOTREADY without a reduction; OKR_ENOMEM; okr_kron's errors
 * with with_ykron. */
okr_status okr_result_take(okr_ctx *ctx, int32_t with_ykron, okr_result **out);
void okr_result_free(okr_result *res);
okr_status okr_result_summary(const okr_result *res, okr_summary *out);
/* super_of: [n_bus] caller ids of each bus's super-node; *n_bus, *n_kept. */
okr_status okr_result_assignment(const okr_result *res, int32_t *super_of, int32_t *n_bus, int32_t *n_kept);
/* The decision sequence as okr_get_decisions; *count = merges (the first
 * min(cap, count) entries are written). */
okr_status okr_result_decisions(const okr_result *res, int32_t cap, int32_t *s, int32_t *r, double *smice,
                                double *max_error, double *gap, int32_t *ncand, int32_t *count);
/* Largest per-phase error and SMICE of the chosen network; vhat, vred:
 * [n_scen][n_bus][3][2] voltages of the full and the reduced network. */
okr_status okr_result_errors(const okr_result *res, double *max_error, double *smice, double *vhat, double *vred,
                             int32_t *n_scen, int32_t *n_bus);
/* Y_Kron of the chosen network as okr_kron writes it (y: [k_phi][k_phi][2],
 * phase_node: [k_phi]; cap >= k_phi when either is given, else OKR_EINVAL);
 * OKR_ENOTREADY when the result was taken without it. */
okr_status okr_result_ykron(const okr_result *res, int32_t cap, double *y, int32_t *phase_node, int32_t *k_phi);
/* Candidates evaluated, merges committed, seconds of the search kernel. */
okr_status okr_result_stats(const okr_result *res, int64_t *candidates, int32_t *iterations, double *seconds);

/* ---- results of the last reduction (host buffers, caller-owned) ---- */
okr_status okr_get_summary(const okr_ctx *ctx, okr_summary *out);
/* Decision sequence, one entry per merge, in caller bus ids: s (absorbing
 * super-node), r (absorbed), the objective after the merge (SMICE, or the
 * largest error with objective 1), largest error after the merge, distance
 * of the next score above the tie band, candidates evaluated.
 * cap = buffer length; any pointer may be NULL. */
okr_status okr_get_decisions(const okr_ctx *ctx, int32_t cap, int32_t *s, int32_t *r, double *smice,
                             double *max_error, double *gap, int32_t *ncand);
/* super_of[n_bus]: the super-node (caller id) each bus is assigned to. */
okr_status okr_get_assignment(const okr_ctx *ctx, int32_t *super_of);
/* vhat, vred: [n_scen][n_bus][3][2]; vred[i] is the reduced-network voltage of
 * bus i (its super-node's).  Either pointer may be NULL. */
okr_status okr_get_voltages(const okr_ctx *ctx, double *vhat, double *vred);
/* Scores of every candidate of iteration `iter` < record_iters (SMICE the
 * candidate would give; +inf if it breaks the margin), in no particular order.
 * With precision 1 these are the FP32 screen values and bound[i] bounds their
 * distance to the FP64 values (0 with precision 0).  cap = buffer length
 * (2*n_bus suffices); *count = candidates of that iteration.  s, r, smice,
 * bound may be NULL. */
okr_status okr_get_recorded(const okr_ctx *ctx, int32_t iter, int32_t cap, int32_t *s, int32_t *r,
                            double *smice, double *bound, int32_t *count);

#ifdef __cplusplus
}
#endif

#endif /* OKRON_H */
