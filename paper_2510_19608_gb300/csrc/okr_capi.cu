// okr_capi.cu -- the C ABI declared in include/okron.h: context, device
// workspace, and the host orchestration of the per-feeder setup kernels and the
// persistent search kernel (one cooperative launch per reduction).
#include "okron.h"
#include "okr_internal.cuh"
#include "okr_kernels.cuh"
#include "okr_layout.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

using namespace okr;

namespace {

constexpr long long kDefaultSpins = 1000000;   // bounded device waits: one L2 round trip per poll, under a second
constexpr double kPfTol = 1e-13;
constexpr int kPfMaxIter = 200;

}  // namespace

struct okr_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;

    // capacity of the workspace
    int cap_n = 0, cap_L = 0, cap_rec = 0;

    FeederBufs fb;                      // device buffers of the current feeder (one allocation)
    void *arena = nullptr;
    int grid = 0;                       // CTAs of the persistent search kernel
    std::vector<void *> work_allocs;    // chunk map and partial sums (grown on demand)
    int cap_chunks = 0;
    int sum_sz = 0, max_depth = 0;      // of the current feeder
    Ctrl *C_host = nullptr;             // pinned
    // the setup steps the load flow does not need (LCA table, path impedances)
    // run on a second stream beside it; ev_side marks their end
    cudaStream_t side = nullptr;
    cudaEvent_t ev_topo = nullptr, ev_lines = nullptr, ev_side = nullptr;
    bool side_pending = false;          // the stream has not waited for ev_side yet

    // counters of the last call
    int64_t launches = 0;
    double search_ms = 0.0;
    int last_engine = 0;                // OKR_ENGINE_SWEEP or OKR_ENGINE_INCREMENTAL

    // Y_Kron work (allocated on the first okr_kron call)
    KronWork kw{};
    int cap_kron_n = 0;
    std::vector<void *> kron_allocs;
    double2 *ykr = nullptr, *kbig = nullptr;
    uint8_t *kron_kept = nullptr, *kron_crit = nullptr;
    int *kron_count = nullptr;
    size_t cap_ykr = 0, cap_kbig = 0;
    double kron_ms = 0.0;

    // multi-feeder batch (grown on demand)
    void *batch_arena = nullptr;
    size_t batch_cap = 0;
    unsigned char *batch_host = nullptr;    // pinned staging
    size_t batch_host_cap = 0;
    int batch_config = 1;                   // team shape of the batched search: 2 CTAs per feeder (autotuned)
    IncShape inc_shape{0, 0, 0, -1};        // launch shape of the incremental search (resolved at launch)
    IncShape last_shape{0, 0, 0, -1};       // shape of the last incremental search, resolved
    int last_rec = -1;                      // its record placement (-1: the sweep engine ran)

    // learned scorer
    MlpBufs mb;
    MlpWork mw;
    std::vector<void *> mlp_allocs, mlp_work_allocs, mlp_data_allocs;
    float *mlp_x = nullptr, *mlp_t = nullptr;    // device copies of a data set
    int *mlp_err = nullptr;                      // error flag of the tensor-core inference
    long long mlp_data_cap = 0;
    int mlp_step = 0;

    // device allocator (cudaMalloc / cudaFree unless the caller registered one)
    okr_alloc_fn alloc_fn = nullptr;
    okr_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    long long live_allocs = 0;  // device blocks currently held

    // last result
    bool have_topo = false;     // T describes the feeder of the last call
    bool have_result = false;
    int n = 0, L = 0, rec_iters = 0, pf_sweeps = 0;
    Ctrl last{};
};

namespace {

// Every device allocation of a context: the registered allocator, else
// cudaMalloc.  Returns cudaErrorMemoryAllocation when it fails.
cudaError_t dev_alloc(okr_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 1;
    if (ctx->alloc_fn) {
        *p = ctx->alloc_fn(ctx->alloc_user, bytes, ctx->device, (void *)ctx->stream);
        if (!*p) return cudaErrorMemoryAllocation;
    } else {
        const cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) { *p = nullptr; return e; }
    }
    ctx->live_allocs += 1;
    return cudaSuccess;
}

// Frees a block of dev_alloc (NULL is ignored).  The work that used it on
// the context's stream has finished: every entry point returns after its work.
void dev_free(okr_ctx *ctx, void *p) {
    if (!p) return;
    if (ctx->free_fn) ctx->free_fn(ctx->alloc_user, p, ctx->device, (void *)ctx->stream);
    else cudaFree(p);
    ctx->live_allocs -= 1;
}

}  // namespace

namespace {

okr_status fail(okr_ctx *c, okr_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? OKR_ENOMEM : OKR_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
    } while (0)

void free_kron(okr_ctx *ctx) {
    for (void *p : ctx->kron_allocs) dev_free(ctx, p);
    ctx->kron_allocs.clear();
    ctx->cap_kron_n = 0;
    dev_free(ctx, ctx->ykr);
    dev_free(ctx, ctx->kbig);
    ctx->ykr = ctx->kbig = nullptr;
    ctx->cap_ykr = ctx->cap_kbig = 0;
}

void free_batch(okr_ctx *ctx) {
    dev_free(ctx, ctx->batch_arena);
    ctx->batch_arena = nullptr;
    ctx->batch_cap = 0;
    if (ctx->batch_host) cudaFreeHost(ctx->batch_host);
    ctx->batch_host = nullptr;
    ctx->batch_host_cap = 0;
}

void free_list(okr_ctx *ctx, std::vector<void *> &v) {
    for (void *p : v) dev_free(ctx, p);
    v.clear();
}

void free_mlp(okr_ctx *ctx) {
    free_list(ctx, ctx->mlp_allocs);
    free_list(ctx, ctx->mlp_work_allocs);
    free_list(ctx, ctx->mlp_data_allocs);
    ctx->mb = MlpBufs{};
    ctx->mw = MlpWork{};
    ctx->mlp_data_cap = 0;
    ctx->mlp_x = ctx->mlp_t = nullptr;
    dev_free(ctx, ctx->mlp_err);
    ctx->mlp_err = nullptr;
}

void free_all(okr_ctx *ctx) {
    free_kron(ctx);
    dev_free(ctx, ctx->arena);
    ctx->arena = nullptr;
    for (void *p : ctx->work_allocs) dev_free(ctx, p);
    ctx->work_allocs.clear();
    ctx->cap_chunks = 0;
    ctx->cap_n = ctx->cap_L = ctx->cap_rec = 0;
}

int log2_ceil(int n) {
    int j = 0;
    while ((1 << j) < n) ++j;
    return j;
}



okr_status ensure_workspace(okr_ctx *ctx, int n, int L, int rec) {
    if (n <= ctx->cap_n && L <= ctx->cap_L && rec <= ctx->cap_rec) return OKR_OK;
    free_all(ctx);
    Carver m;
    FeederBufs f;
    layout_feeder(m, n, L, rec, ctx->num_sms, 0, f);
    void *p = nullptr;
    CK(dev_alloc(ctx, &p, m.used));
    ctx->arena = p;
    Carver c;
    c.base = static_cast<unsigned char *>(p);
    layout_feeder(c, n, L, rec, ctx->num_sms, 0, ctx->fb);
    ctx->cap_n = n;
    ctx->cap_L = L;
    ctx->cap_rec = rec;
    return OKR_OK;
}

}  // namespace

namespace {

int blocks_for(size_t work, int threads, int cap) {
    size_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (size_t)cap) b = cap;
    return (int)b;
}

okr_status check_feeder_shape(okr_ctx *ctx, const okr_feeder *f) {
    if (!f) return fail(ctx, OKR_EINVAL, "feeder is NULL");
    if (f->n_bus < 2 || f->n_bus > kMaxBus) return fail(ctx, OKR_EINVAL, "n_bus=%d outside [2, %d]", f->n_bus, kMaxBus);
    if (f->n_scen < 1 || f->n_scen > kMaxScen) return fail(ctx, OKR_EINVAL, "n_scen=%d outside [1, %d]", f->n_scen, kMaxScen);
    if (!f->parent || !f->phases || !f->z_line) return fail(ctx, OKR_EINVAL, "feeder array is NULL");
    return OKR_OK;
}

okr_status check_params(okr_ctx *ctx, const okr_params *p) {
    if (!p) return fail(ctx, OKR_EINVAL, "params is NULL");
    if (!(p->margin > 0.0) || !std::isfinite(p->margin)) return fail(ctx, OKR_EINVAL, "margin must be positive");
    if (!(p->tie_tol >= 0.0) || !std::isfinite(p->tie_tol)) return fail(ctx, OKR_EINVAL, "tie_tol must be >= 0");
    if (p->max_merges < 0 && !(p->target_reduction >= 0.0 && p->target_reduction <= 1.0))
        return fail(ctx, OKR_EINVAL, "target_reduction outside [0, 1]");
    if (p->objective != 0 && p->objective != 1) return fail(ctx, OKR_EINVAL, "objective %d not supported", p->objective);
    if (p->precision != 0 && p->precision != 1) return fail(ctx, OKR_EINVAL, "precision %d not supported", p->precision);
    if (p->record_iters < 0) return fail(ctx, OKR_EINVAL, "record_iters < 0");
    if (p->scorer_topk < 0) return fail(ctx, OKR_EINVAL, "scorer_topk < 0");
    if (p->scorer_topk > 0 && (!ctx || ctx->mb.F != kScorerFeatures))
        return fail(ctx, OKR_EINVAL, "scorer_topk needs a scorer with %d features (okr_scorer_init)", kScorerFeatures);
    if (p->engine < OKR_ENGINE_AUTO || p->engine > OKR_ENGINE_VERIFY)
        return fail(ctx, OKR_EINVAL, "engine %d not supported", p->engine);
    if (p->engine >= OKR_ENGINE_INCREMENTAL && (p->objective != 0 || p->scorer_topk != 0))
        return fail(ctx, OKR_EINVAL, "the incremental engine needs objective 0 and scorer_topk 0");
    if (p->prune_exact != 0 && p->prune_exact != 1) return fail(ctx, OKR_EINVAL, "prune_exact must be 0 or 1");
    if (p->prune_exact && (p->scorer_topk <= 0 || p->objective != 0 || p->precision != 0 ||
                           p->engine >= OKR_ENGINE_INCREMENTAL))
        return fail(ctx, OKR_EINVAL, "prune_exact needs scorer_topk > 0, objective 0, precision 0 and the sweep engine");
    return OKR_OK;
}

// The engine a valid parameter set runs: OKR_ENGINE_SWEEP or OKR_ENGINE_INCREMENTAL.
int resolve_engine(const okr_params *p) {
    if (p->engine == OKR_ENGINE_SWEEP) return OKR_ENGINE_SWEEP;
    if (p->engine >= OKR_ENGINE_INCREMENTAL) return OKR_ENGINE_INCREMENTAL;
    return (p->objective == 0 && p->scorer_topk == 0) ? OKR_ENGINE_INCREMENTAL : OKR_ENGINE_SWEEP;
}

// False when the automatic engine would pick the incremental one for an
// n-bus feeder whose per-merge data does not fit one SM's shared memory
// (about 13,900 buses): that feeder runs on the sweep instead.
bool inc_fits(const okr_ctx *ctx, int n, const okr_params *p) {
    if (p->engine != OKR_ENGINE_AUTO || resolve_engine(p) != OKR_ENGINE_INCREMENTAL) return true;
    IncShape sh = inc_shape_resolve(ctx->inc_shape);
    sh.rec = -1;
    int rec = 0;
    size_t bytes = 0;
    return inc_smem(n, true, sh, &rec, &bytes);
}

// The engine a reduction of an n-bus feeder runs.
int run_engine(const okr_ctx *ctx, int n, const okr_params *p) {
    return inc_fits(ctx, n, p) ? resolve_engine(p) : OKR_ENGINE_SWEEP;
}

int merges_for(int n, const okr_params *p) {
    long m;
    if (p->max_merges >= 0) m = p->max_merges;
    else m = (long)std::ceil(p->target_reduction * n - 1e-12);
    if (m > n - 1) m = n - 1;
    if (m < 0) m = 0;
    return (int)m;
}

okr_status read_setup_errors(okr_ctx *ctx);

// The stream waits for the setup steps on the side stream (a no-op when it already has).
cudaError_t join_side(okr_ctx *ctx) {
    if (!ctx->side_pending) return cudaSuccess;
    ctx->side_pending = false;
    return cudaStreamWaitEvent(ctx->stream, ctx->ev_side, 0);
}

// Pinned host staging: the search's Ctrl, then the setup's error flag and the
// load flow's sweep count per scenario (read together after the last launch).
constexpr size_t kHostStageBytes = sizeof(Ctrl) + 16 + sizeof(int) * (1 + kMaxScen);
int *host_err(okr_ctx *ctx) { return reinterpret_cast<int *>(reinterpret_cast<char *>(ctx->C_host) + sizeof(Ctrl) + 16); }
int *host_pf_iters(okr_ctx *ctx) { return host_err(ctx) + 1; }

// Per-feeder setup on the device: topology, LCA table, lines, path impedances.
// The host waits for the topology's check of the tree (the later kernels index
// through its renumbering); with check_lines it also waits for the lines and
// reads the tree's statistics, else a singular line is reported with the
// caller's last read of the error flag (the load flow skips its work then).
okr_status build_topology(okr_ctx *ctx, int n, int L, const double *vslack, bool check_lines = true) {
    cudaStream_t st = ctx->stream;
    CK(join_side(ctx));                     // (a failed call may have left side work unjoined)
    Topo &T = ctx->fb.T;
    T.n = n;
    T.L = L;
    double2 vs[3];
    for (int p = 0; p < 3; ++p) vs[p] = make_double2(vslack[2 * p], vslack[2 * p + 1]);
    CK(cudaMemcpyAsync(T.vslack, vs, sizeof vs, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(ctx->fb.err_dev, 0, sizeof(int), st));
    k_topology<<<1, 1024, 0, st>>>(n, ctx->fb.parent_in, ctx->fb.ph_in, T, ctx->fb.dep, ctx->fb.anc, ctx->fb.anc2, ctx->fb.d2,
                                   ctx->fb.size, ctx->fb.ccount, ctx->fb.coff_c, ctx->fb.child_c, ctx->fb.err_dev);
    ctx->launches += 1;
    CK(cudaGetLastError());
    // the later setup kernels index with the renumbering: stop here on an invalid tree
    okr_status s = read_setup_errors(ctx);
    if (s != OKR_OK) return s;
    // the LCA table and the path impedances (on the side stream) are not read
    // by the load flow: they run beside it, and the stream waits for them
    // before the search (join_side)
    cudaStream_t sd = ctx->side;
    CK(cudaEventRecord(ctx->ev_topo, st));
    CK(cudaStreamWaitEvent(sd, ctx->ev_topo, 0));
    k_child_offsets<<<1, 1024, 0, st>>>(n, T, ctx->fb.coff_c, ctx->fb.child_c);
    const int LOG = log2_ceil(n) + 1;
    k_rmq_all<<<1, 1024, 0, sd>>>(n, LOG, T.depth, ctx->fb.rmq);
    k_lca_fill<<<blocks_for((size_t)n * n, 256, ctx->num_sms * 8), 256, 0, sd>>>(n, T.parent, T.sz, T.depth, ctx->fb.rmq, T.lca);
    CK(launch_line_inverses(n, T, ctx->fb.z_in, ctx->fb.err_dev, ctx->num_sms, st));
    CK(cudaEventRecord(ctx->ev_lines, st));
    CK(cudaStreamWaitEvent(sd, ctx->ev_lines, 0));
    CK(launch_path_impedance(n, T, sd));
    CK(cudaEventRecord(ctx->ev_side, sd));
    ctx->side_pending = true;
    ctx->launches += 5;
    CK(cudaGetLastError());
    if (!check_lines) {
        ctx->have_topo = true;
        return OKR_OK;
    }
    CK(join_side(ctx));
    s = read_setup_errors(ctx);
    if (s != OKR_OK) return s;
    int stats[2] = {0, 0};
    CK(cudaMemcpy(stats, T.maxd, sizeof stats, cudaMemcpyDeviceToHost));
    ctx->max_depth = stats[0];
    ctx->sum_sz = stats[1];
    ctx->have_topo = true;
    return OKR_OK;
}

okr_status setup_status(okr_ctx *ctx, int e);

okr_status read_setup_errors(okr_ctx *ctx) {
    CK(cudaMemcpyAsync(host_err(ctx), ctx->fb.err_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return setup_status(ctx, *host_err(ctx));
}

// The status of a setup error code (0: none).
okr_status setup_status(okr_ctx *ctx, int e) {
    if (e == 1) return fail(ctx, OKR_EINVAL, "invalid feeder: parent[0] must be -1, parent[i] < i, phases non-empty and within the parent's");
    if (e == 2) return fail(ctx, OKR_ESINGULAR, "singular line impedance block");
    if (e == 3) return fail(ctx, OKR_EPF, "load flow did not converge in %d sweeps", kPfMaxIter);
    if (e == 6) return fail(ctx, OKR_ETIMEOUT, "a grid barrier of the load flow gave up");
    if (e) return fail(ctx, OKR_EINTERNAL, "device error %d", e);
    return OKR_OK;
}

// max_spins: polls per grid barrier of the load flow (params.max_spins; 0 = default).
okr_status run_power_flow(okr_ctx *ctx, int n, int L, long long max_spins = 0) {
    cudaStream_t st = ctx->stream;
    Topo &T = ctx->fb.T;
    // the load flow's work buffers alias T.ihat and T.amag, which the next two kernels fill
    CK(launch_power_flow(n, L, T, ctx->fb.s_in, kPfTol, kPfMaxIter, ctx->fb.J, T.ihat, T.amag, ctx->fb.pf_iters,
                         ctx->fb.err_dev, ctx->num_sms, st, max_spins > 0 ? max_spins : kDefaultSpins));
    k_line_currents<<<blocks_for((size_t)L * n, 256, ctx->num_sms * 8), 256, 0, st>>>(n, L, T, ctx->fb.J);
    k_injections<<<blocks_for((size_t)L * n, 256, ctx->num_sms * 8), 256, 0, st>>>(n, L, T, ctx->fb.J);
    ctx->launches += 3;
    CK(cudaGetLastError());
    return OKR_OK;
}

// Chunk map and partial sums for up to `chunks` chunks of one sweep.
okr_status ensure_work(okr_ctx *ctx, long long chunks) {
    if (chunks <= ctx->cap_chunks) return OKR_OK;
    if (chunks > (long long)INT32_MAX / 2) return fail(ctx, OKR_EINVAL, "feeder too large for the search buffers");
    for (void *p : ctx->work_allocs) dev_free(ctx, p);
    ctx->work_allocs.clear();
    ctx->cap_chunks = 0;
    void *a = nullptr, *b = nullptr;
    cudaError_t e = dev_alloc(ctx, &a, sizeof(int) * (size_t)chunks);
    if (e == cudaSuccess) e = dev_alloc(ctx, &b, sizeof(double2) * ((size_t)chunks + 2 * (size_t)ctx->cap_n));
    if (e != cudaSuccess) {
        dev_free(ctx, a);
        return fail(ctx, OKR_ENOMEM, "search buffers: %s", cudaGetErrorString(e));
    }
    ctx->work_allocs.push_back(a);
    ctx->work_allocs.push_back(b);
    ctx->fb.X.chunk_first = (int *)a;
    ctx->fb.X.partial = (double2 *)b;
    ctx->fb.X.max_chunks = (int)chunks;
    ctx->cap_chunks = (int)chunks;
    return OKR_OK;
}

int positions_per_chunk(int L) { return 32 / (4 * (L <= 1 ? 1 : (L <= 2 ? 2 : 4))); }

// Initial state, then the persistent search kernel.  The kernel stops by itself
// (target reached or nothing feasible); if one sweep needs more work buffer than
// allocated it saves its state and exits, and is relaunched with a larger one.
okr_status run_search_inc(okr_ctx *ctx, const okr_params *p);

okr_status run_search(okr_ctx *ctx, const okr_params *p) {
    ctx->last_engine = run_engine(ctx, ctx->fb.T.n, p);
    ctx->last_rec = -1;
    if (ctx->last_engine == OKR_ENGINE_INCREMENTAL) return run_search_inc(ctx, p);
    cudaStream_t st = ctx->stream;
    const int n = ctx->fb.T.n, L = ctx->fb.T.L;
    Search &X = ctx->fb.X;
    X.rec_iters = p->record_iters;
    X.topk = p->scorer_topk;
    X.prune_exact = p->prune_exact;
    if (X.topk > 0) {
        X.mlp_theta = ctx->mb.theta;
        X.mlp_w1 = reinterpret_cast<const uint16_t *>(ctx->mb.w1);
        X.mlp_w2 = reinterpret_cast<const uint16_t *>(ctx->mb.w2);
        X.mlp_w3 = reinterpret_cast<const uint16_t *>(ctx->mb.w3);
        X.mlp_w4 = reinterpret_cast<const uint16_t *>(ctx->mb.w4);
    }
    k_state_init<<<blocks_for((size_t)L * n, 256, ctx->num_sms * 8), 256, 0, st>>>(n, L, ctx->fb.T, ctx->fb.S);
    ctx->launches += 1;
    CK(cudaGetLastError());
    const int mm = merges_for(n, p);
    Ctrl c{};
    c.max_merges = mm;
    c.done = (mm == 0);
    c.margin = p->margin;
    c.tau = p->tie_tol;
    c.profile = p->profile ? 1 : 0;
    c.n_super = n;
    c.precision = p->precision;
    c.objective = p->objective;
    c.max_spins = p->max_spins > 0 ? p->max_spins : kDefaultSpins;
    CK(cudaMemcpyAsync(ctx->fb.C, &c, sizeof c, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(X.dec_maxerr, 0, sizeof(double) * n, st));
    CK(cudaMemsetAsync(X.arrive, 0, sizeof(int) * 2 * n, st));
    CK(cudaMemsetAsync(X.mrank, 0, sizeof(double) * n, st));           // every MICE starts at 0
    CK(cudaMemsetAsync(X.bmax, 0, sizeof(double) * (n / 32 + 2), st));
    if (p->scorer_topk > 0) {                   // no kept prediction; no super-node changed yet
        CK(cudaMemsetAsync(X.pkey, 0xff, sizeof(unsigned long long) * 2 * n, st));
        CK(cudaMemsetAsync(X.moved, 0xff, sizeof(int) * n, st));
    }
    if (p->prune_exact) {                       // every g_k starts at 0 (singletons: no spread, MICE 0)
        CK(cudaMemsetAsync(X.gpre, 0, sizeof(long long) * n, st));
        CK(cudaMemsetAsync(X.gbp, 0, sizeof(long long) * (n / 32 + 2), st));
        CK(cudaMemsetAsync(X.lbkey, 0xff, sizeof(unsigned long long) * 2 * n, st));
    }
    CK(cudaMemsetAsync(ctx->fb.gb, 0, sizeof(GridBar), st));
    if (p->record_iters > 0) CK(cudaMemsetAsync(X.rec_count, 0, sizeof(int) * p->record_iters, st));
    ctx->rec_iters = p->record_iters;
    ctx->search_ms = 0.0;
    // first sweep: every bus is a super-node; candidate (p -> w) and (w -> p)
    // cover subtree(w) and one extra position, so 2 * sum(sz) + 2 n bounds it
    const int ppc = positions_per_chunk(L);
    long long want = (2LL * ctx->sum_sz + 2LL * n + ppc - 1) / ppc + 1;
    okr_status s = ensure_work(ctx, want);
    if (s != OKR_OK) return s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int attempt = 0; attempt < 16 && !c.done; ++attempt) {
        CK(cudaMemsetAsync(ctx->fb.gb, 0, sizeof(GridBar), st));
        cudaEventRecord(e0, st);
        cudaError_t e = launch_search(p->precision, ctx->grid, ctx->fb.T, ctx->fb.S, ctx->fb.X, ctx->fb.C, ctx->fb.gb, st);
        cudaEventRecord(e1, st);
        ctx->launches += 1;
        if (e != cudaSuccess) { s = fail(ctx, OKR_ECUDA, "search launch: %s", cudaGetErrorString(e)); break; }
        e = cudaMemcpyAsync(ctx->C_host, ctx->fb.C, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = fail(ctx, OKR_ECUDA, "search: %s", cudaGetErrorString(e)); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ctx->search_ms += ms;
        c = *ctx->C_host;
        if (c.err == 7) {                       // grow the work buffers and continue
            want = 2LL * ((c.total_pos + ppc - 1) / ppc + 1);
            s = ensure_work(ctx, want);
            if (s != OKR_OK) break;
            int zero = 0;
            CK(cudaMemcpyAsync(&ctx->fb.C->err, &zero, sizeof zero, cudaMemcpyHostToDevice, st));
            c.done = 0;
            continue;
        }
        break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != OKR_OK) return s;
    if (c.err == 6) return fail(ctx, OKR_ETIMEOUT, "a grid barrier of the search gave up after %lld polls", c.max_spins);
    if (c.err) return fail(ctx, OKR_EINTERNAL, "search device error %d", c.err);
    if (!c.done) return fail(ctx, OKR_EINTERNAL, "search stopped without a result");
    k_export<<<blocks_for((size_t)L * n, 256, ctx->num_sms * 8), 256, 0, st>>>(ctx->fb.T, ctx->fb.S, ctx->fb.vred_out,
                                                                                ctx->fb.super_out, ctx->fb.vhat_out);
    ctx->launches += 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->C_host, ctx->fb.C, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ctx->last = *ctx->C_host;
    return OKR_OK;
}

// Initial state, then one CTA runs the whole search with carried scores
// (okr_incr.cu); then the export.
okr_status run_search_inc(okr_ctx *ctx, const okr_params *p) {
    cudaStream_t st = ctx->stream;
    const int n = ctx->fb.T.n, L = ctx->fb.T.L;
    Search &X = ctx->fb.X;
    X.setup_err = ctx->fb.err_dev;          // a failed setup step leaves the search idle
    X.rec_iters = p->record_iters;
    X.topk = 0;
    X.prune_exact = 0;
    k_state_init<<<blocks_for((size_t)L * n, 256, ctx->num_sms * 8), 256, 0, st>>>(n, L, ctx->fb.T, ctx->fb.S);
    ctx->launches += 1;
    CK(cudaGetLastError());
    const int mm = merges_for(n, p);
    Ctrl c{};
    c.max_merges = mm;
    c.done = (mm == 0);
    c.margin = p->margin;
    c.tau = p->tie_tol;
    c.profile = p->profile ? 1 : 0;
    c.n_super = n;
    c.precision = p->precision;
    c.objective = 0;
    c.max_spins = p->max_spins > 0 ? p->max_spins : kDefaultSpins;
    CK(cudaMemcpyAsync(ctx->fb.C, &c, sizeof c, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(X.dec_maxerr, 0, sizeof(double) * n, st));
    if (p->record_iters > 0) {
        CK(cudaMemsetAsync(X.rec_count, 0, sizeof(int) * p->record_iters, st));
        CK(cudaMemsetAsync(X.rec_feat, 0, sizeof(float) * (size_t)p->record_iters * 2 * n * kScorerFeatures, st));
    }
    ctx->rec_iters = p->record_iters;
    ctx->search_ms = 0.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const IncShape sh = inc_shape_resolve(ctx->inc_shape);
    int rec_used = -1;
    {
        size_t bytes = 0;
        if (!inc_smem(n, true, sh, &rec_used, &bytes))
            return fail(ctx, OKR_EINVAL, "incremental search: the forced record placement does not fit shared memory "
                                         "for %d buses", n);
    }
    ctx->last_shape = sh;
    ctx->last_rec = rec_used;
    cudaEventRecord(e0, st);
    cudaError_t e = launch_search_inc(p->precision, ctx->fb.T, ctx->fb.S, X, ctx->fb.I, ctx->fb.C,
                                      p->engine == OKR_ENGINE_VERIFY ? 1 : 0, sh, &rec_used, st);
    cudaEventRecord(e1, st);
    ctx->launches += 2;                     // the first evaluation on many CTAs, the search on one
    okr_status s = OKR_OK;
    if (e != cudaSuccess) s = fail(ctx, OKR_ECUDA, "search launch: %s", cudaGetErrorString(e));
    if (s == OKR_OK) {
        // the export needs no check first (a failed search leaves valid indices);
        // then one wait for everything: the search's control block, the setup's
        // error flag and the load flow's sweep counts
        k_export<<<blocks_for((size_t)L * n, 256, ctx->num_sms * 8), 256, 0, st>>>(ctx->fb.T, ctx->fb.S, ctx->fb.vred_out,
                                                                                    ctx->fb.super_out, ctx->fb.vhat_out);
        ctx->launches += 1;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->C_host, ctx->fb.C, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host_err(ctx), ctx->fb.err_dev, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_pf_iters(ctx), ctx->fb.pf_iters, sizeof(int) * L, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = fail(ctx, OKR_ECUDA, "search: %s", cudaGetErrorString(e));
    }
    if (s == OKR_OK) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ctx->search_ms = ms;
        c = *ctx->C_host;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    X.setup_err = nullptr;
    if (s != OKR_OK) return s;
    s = setup_status(ctx, *host_err(ctx));
    if (s != OKR_OK) {
        ctx->have_topo = false;
        return s;
    }
    if (ctx->pf_sweeps < 0) {               // the load flow ran in this call: its sweeps, read with the rest
        int w = 0;
        for (int l = 0; l < L; ++l) w = host_pf_iters(ctx)[l] > w ? host_pf_iters(ctx)[l] : w;
        ctx->pf_sweeps = w;
    }
    if (c.err) return fail(ctx, OKR_EINTERNAL, "search device error %d", c.err);
    if (!c.done) return fail(ctx, OKR_EINTERNAL, "search stopped without a result");
    ctx->last = c;
    return OKR_OK;
}

enum class Src { Host, Device, Ops };

okr_status reduce_impl(okr_ctx *ctx, const okr_feeder *f, const double *vhat, const double *ihat,
                       const okr_params *p, Src src) {
    if (!ctx) return OKR_EINVAL;
    ctx->have_result = false;
    ctx->have_topo = false;
    ctx->launches = 0;
    ctx->kron_ms = 0.0;
    okr_status s = check_feeder_shape(ctx, f);
    if (s != OKR_OK) return s;
    s = check_params(ctx, p);
    if (s != OKR_OK) return s;
    if (src != Src::Ops && !f->s_load) return fail(ctx, OKR_EINVAL, "s_load is NULL");
    if (src == Src::Ops && (!vhat || !ihat)) return fail(ctx, OKR_EINVAL, "vhat/ihat is NULL");
    const int n = f->n_bus, L = f->n_scen;
    CK(cudaSetDevice(ctx->device));
    s = ensure_workspace(ctx, n, L, p->record_iters);
    if (s != OKR_OK) return s;
    cudaStream_t st = ctx->stream;
    const cudaMemcpyKind kind = (src == Src::Device) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(ctx->fb.parent_in, f->parent, sizeof(int) * n, kind, st));
    CK(cudaMemcpyAsync(ctx->fb.ph_in, f->phases, n, kind, st));
    CK(cudaMemcpyAsync(ctx->fb.z_in, f->z_line, sizeof(double) * 18 * n, kind, st));
    if (src == Src::Ops) {
        CK(cudaMemcpyAsync(ctx->fb.vh_in, vhat, sizeof(double) * 6 * L * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ctx->fb.ih_in, ihat, sizeof(double) * 6 * L * n, cudaMemcpyHostToDevice, st));
    } else {
        CK(cudaMemcpyAsync(ctx->fb.s_in, f->s_load, sizeof(double) * 6 * L * n, kind, st));
    }
    // the incremental engine's path waits once, after the last launch (the
    // sweep engine sizes its work buffers from the tree's statistics first)
    const bool one_wait = run_engine(ctx, n, p) == OKR_ENGINE_INCREMENTAL;
    s = build_topology(ctx, n, L, &f->v_slack[0][0], !one_wait);
    if (s != OKR_OK) return s;
    if (src == Src::Ops) {
        k_import_ops<<<blocks_for((size_t)L * n, 256, ctx->num_sms * 8), 256, 0, st>>>(n, L, ctx->fb.T, ctx->fb.vh_in, ctx->fb.ih_in);
        ctx->launches += 1;
        CK(cudaGetLastError());
        ctx->pf_sweeps = 0;
    } else {
        s = run_power_flow(ctx, n, L, p->max_spins);
        if (s != OKR_OK) return s;
    }
    if (one_wait) {
        if (src != Src::Ops) ctx->pf_sweeps = -1;   // read after the search
    } else {
        s = read_setup_errors(ctx);
        if (s != OKR_OK) return s;
        if (src != Src::Ops) {
            int it[kMaxScen];
            CK(cudaMemcpy(it, ctx->fb.pf_iters, sizeof(int) * L, cudaMemcpyDeviceToHost));
            int w = 0;
            for (int l = 0; l < L; ++l) w = it[l] > w ? it[l] : w;
            ctx->pf_sweeps = w;
        }
    }
    CK(join_side(ctx));
    s = run_search(ctx, p);
    if (s != OKR_OK) return s;
    ctx->n = n;
    ctx->L = L;
    ctx->have_result = true;
    return OKR_OK;
}

}  // namespace

// ======================================================================= C ABI
namespace {

okr_status ensure_kron_work(okr_ctx *ctx, int n) {
    if (ctx->cap_kron_n < n) {
        for (void *q : ctx->kron_allocs) dev_free(ctx, q);
        ctx->kron_allocs.clear();
        ctx->cap_kron_n = 0;
        KronWork &W = ctx->kw;
        auto take = [&](auto **ptr, size_t count) -> cudaError_t {
            void *q = nullptr;
            cudaError_t e = dev_alloc(ctx, &q, sizeof(**ptr) * (count ? count : 1));
            if (e == cudaSuccess) { ctx->kron_allocs.push_back(q); *ptr = static_cast<std::remove_reference_t<decltype(*ptr)>>(q); }
            return e;
        };
        const size_t N = n;
        CK(take(&W.keptp, N));
        CK(take(&W.g, N));
        CK(take(&W.key, N));
        CK(take(&W.cnt, N));
        CK(take(&W.dsum, N));
        CK(take(&W.fill, N));
        CK(take(&W.goff, N));
        CK(take(&W.ports, N));
        CK(take(&W.out_off, N + 1));
        CK(take(&W.pn, 3 * N));
        CK(take(&W.gkey, N));
        CK(take(&W.gp, N));
        CK(take(&W.gd, N));
        CK(take(&W.gport, N + 1));
        CK(take(&W.grow, N + 1));
        CK(take(&W.rows, 3 * N));
        CK(take(&W.gbig, N));
        CK(take(&W.hdr, 1));
        CK(take(&ctx->kron_kept, N));
        CK(take(&ctx->kron_crit, N));
        CK(take(&ctx->kron_count, 1));
        ctx->cap_kron_n = n;
    }
    return OKR_OK;
}

}  // namespace

extern "C" {

void okr_default_params(okr_params *p) {
    if (!p) return;
    p->margin = 0.005;
    p->target_reduction = 1.0;
    p->tie_tol = 1e-9;
    p->objective = 0;
    p->precision = 0;
    p->record_iters = 0;
    p->max_merges = -1;
    p->profile = 0;
    p->scorer_topk = 0;
    p->engine = OKR_ENGINE_AUTO;
    p->max_spins = 0;
    p->prune_exact = 0;
    p->reserved = 0;
}

const char *okr_status_str(okr_status s) {
    switch (s) {
    case OKR_OK: return "ok";
    case OKR_EINVAL: return "invalid argument";
    case OKR_ENOMEM: return "out of memory";
    case OKR_ECUDA: return "CUDA error";
    case OKR_EPF: return "load flow did not converge";
    case OKR_ETIMEOUT: return "device wait timed out";
    case OKR_ENOTREADY: return "no result";
    case OKR_ESINGULAR: return "singular line impedance";
    case OKR_EINTERNAL: return "internal error";
    }
    return "unknown status";
}

const char *okr_last_error(const okr_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

okr_status okr_create(okr_ctx **out, int device, void *stream) {
    if (!out) return OKR_EINVAL;
    *out = nullptr;
    okr_ctx *ctx = new (std::nothrow) okr_ctx();
    if (!ctx) return OKR_ENOMEM;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device < 0 || device >= count) {
        delete ctx;
        return e != cudaSuccess ? OKR_ECUDA : OKR_EINVAL;
    }
    ctx->device = device;
    if ((e = cudaSetDevice(device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) {
        delete ctx;
        return OKR_ECUDA;
    }
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop ||
        search_blocks_per_sm() < 1) {
        delete ctx;
        return OKR_ECUDA;
    }
    ctx->grid = ctx->num_sms;               // one CTA per SM: all co-resident
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return OKR_ECUDA; }
        ctx->own_stream = true;
    }
    if (cudaMallocHost((void **)&ctx->C_host, kHostStageBytes) != cudaSuccess) {
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return OKR_ENOMEM;
    }
    if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_topo, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_lines, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_side, cudaEventDisableTiming) != cudaSuccess) {
        okr_destroy(ctx);
        return OKR_ECUDA;
    }
    *out = ctx;
    return OKR_OK;
}

okr_status okr_set_allocator(okr_ctx *ctx, okr_alloc_fn alloc, okr_free_fn free_fn, void *user) {
    if (!ctx) return OKR_EINVAL;
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(ctx, OKR_EINVAL, "allocator: give both alloc and free, or neither");
    if (ctx->live_allocs != 0)
        return fail(ctx, OKR_EINVAL, "allocator: the context already holds %lld device blocks (set it right after "
                                     "okr_create)", ctx->live_allocs);
    ctx->alloc_fn = alloc;
    ctx->free_fn = free_fn;
    ctx->alloc_user = user;
    return OKR_OK;
}

okr_status okr_destroy(okr_ctx *ctx) {
    if (!ctx) return OKR_EINVAL;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    free_batch(ctx);
    free_mlp(ctx);
    if (ctx->C_host) cudaFreeHost(ctx->C_host);
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
    }
    for (cudaEvent_t ev : {ctx->ev_topo, ctx->ev_lines, ctx->ev_side})
        if (ev) cudaEventDestroy(ev);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return OKR_OK;
}

okr_status okr_reduce(okr_ctx *ctx, const okr_feeder *f, const okr_params *p) {
    return reduce_impl(ctx, f, nullptr, nullptr, p, Src::Host);
}

okr_status okr_reduce_device(okr_ctx *ctx, const okr_feeder *f, const okr_params *p) {
    return reduce_impl(ctx, f, nullptr, nullptr, p, Src::Device);
}

okr_status okr_reduce_ops(okr_ctx *ctx, const okr_feeder *f, const double *vhat, const double *ihat,
                          const okr_params *p) {
    return reduce_impl(ctx, f, vhat, ihat, p, Src::Ops);
}

okr_status okr_power_flow(okr_ctx *ctx, const okr_feeder *f, double *vhat_out, double *ihat_out, int32_t *sweeps) {
    if (!ctx) return OKR_EINVAL;
    ctx->have_result = false;
    ctx->have_topo = false;
    okr_status s = check_feeder_shape(ctx, f);
    if (s != OKR_OK) return s;
    if (!f->s_load || !vhat_out) return fail(ctx, OKR_EINVAL, "s_load or vhat_out is NULL");
    const int n = f->n_bus, L = f->n_scen;
    CK(cudaSetDevice(ctx->device));
    s = ensure_workspace(ctx, n, L, ctx->cap_rec);
    if (s != OKR_OK) return s;
    cudaStream_t st = ctx->stream;
    CK(cudaMemcpyAsync(ctx->fb.parent_in, f->parent, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->fb.ph_in, f->phases, n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->fb.z_in, f->z_line, sizeof(double) * 18 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->fb.s_in, f->s_load, sizeof(double) * 6 * L * n, cudaMemcpyHostToDevice, st));
    s = build_topology(ctx, n, L, &f->v_slack[0][0]);
    if (s != OKR_OK) return s;
    s = run_power_flow(ctx, n, L);
    if (s != OKR_OK) return s;
    s = read_setup_errors(ctx);
    if (s != OKR_OK) return s;
    // export: reuse k_export with the initial state (each bus its own super-node)
    k_state_init<<<blocks_for((size_t)L * n, 256, ctx->num_sms * 8), 256, 0, st>>>(n, L, ctx->fb.T, ctx->fb.S);
    k_export<<<blocks_for((size_t)L * n, 256, ctx->num_sms * 8), 256, 0, st>>>(ctx->fb.T, ctx->fb.S, nullptr, nullptr,
                                                                                ctx->fb.vhat_out);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(vhat_out, ctx->fb.vhat_out, sizeof(double) * 6 * L * n, cudaMemcpyDeviceToHost, st));
    if (ihat_out) {
        // S.icur == Ihat after the initial state; export it through vred's slot
        State si = ctx->fb.S;
        si.vcur = ctx->fb.S.icur;                  // export the injections through the voltage slot
        k_export<<<blocks_for((size_t)L * n, 256, ctx->num_sms * 8), 256, 0, st>>>(ctx->fb.T, si, ctx->fb.vred_out,
                                                                                    nullptr, nullptr);
        CK(cudaMemcpyAsync(ihat_out, ctx->fb.vred_out, sizeof(double) * 6 * L * n, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    if (sweeps) {
        int it[kMaxScen];
        CK(cudaMemcpy(it, ctx->fb.pf_iters, sizeof(int) * L, cudaMemcpyDeviceToHost));
        int w = 0;
        for (int l = 0; l < L; ++l) w = it[l] > w ? it[l] : w;
        *sweeps = w;
    }
    return OKR_OK;
}

okr_status okr_evaluate(okr_ctx *ctx, const okr_feeder *f, const int32_t *super_of, double *max_error, double *vred) {
    if (!ctx) return OKR_EINVAL;
    ctx->have_result = false;
    ctx->have_topo = false;
    okr_status s = check_feeder_shape(ctx, f);
    if (s != OKR_OK) return s;
    if (!f->s_load || !super_of || !max_error) return fail(ctx, OKR_EINVAL, "s_load, super_of or max_error is NULL");
    const int n = f->n_bus, L = f->n_scen;
    if (super_of[0] != 0) return fail(ctx, OKR_EINVAL, "the slack bus must be its own super-node");
    std::vector<int> moff(n + 1, 0), mem(n);
    for (int i = 0; i < n; ++i) {
        const int k = super_of[i];
        if (k < 0 || k >= n || super_of[k] != k) return fail(ctx, OKR_EINVAL, "super_of[%d] = %d is not a super-node", i, k);
        moff[k + 1] += 1;
    }
    for (int i = 0; i < n; ++i) moff[i + 1] += moff[i];
    {
        std::vector<int> fill(moff.begin(), moff.end() - 1);
        for (int i = 0; i < n; ++i) mem[fill[super_of[i]]++] = i;      // members in increasing caller id
    }
    CK(cudaSetDevice(ctx->device));
    s = ensure_workspace(ctx, n, L, ctx->cap_rec);
    if (s != OKR_OK) return s;
    cudaStream_t st = ctx->stream;
    FeederBufs &B = ctx->fb;
    CK(cudaMemcpyAsync(B.parent_in, f->parent, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.ph_in, f->phases, n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.z_in, f->z_line, sizeof(double) * 18 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.s_in, f->s_load, sizeof(double) * 6 * L * n, cudaMemcpyHostToDevice, st));
    s = build_topology(ctx, n, L, &f->v_slack[0][0]);
    if (s != OKR_OK) return s;
    s = run_power_flow(ctx, n, L);
    if (s != OKR_OK) return s;
    s = read_setup_errors(ctx);
    if (s != OKR_OK) return s;
    // the member lists go into buffers this call does not otherwise use
    // (super_out [n], base [2n+1], dec_s [n], score [2n >= 4])
    int *sup_d = B.super_out, *moff_d = B.X.base, *mem_d = B.X.dec_s;
    CK(cudaMemcpyAsync(sup_d, super_of, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(moff_d, moff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(mem_d, mem.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    double *err_d = B.X.score;
    k_eval_reduced<<<L, 1024, 0, st>>>(B.T, sup_d, moff_d, mem_d, B.J, B.S.vcur, vred ? B.vred_out : nullptr, err_d);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(max_error, err_d, sizeof(double) * L, cudaMemcpyDeviceToHost, st));
    if (vred) CK(cudaMemcpyAsync(vred, B.vred_out, sizeof(double) * 6 * L * n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return OKR_OK;
}

okr_status okr_radialize(okr_ctx *ctx, const uint8_t *kept, uint8_t *critical, int32_t *n_critical) {
    if (!ctx || !critical) return OKR_EINVAL;
    if (!ctx->have_topo) return fail(ctx, OKR_ENOTREADY, "no feeder: run a reduction or a load flow first");
    if (!kept && !ctx->have_result) return fail(ctx, OKR_ENOTREADY, "no reduction result to take the kept set from");
    if (kept && !kept[0]) return fail(ctx, OKR_EINVAL, "the slack bus (bus 0) must be kept");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int n = ctx->fb.T.n;
    okr_status ks = ensure_kron_work(ctx, n);
    if (ks != OKR_OK) return ks;
    if (kept) CK(cudaMemcpyAsync(ctx->kron_kept, kept, n, cudaMemcpyHostToDevice, st));
    k_radial_critical<<<1, 1024, 0, st>>>(ctx->fb.T, kept ? nullptr : ctx->fb.S.label, kept ? ctx->kron_kept : nullptr,
                                          ctx->kw, ctx->kron_crit, ctx->kron_count);
    CK(cudaGetLastError());
    int cnt = 0;
    CK(cudaMemcpyAsync(critical, ctx->kron_crit, n, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&cnt, ctx->kron_count, sizeof cnt, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (n_critical) *n_critical = cnt;
    return OKR_OK;
}

okr_status okr_kron(okr_ctx *ctx, const uint8_t *kept, int32_t cap, double *y_out, int32_t *phase_node,
                    int32_t *k_phi) {
    if (!ctx || !k_phi) return OKR_EINVAL;
    if (!ctx->have_topo) return fail(ctx, OKR_ENOTREADY, "no feeder: run a reduction or a load flow first");
    if (!kept && !ctx->have_result) return fail(ctx, OKR_ENOTREADY, "no reduction result to take the kept set from");
    if ((y_out || phase_node) && cap < 0) return fail(ctx, OKR_EINVAL, "cap < 0");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int n = ctx->fb.T.n;
    okr_status ks = ensure_kron_work(ctx, n);
    if (ks != OKR_OK) return ks;
    KronWork &W = ctx->kw;
    uint8_t *kept_dev = nullptr;
    if (kept) {
        kept_dev = ctx->kron_kept;
        CK(cudaMemcpyAsync(kept_dev, kept, n, cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemsetAsync(W.hdr, 0, sizeof(KronHdr), st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, st));
    k_kron_groups<<<1, 1024, 0, st>>>(ctx->fb.T, kept ? nullptr : ctx->fb.S.label, kept_dev, W);
    CK(cudaGetLastError());
    KronHdr h{};
    CK(cudaMemcpyAsync(&h, W.hdr, sizeof h, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    okr_status s = OKR_OK;
    if (h.err == 1) s = fail(ctx, OKR_EINVAL, "the slack bus (bus 0) must be kept");
    else if (h.max_d > kKronMaxGroup)
        s = fail(ctx, OKR_EINVAL, "a reduced component has %d boundary phase-nodes (at most %d)", h.max_d, kKronMaxGroup);
    if (s != OKR_OK || (!y_out && !phase_node)) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *k_phi = h.k_phi;
        return s;
    }
    *k_phi = h.k_phi;
    if (cap < h.k_phi) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(ctx, OKR_EINVAL, "cap %d < k_phi %d", cap, h.k_phi);
    }
    const size_t K = h.k_phi, need_y = K * K, need_big = (size_t)h.big_total;
    if (need_y > ctx->cap_ykr) {
        dev_free(ctx, ctx->ykr);
        ctx->ykr = nullptr;
        ctx->cap_ykr = 0;
        CK(dev_alloc(ctx, (void **)&ctx->ykr, sizeof(double2) * need_y));
        ctx->cap_ykr = need_y;
    }
    if (need_big > ctx->cap_kbig) {
        dev_free(ctx, ctx->kbig);
        ctx->kbig = nullptr;
        ctx->cap_kbig = 0;
        CK(dev_alloc(ctx, (void **)&ctx->kbig, sizeof(double2) * need_big));
        ctx->cap_kbig = need_big;
    }
    CK(cudaMemsetAsync(ctx->ykr, 0, sizeof(double2) * need_y, st));
    CK(launch_kron_solve(h.n_groups, ctx->fb.T, W, ctx->kbig, ctx->ykr, (int)K, st));
    if (K > 0) k_kron_diag<<<blocks_for(K * 32, 256, ctx->num_sms * 8), 256, 0, st>>>(W, ctx->ykr, (int)K);
    CK(cudaGetLastError());
    CK(cudaEventRecord(e1, st));
    CK(cudaMemcpyAsync(&h, W.hdr, sizeof h, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ctx->kron_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (h.err == 2) return fail(ctx, OKR_ESINGULAR, "singular port impedance block in the Kron reduction");
    if (y_out) CK(cudaMemcpy(y_out, ctx->ykr, sizeof(double2) * need_y, cudaMemcpyDeviceToHost));
    if (phase_node) CK(cudaMemcpy(phase_node, W.pn, sizeof(int) * K, cudaMemcpyDeviceToHost));
    return OKR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- many feeders
namespace {

// Host check of the tree rules (the batched setup does not stop between kernels).
bool valid_tree(const okr_feeder *f) {
    const int n = f->n_bus;
    if (f->parent[0] != -1 || f->phases[0] == 0 || f->phases[0] > 7) return false;
    for (int i = 1; i < n; ++i) {
        const int p = f->parent[i];
        const unsigned m = f->phases[i];
        if (p < 0 || p >= i || m == 0 || m > 7 || (m & f->phases[p]) != m) return false;
    }
    return true;
}

okr_status batch_status_of_setup(int e) {
    switch (e) {
    case 0: return OKR_OK;
    case 1: return OKR_EINVAL;
    case 2: return OKR_ESINGULAR;
    case 3: return OKR_EPF;
    case 6: return OKR_ETIMEOUT;
    default: return OKR_EINTERNAL;
    }
}

}  // namespace

// One batch of feeders, laid out in one device arena and one pinned host
// block.  The host block holds the staged inputs (descriptors, controls, the
// order, queues, feeder arrays), then a result area (controls, setup errors,
// largest errors, copied back after the run) and the assignments.
struct BatchRun {
    int nf = 0, config = 0, team = 1, max_teams = 1, maxL = 1, ctas = 0;
    IncShape shape{0, 0, 0, -1};                    // incremental engine: launch shape (resolved)
    long long max_nn = 1, tot_n = 0;
    int per_sm[2] = {0, 0};
    std::vector<int> merges, nbus, nscen, ord[4];
    std::vector<long long> sum_sz;
    std::vector<size_t> in_off, fb_off, super_pos;
    std::vector<okr_params> params;                 // one per feeder
    size_t staged = 0, total = 0, super_off = 0, res_off = 0, res_len = 0, host_bytes = 0;
    unsigned char *base = nullptr, *hb = nullptr;
    BatchSetup *bs_d = nullptr;
    BatchFeeder *bf_d = nullptr;
    Ctrl *ctrl_d = nullptr;
    int *order_d = nullptr, *queue_d = nullptr, *err_d = nullptr, *super_all_d = nullptr;
    double *maxerr_d = nullptr;
    BatchTeam *teams_d = nullptr;
    int *ictas_d = nullptr;                         // incremental groups: first CTA of each feeder's first evaluation
    int init_ctas[2] = {0, 0};                      // CTAs of that evaluation, per precision
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;    // the setup's side-stream fork and join
    ~BatchRun() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
    }
    // host views of the result area and of the assignments
    const Ctrl *ctrl_res() const { return reinterpret_cast<const Ctrl *>(hb + staged); }
    const int *err_res() const { return reinterpret_cast<const int *>(hb + staged + ((unsigned char *)err_d - (unsigned char *)ctrl_d)); }
    const double *maxerr_res() const {
        return reinterpret_cast<const double *>(hb + staged + ((unsigned char *)maxerr_d - (unsigned char *)ctrl_d));
    }
    int *super_res() const { return reinterpret_cast<int *>(hb + staged + res_len); }
};

// Checks the batch and computes every size and offset (no memory touched).
static okr_status batch_measure(okr_ctx *ctx, int32_t nf, const okr_feeder *feeders, const okr_params *params,
                                int32_t n_params, int config, BatchRun &R) {
    if (nf < 1 || !feeders || !params) return fail(ctx, OKR_EINVAL, "batch: bad arguments");
    if (n_params != 1 && n_params != nf) return fail(ctx, OKR_EINVAL, "batch: n_params must be 1 or n_feeders");
    if (config < 0 || config > 3) return fail(ctx, OKR_EINVAL, "batch: config %d", config);
    R.nf = nf;
    R.config = config;
    R.team = 1 << config;                               // CTAs per feeder: 1, 2, 4, 8
    R.shape = inc_shape_resolve(ctx->inc_shape);
    R.per_sm[0] = search_batch_blocks_per_sm(0);
    R.per_sm[1] = search_batch_blocks_per_sm(1);
    if (R.per_sm[0] < 1 || R.per_sm[1] < 1) return fail(ctx, OKR_ECUDA, "batched search: no CTA fits an SM");
    R.max_teams = std::max(1, ctx->num_sms * std::max(R.per_sm[0], R.per_sm[1]) / R.team);
    R.sum_sz.assign(nf, 0);
    R.merges.assign(nf, 0);
    R.nbus.assign(nf, 0);
    R.nscen.assign(nf, 0);
    R.params.assign(nf, okr_params{});
    for (int f = 0; f < nf; ++f) {
        const okr_feeder *F = &feeders[f];
        const okr_params *P = &params[n_params == 1 ? 0 : f];
        okr_status st = check_feeder_shape(ctx, F);
        if (st == OKR_OK) st = check_params(ctx, P);
        if (st != OKR_OK) return fail(ctx, st, "batch feeder %d: %s", f, ctx->err.c_str());
        if (!F->s_load) return fail(ctx, OKR_EINVAL, "batch feeder %d: s_load is NULL", f);
        if (P->record_iters != 0) return fail(ctx, OKR_EINVAL, "batch feeder %d: record_iters must be 0", f);
        if (P->scorer_topk != 0) return fail(ctx, OKR_EINVAL, "batch feeder %d: scorer_topk must be 0", f);
        if (!valid_tree(F)) return fail(ctx, OKR_EINVAL, "batch feeder %d: invalid tree or phases", f);
        const int n = F->n_bus;
        std::vector<int> dep(n, 0);
        long long ss = 0;
        for (int i = 0; i < n; ++i) {
            if (i > 0) dep[i] = dep[F->parent[i]] + 1;
            ss += dep[i] + 1;
        }
        R.sum_sz[f] = ss;
        R.merges[f] = merges_for(n, P);
        R.nbus[f] = n;
        R.nscen[f] = F->n_scen;
        R.params[f] = *P;
        R.maxL = std::max(R.maxL, (int)F->n_scen);
        R.max_nn = std::max(R.max_nn, (long long)n * n);
        R.tot_n += n;
    }
    // largest expected work first; lists: sweep FP64, sweep mixed precision,
    // incremental FP64, incremental mixed precision
    for (int g = 0; g < 4; ++g) R.ord[g].clear();
    for (int f = 0; f < nf; ++f) {
        const okr_params &P = R.params[f];
        const bool inc = resolve_engine(&P) == OKR_ENGINE_INCREMENTAL && inc_fits(ctx, R.nbus[f], &P);
        R.ord[(inc ? 2 : 0) + P.precision].push_back(f);
    }
    for (int g = 0; g < 4; ++g)
        std::stable_sort(R.ord[g].begin(), R.ord[g].end(), [&](int a, int b) {
            return (double)R.nbus[a] * R.merges[a] > (double)R.nbus[b] * R.merges[b];
        });
    // the incremental launches need their shape's record placement to fit
    for (int g = 2; g < 4; ++g) {
        if (R.ord[g].empty()) continue;
        int max_n = 2;
        for (int f : R.ord[g]) max_n = std::max(max_n, R.nbus[f]);
        int rec = 0;
        size_t bytes = 0;
        if (!inc_smem(max_n, false, R.shape, &rec, &bytes))
            return fail(ctx, OKR_EINVAL, "batch: the incremental shape's record placement does not fit (%d buses; "
                                         "the largest MICE per super-node is single-feeder only)", max_n);
    }
    // ---- layout: [staged block: descriptors, controls, order, queues, flags, inputs] [per-feeder buffers] [outputs]
    Carver m;
    m.take(R.bs_d, nf);
    m.take(R.bf_d, nf);
    R.res_off = m.used;                         // result area: controls .. largest errors
    m.take(R.ctrl_d, nf);
    m.take(R.order_d, nf);
    m.take(R.queue_d, 2);
    m.take(R.err_d, nf);
    m.take(R.maxerr_d, nf);
    R.res_len = m.used - R.res_off;
    m.take(R.teams_d, 2 * (size_t)R.max_teams);
    m.take(R.ictas_d, (size_t)nf + 1);
    R.in_off.assign(nf, 0);
    for (int f = 0; f < nf; ++f) {
        const size_t n = R.nbus[f], L = R.nscen[f];
        R.in_off[f] = m.used;
        int *a; uint8_t *b; double *c, *d; double2 *e;
        m.take(a, n);
        m.take(b, n);
        m.take(c, 18 * n);
        m.take(d, 6 * L * n);
        m.take(e, 3);
    }
    R.staged = m.used;
    R.fb_off.assign(nf, 0);
    Carver w;
    w.used = R.staged;
    for (int f = 0; f < nf; ++f) {
        const int n = R.nbus[f], L = R.nscen[f];
        const int ppc = positions_per_chunk(L);
        const long long chunks = 2LL * ((2LL * R.sum_sz[f] + 2LL * n + ppc - 1) / ppc + 1);
        R.fb_off[f] = w.used;
        FeederBufs tmp;
        layout_feeder(w, n, L, 0, 8, chunks, tmp);          // per-CTA sums for teams of up to 8
    }
    R.super_off = w.used;
    int *sup = nullptr;
    w.take(sup, (size_t)R.tot_n);
    R.total = w.used;
    R.host_bytes = R.staged + R.res_len + sizeof(int) * (size_t)R.tot_n;
    return OKR_OK;
}

// Device pointers of the arena at R.base and the staged inputs in R.hb.
static okr_status batch_fill(okr_ctx *ctx, BatchRun &R, const okr_feeder *feeders) {
    const int nf = R.nf;
    unsigned char *base = R.base, *hb = R.hb;
    std::memset(hb, 0, R.staged);
    Carver md;
    md.base = base;
    md.take(R.bs_d, nf);
    md.take(R.bf_d, nf);
    md.take(R.ctrl_d, nf);
    md.take(R.order_d, nf);
    md.take(R.queue_d, 2);
    md.take(R.err_d, nf);
    md.take(R.maxerr_d, nf);
    md.take(R.teams_d, 2 * (size_t)R.max_teams);
    md.take(R.ictas_d, (size_t)nf + 1);
    R.super_all_d = reinterpret_cast<int *>(base + R.super_off);
    Carver mh;                                  // the same offsets in the host buffer
    mh.base = hb;
    BatchSetup *bs_h; BatchFeeder *bf_h; Ctrl *ctrl_h; int *order_h, *queue_h, *err_h; double *maxerr_h;
    mh.take(bs_h, nf);
    mh.take(bf_h, nf);
    mh.take(ctrl_h, nf);
    mh.take(order_h, nf);
    mh.take(queue_h, 2);
    mh.take(err_h, nf);
    mh.take(maxerr_h, nf);
    BatchTeam *teams_h;
    mh.take(teams_h, 2 * (size_t)R.max_teams);
    int *ictas_h;
    mh.take(ictas_h, (size_t)nf + 1);
    for (int i = 0; i < 2 * R.max_teams; ++i) {
        teams_h[i].ctrl.max_spins = R.params[0].max_spins > 0 ? R.params[0].max_spins : kDefaultSpins;
        teams_h[i].slot = 0;
    }
    size_t soff = 0;
    R.super_pos.assign(nf, 0);
    for (int f = 0; f < nf; ++f) {
        const okr_feeder *F = &feeders[f];
        const okr_params *P = &R.params[f];
        const int n = F->n_bus, L = F->n_scen;
        const int ppc = positions_per_chunk(L);
        const long long chunks = 2LL * ((2LL * R.sum_sz[f] + 2LL * n + ppc - 1) / ppc + 1);
        Carver c;
        c.base = base + R.fb_off[f];
        FeederBufs B;
        layout_feeder(c, n, L, 0, 8, chunks, B);
        // inputs live in the staged block
        Carver ci;
        ci.base = base + R.in_off[f];
        Carver chh;
        chh.base = hb + R.in_off[f];
        int *pd, *ph_; uint8_t *phd, *phh; double *zd, *zh_, *sd, *sh_; double2 *vd, *vh_;
        ci.take(pd, n); ci.take(phd, n); ci.take(zd, 18 * (size_t)n); ci.take(sd, 6 * (size_t)L * n); ci.take(vd, 3);
        chh.take(ph_, n); chh.take(phh, n); chh.take(zh_, 18 * (size_t)n); chh.take(sh_, 6 * (size_t)L * n); chh.take(vh_, 3);
        std::memcpy(ph_, F->parent, sizeof(int) * n);
        std::memcpy(phh, F->phases, n);
        std::memcpy(zh_, F->z_line, sizeof(double) * 18 * n);
        std::memcpy(sh_, F->s_load, sizeof(double) * 6 * L * n);
        for (int p = 0; p < 3; ++p) vh_[p] = make_double2(F->v_slack[p][0], F->v_slack[p][1]);
        B.T.vslack = vd;
        B.C = R.ctrl_d + f;
        B.err_dev = R.err_d + f;
        R.super_pos[f] = soff;
        B.super_out = R.super_all_d + soff;
        soff += n;
        BatchSetup &S = bs_h[f];
        S.n = n;
        S.L = L;
        S.nlev = log2_ceil(n) + 1;
        S.parent_in = pd;
        S.ph_in = phd;
        S.z_in = zd;
        S.s_in = sd;
        S.T = B.T;
        S.S = B.S;
        S.dep = B.dep; S.anc = B.anc; S.anc2 = B.anc2; S.d2 = B.d2; S.size = B.size; S.ccount = B.ccount;
        S.coff_c = B.coff_c; S.child_c = B.child_c;
        S.rmq = B.rmq;
        S.J = B.J;
        S.pf_iters = B.pf_iters;
        S.err = B.err_dev;
        S.dec_maxerr = B.X.dec_maxerr;
        S.mrank = B.X.mrank;
        S.bmax = B.X.bmax;
        S.arrive = B.X.arrive;
        BatchFeeder &D = bf_h[f];
        D.T = B.T;
        D.S = B.S;
        D.X = B.X;
        D.X.rec_iters = 0;
        D.I = B.I;
        D.C = B.C;
        D.setup_err = B.err_dev;
        D.super_out = B.super_out;
        D.max_err = R.maxerr_d + f;
        Ctrl &cc = ctrl_h[f];
        cc.max_merges = R.merges[f];
        cc.done = (R.merges[f] == 0);
        cc.margin = P->margin;
        cc.tau = P->tie_tol;
        cc.profile = 0;
        cc.n_super = n;
        cc.precision = P->precision;
        cc.objective = P->objective;
        cc.max_spins = P->max_spins > 0 ? P->max_spins : kDefaultSpins;
    }
    int k = 0;
    for (int g = 0; g < 4; ++g) {
        int ctas = 0;
        for (int f : R.ord[g]) {
            if (g >= 2) {                           // the incremental groups' first evaluation on many CTAs
                ictas_h[k] = ctas;
                ctas += inc_init_batch_ctas(R.nbus[f]);
            }
            order_h[k++] = f;
        }
        if (g >= 2) R.init_ctas[g - 2] = ctas;
    }
    for (cudaEvent_t &e : R.ev)
        if (!e) CK(cudaEventCreate(&e));
    if (!R.ev_fork) CK(cudaEventCreateWithFlags(&R.ev_fork, cudaEventDisableTiming));
    if (!R.ev_join) CK(cudaEventCreateWithFlags(&R.ev_join, cudaEventDisableTiming));
    // attributes the launches need, set before any stream capture
    for (int g = 2; g < 4; ++g) {
        int max_n = 2;
        for (int f : R.ord[g]) max_n = std::max(max_n, R.nbus[f]);
        if (!R.ord[g].empty()) {
            CK(prepare_search_inc_batch(g - 2, max_n, R.shape));
            CK(prepare_inc_init_batch(g - 2, max_n));
        }
    }
    return OKR_OK;
}

// The device work of one run on stream st: inputs, setup, searches, results.
static okr_status batch_enqueue(okr_ctx *ctx, BatchRun &R, cudaStream_t st, bool want_super, bool captured) {
    const int nf = R.nf;
    // in a graph, event records are nodes of their own only when external
    const unsigned evf = captured ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (!captured) CK(join_side(ctx));          // (the setup forks onto the side stream)
    CK(cudaMemcpyAsync(R.base, R.hb, R.staged, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecordWithFlags(R.ev[0], st, evf));
    CK(launch_batch_setup(nf, R.maxL, R.max_nn, R.bs_d, kPfTol, kPfMaxIter, ctx->num_sms, st, ctx->side, R.ev_fork,
                          R.ev_join));
    CK(cudaEventRecordWithFlags(R.ev[1], st, evf));
    R.ctas = 0;
    for (int g = 0, first = 0; g < 4; first += (int)R.ord[g].size(), ++g) {
        const int cnt = (int)R.ord[g].size();
        if (cnt == 0) continue;
        if (g >= 2) {                           // one CTA per feeder
            R.ctas = std::max(R.ctas, cnt);
            int max_n = 2;
            for (int f : R.ord[g]) max_n = std::max(max_n, R.nbus[f]);
            CK(launch_inc_init_batch(g - 2, max_n, R.bf_d, R.order_d + first, R.ictas_d + first, cnt,
                                     R.init_ctas[g - 2], st));
            CK(launch_search_inc_batch(g - 2, max_n, R.bf_d, R.order_d + first, cnt, R.shape, st));
            continue;
        }
        const int nteams = std::min(cnt, ctx->num_sms * R.per_sm[g] / R.team);
        if (nteams < 1) return fail(ctx, OKR_EINVAL, "batched search: team of %d CTAs does not fit", R.team);
        const int grid = nteams * R.team;
        R.ctas = std::max(R.ctas, grid);
        CK(launch_search_batch(g, R.team, grid, R.bf_d, R.order_d + first, cnt, R.queue_d + g,
                               R.teams_d + g * R.max_teams, st));
    }
    CK(cudaEventRecordWithFlags(R.ev[2], st, evf));
    // results: controls, setup errors and largest errors (one copy), assignments
    CK(cudaMemcpyAsync(R.hb + R.staged, R.base + R.res_off, R.res_len, cudaMemcpyDeviceToHost, st));
    if (want_super)
        CK(cudaMemcpyAsync(R.super_res(), R.base + R.super_off, sizeof(int) * (size_t)R.tot_n, cudaMemcpyDeviceToHost, st));
    return OKR_OK;
}

// After the stream finished: the items, the assignments and the statistics.
// A feeder whose sweep work buffer overflowed is re-run alone (its feeder is
// read back from the staged block).
static okr_status batch_finish(okr_ctx *ctx, BatchRun &R, okr_batch_item *items, int32_t *super_of,
                               okr_batch_stats *stats) {
    const int nf = R.nf;
    float ms_setup = 0.f, ms_search = 0.f;
    cudaEventElapsedTime(&ms_setup, R.ev[0], R.ev[1]);
    cudaEventElapsedTime(&ms_search, R.ev[1], R.ev[2]);
    const Ctrl *ctrl = R.ctrl_res();
    const int *serr = R.err_res();
    const double *maxerr = R.maxerr_res();
    if (super_of) std::memcpy(super_of, R.super_res(), sizeof(int) * (size_t)R.tot_n);
    int64_t cand_total = 0;
    int fallbacks = 0;
    for (int f = 0; f < nf; ++f) {
        okr_batch_item &it = items[f];
        std::memset(&it, 0, sizeof it);
        const Ctrl c = ctrl[f];
        if (serr[f]) { it.status = batch_status_of_setup(serr[f]); continue; }
        if (c.err == 7) {                       // work buffers too small: run this feeder alone
            ++fallbacks;
            const int n = R.nbus[f], L = R.nscen[f];
            Carver chh;
            chh.base = R.hb + R.in_off[f];
            int *ph_; uint8_t *phh; double *zh_, *sh_; double2 *vh_;
            chh.take(ph_, n); chh.take(phh, n); chh.take(zh_, 18 * (size_t)n); chh.take(sh_, 6 * (size_t)L * n);
            chh.take(vh_, 3);
            okr_feeder F{};
            F.n_bus = n;
            F.n_scen = L;
            F.parent = ph_;
            F.phases = phh;
            F.z_line = zh_;
            F.s_load = sh_;
            for (int p = 0; p < 3; ++p) { F.v_slack[p][0] = vh_[p].x; F.v_slack[p][1] = vh_[p].y; }
            okr_status s2 = reduce_impl(ctx, &F, nullptr, nullptr, &R.params[f], Src::Host);
            it.status = s2;
            if (s2 != OKR_OK) continue;
            const Ctrl &l = ctx->last;
            it.n_iter = l.t;
            it.stop_reason = l.stop_reason;
            it.n_kept = n - l.t;
            it.candidates = l.candidates;
            it.smice = l.s_cur;
            double me = 0.0;
            if (l.t > 0) CK(cudaMemcpy(&me, ctx->fb.X.dec_maxerr + (l.t - 1), sizeof me, cudaMemcpyDeviceToHost));
            it.max_error = me;
            if (super_of) CK(cudaMemcpy(super_of + R.super_pos[f], ctx->fb.super_out, sizeof(int) * n,
                                        cudaMemcpyDeviceToHost));
            cand_total += l.candidates;
            continue;
        }
        if (c.err == 6) { it.status = OKR_ETIMEOUT; continue; }
        if (c.err || !c.done) { it.status = OKR_EINTERNAL; continue; }
        it.status = OKR_OK;
        it.n_iter = c.t;
        it.stop_reason = c.stop_reason;
        it.n_kept = R.nbus[f] - c.t;
        it.candidates = c.candidates;
        it.smice = c.s_cur;
        it.max_error = maxerr[f];
        cand_total += c.candidates;
    }
    if (stats) {
        stats->setup_ms = ms_setup;
        stats->search_ms = ms_search;
        stats->candidates = cand_total;
        stats->config = R.config;
        stats->ctas = R.ctas;
        stats->fallbacks = fallbacks;
        stats->reserved = 0;
    }
    return OKR_OK;
}

static okr_status reduce_batch_impl(okr_ctx *ctx, int32_t nf, const okr_feeder *feeders, const okr_params *params,
                                    int32_t n_params, okr_batch_item *items, int32_t *super_of,
                                    okr_batch_stats *stats, int config) {
    if (!ctx) return OKR_EINVAL;
    if (!items) return fail(ctx, OKR_EINVAL, "batch: bad arguments");
    ctx->have_result = false;
    ctx->have_topo = false;
    BatchRun R;
    okr_status s = batch_measure(ctx, nf, feeders, params, n_params, config, R);
    if (s != OKR_OK) return s;
    if (R.total > ctx->batch_cap) {
        dev_free(ctx, ctx->batch_arena);
        ctx->batch_arena = nullptr;
        ctx->batch_cap = 0;
        CK(dev_alloc(ctx, &ctx->batch_arena, R.total));
        ctx->batch_cap = R.total;
    }
    // host block: staged inputs, then the result area and the assignments
    const size_t host_need = R.host_bytes;
    if (host_need > ctx->batch_host_cap) {
        if (ctx->batch_host) cudaFreeHost(ctx->batch_host);
        ctx->batch_host = nullptr;
        ctx->batch_host_cap = 0;
        CK(cudaMallocHost((void **)&ctx->batch_host, host_need));
        ctx->batch_host_cap = host_need;
    }
    R.base = static_cast<unsigned char *>(ctx->batch_arena);
    R.hb = ctx->batch_host;
    s = batch_fill(ctx, R, feeders);
    if (s != OKR_OK) return s;
    s = batch_enqueue(ctx, R, ctx->stream, super_of != nullptr, false);
    if (s != OKR_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    return batch_finish(ctx, R, items, super_of, stats);
}

// A batch staged once and captured as one CUDA graph (okr_batch_plan_*).
struct okr_batch_plan {
    okr_ctx *ctx = nullptr;
    BatchRun R;
    void *arena = nullptr;
    unsigned char *host = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~okr_batch_plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (arena) dev_free(ctx, arena);
        if (host) cudaFreeHost(host);
    }
};

extern "C" {

okr_status okr_reduce_batch(okr_ctx *ctx, int32_t n_feeders, const okr_feeder *feeders, const okr_params *params,
                            int32_t n_params, okr_batch_item *items, int32_t *super_of, okr_batch_stats *stats) {
    if (!ctx) return OKR_EINVAL;
    CK(cudaSetDevice(ctx->device));
    return reduce_batch_impl(ctx, n_feeders, feeders, params, n_params, items, super_of, stats, ctx->batch_config);
}

okr_status okr_set_batch_config(okr_ctx *ctx, int32_t config) {
    if (!ctx) return OKR_EINVAL;
    if (config < 0 || config > 3) return fail(ctx, OKR_EINVAL, "batch config %d outside [0, 3]", config);
    ctx->batch_config = config;
    return OKR_OK;
}

okr_status okr_batch_autotune(okr_ctx *ctx, int32_t n_feeders, const okr_feeder *feeders, const okr_params *params,
                              int32_t n_params, int32_t *config, double *search_ms) {
    if (!ctx) return OKR_EINVAL;
    CK(cudaSetDevice(ctx->device));
    std::vector<okr_batch_item> items(n_feeders > 0 ? n_feeders : 1);
    double best = 1e300;
    int best_c = ctx->batch_config;
    for (int c = 0; c < 4; ++c) {
        okr_batch_stats st{};
        double t = 1e300;
        for (int rep = 0; rep < 2; ++rep) {     // the first run warms the buffers
            okr_status s = reduce_batch_impl(ctx, n_feeders, feeders, params, n_params, items.data(), nullptr, &st, c);
            if (s != OKR_OK) return s;
            t = std::min(t, st.search_ms);
        }
        if (search_ms) search_ms[c] = t;
        if (t < best) { best = t; best_c = c; }
    }
    ctx->batch_config = best_c;
    if (config) *config = best_c;
    return OKR_OK;
}

// Shapes the incremental-engine autotuner times, in this order.
static const okr_inc_shape kIncTuneShapes[] = {
    {384, 2, 0, 0}, {384, 3, 0, 0}, {512, 2, 0, 0}, {512, 4, 0, 0}, {256, 2, 0, 0}, {256, 1, 0, 0},
    {384, 2, 128, 0}, {384, 2, 0, 1},
};
static const int kIncTuneCount = (int)(sizeof kIncTuneShapes / sizeof kIncTuneShapes[0]);

okr_status okr_inc_autotune(okr_ctx *ctx, int32_t n_feeders, const okr_feeder *feeders, const okr_params *params,
                            int32_t n_params, okr_inc_shape *best, okr_inc_shape *shapes, double *search_ms,
                            int32_t cap, int32_t *n_tried) {
    if (!ctx) return OKR_EINVAL;
    if (n_feeders < 1 || !feeders || !params || cap < 0) return fail(ctx, OKR_EINVAL, "inc autotune: bad arguments");
    if (n_params != 1 && n_params != n_feeders) return fail(ctx, OKR_EINVAL, "inc autotune: n_params must be 1 or n_feeders");
    for (int f = 0; f < n_params; ++f) {
        okr_status st = check_params(ctx, &params[f]);
        if (st != OKR_OK) return st;
        if (resolve_engine(&params[f]) != OKR_ENGINE_INCREMENTAL)
            return fail(ctx, OKR_EINVAL, "inc autotune: the parameters select the sweep engine");
    }
    CK(cudaSetDevice(ctx->device));
    const IncShape saved = ctx->inc_shape;
    std::vector<okr_batch_item> items(n_feeders);
    double best_t = 1e300;
    int best_i = -1;
    for (int i = 0; i < kIncTuneCount; ++i) {
        okr_status s = okr_set_inc_shape(ctx, &kIncTuneShapes[i]);
        double t = 1e300;
        for (int rep = 0; rep < 2 && s == OKR_OK; ++rep) {     // the first run warms the buffers
            double ms = 0.0;
            if (n_feeders == 1) {
                s = reduce_impl(ctx, &feeders[0], nullptr, nullptr, &params[0], Src::Host);
                ms = ctx->search_ms;
            } else {
                okr_batch_stats st{};
                s = reduce_batch_impl(ctx, n_feeders, feeders, params, n_params, items.data(), nullptr, &st,
                                      ctx->batch_config);
                ms = st.search_ms;
            }
            if (s == OKR_OK) t = std::min(t, ms);
        }
        if (s == OKR_EINVAL) {
            t = INFINITY;                       // this shape's record placement does not fit the workload
        } else if (s != OKR_OK) {
            ctx->inc_shape = saved;
            return s;
        }
        if (i < cap) {
            if (shapes) shapes[i] = kIncTuneShapes[i];
            if (search_ms) search_ms[i] = t;
        }
        if (t < best_t) { best_t = t; best_i = i; }
    }
    if (n_tried) *n_tried = kIncTuneCount;
    if (best_i < 0) {
        ctx->inc_shape = saved;
        return fail(ctx, OKR_EINVAL, "inc autotune: no shape ran");
    }
    okr_set_inc_shape(ctx, &kIncTuneShapes[best_i]);
    if (best) okr_get_inc_shape(ctx, best);
    return OKR_OK;
}

okr_status okr_batch_plan_create(okr_ctx *ctx, int32_t n_feeders, const okr_feeder *feeders, const okr_params *params,
                                 int32_t n_params, okr_batch_plan **plan) {
    if (!ctx || !plan) return OKR_EINVAL;
    *plan = nullptr;
    CK(cudaSetDevice(ctx->device));
    okr_batch_plan *P = new (std::nothrow) okr_batch_plan;
    if (!P) return fail(ctx, OKR_ENOMEM, "batch plan: out of host memory");
    P->ctx = ctx;
    okr_status s = batch_measure(ctx, n_feeders, feeders, params, n_params, ctx->batch_config, P->R);
    cudaError_t e = cudaSuccess;
    if (s == OKR_OK) e = dev_alloc(ctx, &P->arena, P->R.total);
    if (s == OKR_OK && e == cudaSuccess) e = cudaMallocHost((void **)&P->host, P->R.host_bytes);
    if (s == OKR_OK && e != cudaSuccess) s = fail(ctx, OKR_ENOMEM, "batch plan: %s", cudaGetErrorString(e));
    if (s == OKR_OK) {
        P->R.base = static_cast<unsigned char *>(P->arena);
        P->R.hb = P->host;
        s = batch_fill(ctx, P->R, feeders);
    }
    if (s == OKR_OK) {
        // the whole device sequence of one run, captured once (the side stream,
        // which the setup forks onto, has no earlier work left to join)
        cudaStream_t st = ctx->stream;
        e = join_side(ctx);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->side);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            s = fail(ctx, OKR_ECUDA, "batch plan capture: %s", cudaGetErrorString(e));
        } else {
            s = batch_enqueue(ctx, P->R, st, true, true);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(st, &g);
            P->graph = g;
            if (s == OKR_OK && e != cudaSuccess) s = fail(ctx, OKR_ECUDA, "batch plan capture: %s", cudaGetErrorString(e));
        }
    }
    if (s == OKR_OK) {
        e = cudaGraphInstantiate(&P->exec, P->graph, 0);
        if (e != cudaSuccess) s = fail(ctx, OKR_ECUDA, "batch plan instantiate: %s", cudaGetErrorString(e));
    }
    if (s != OKR_OK) {
        delete P;
        return s;
    }
    *plan = P;
    return OKR_OK;
}

okr_status okr_batch_plan_run(okr_batch_plan *plan, okr_batch_item *items, int32_t *super_of,
                              okr_batch_stats *stats) {
    if (!plan || !items) return OKR_EINVAL;
    okr_ctx *ctx = plan->ctx;
    CK(cudaSetDevice(ctx->device));
    ctx->have_result = false;
    ctx->have_topo = false;
    CK(cudaGraphLaunch(plan->exec, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return batch_finish(ctx, plan->R, items, super_of, stats);
}

okr_status okr_batch_plan_set_loads(okr_batch_plan *plan, int32_t feeder, const double *s_load) {
    if (!plan || !s_load || feeder < 0 || feeder >= plan->R.nf) return OKR_EINVAL;
    const int n = plan->R.nbus[feeder], L = plan->R.nscen[feeder];
    Carver chh;
    chh.base = plan->R.hb + plan->R.in_off[feeder];
    int *a; uint8_t *b; double *z, *sl;
    chh.take(a, n);
    chh.take(b, n);
    chh.take(z, 18 * (size_t)n);
    chh.take(sl, 6 * (size_t)L * n);
    std::memcpy(sl, s_load, sizeof(double) * 6 * (size_t)L * n);
    return OKR_OK;
}

void okr_batch_plan_destroy(okr_batch_plan *plan) {
    if (!plan) return;
    cudaSetDevice(plan->ctx->device);
    delete plan;
}

}  // extern "C"

extern "C" {

okr_status okr_get_summary(const okr_ctx *ctx, okr_summary *out) {
    if (!ctx || !out) return OKR_EINVAL;
    if (!ctx->have_result) return OKR_ENOTREADY;
    const Ctrl &c = ctx->last;
    out->n_bus = ctx->n;
    out->n_scen = ctx->L;
    out->n_iter = c.t;
    out->stop_reason = c.stop_reason;
    out->pf_sweeps = ctx->pf_sweeps;
    out->n_kept = ctx->n - c.t;
    out->candidates = c.candidates;
    out->smice = c.s_cur;
    double me = 0.0;
    if (c.t > 0) cudaMemcpy(&me, ctx->fb.X.dec_maxerr + (c.t - 1), sizeof me, cudaMemcpyDeviceToHost);
    out->max_error = me;
    out->launches = ctx->launches;
    out->search_ms = ctx->search_ms;
    out->sweeps = ctx->last.iters;
    out->sweep_ms = (ctx->last.profile && ctx->last_engine == OKR_ENGINE_SWEEP) ? 1e-6 * (double)ctx->last.sweep_ns : 0.0;
    out->flops = (ctx->last.profile && ctx->last_engine == OKR_ENGINE_SWEEP) ? ctx->last.sweep_flops : 0.0;
    out->kron_ms = ctx->kron_ms;
    out->scorer_fallbacks = c.scorer_fallbacks;
    out->inc_mismatches = c.inc_mismatch;
    out->engine = ctx->last_engine;
    out->pad = 0;
    out->terms = (ctx->last_engine == OKR_ENGINE_INCREMENTAL && c.profile) ? (int64_t)c.sweep_ns : 0;
    out->rechecks = ctx->last.rechecks;
    out->recheck_cands = ctx->last.recheck_cands;
    for (int i = 0; i < 16; ++i) out->phase_ms[i] = ctx->last.profile ? 1e-6 * (double)ctx->last.phase_ns[i] : 0.0;
    const bool inc = ctx->last_engine == OKR_ENGINE_INCREMENTAL && ctx->last_rec >= 0;
    out->inc_threads = inc ? ctx->last_shape.threads : 0;
    out->inc_eval_warps = inc ? ctx->last_shape.cw : 0;
    out->inc_shared_entries = inc ? ctx->last_shape.se : 0;
    out->inc_records = inc ? ctx->last_rec + 1 : 0;
    out->pruned = ctx->last_engine == OKR_ENGINE_SWEEP ? c.pruned : 0;
    return OKR_OK;
}

okr_status okr_set_inc_shape(okr_ctx *ctx, const okr_inc_shape *shape) {
    if (!ctx) return OKR_EINVAL;
    if (!shape) {
        ctx->inc_shape = IncShape{0, 0, 0, -1};
        return OKR_OK;
    }
    const int t = shape->threads, w = shape->eval_warps, e = shape->shared_entries, r = shape->records;
    if (t != 0 && t != 256 && t != 384 && t != 512)
        return fail(ctx, OKR_EINVAL, "inc shape: threads %d (0, 256, 384 or 512)", t);
    const int nw = (t == 0 ? kIncDefaultThreads : t) / 32;
    if (w < 0 || w > nw - 1) return fail(ctx, OKR_EINVAL, "inc shape: eval_warps %d outside [0, %d]", w, nw - 1);
    if (e < 0 || e > 256) return fail(ctx, OKR_EINVAL, "inc shape: shared_entries %d outside [0, 256]", e);
    if (r < 0 || r > 3) return fail(ctx, OKR_EINVAL, "inc shape: records %d outside [0, 3]", r);
    ctx->inc_shape = IncShape{t, w, e, r - 1};
    return OKR_OK;
}

okr_status okr_get_inc_shape(const okr_ctx *ctx, okr_inc_shape *shape) {
    if (!ctx || !shape) return OKR_EINVAL;
    const IncShape sh = inc_shape_resolve(ctx->inc_shape);
    shape->threads = sh.threads;
    shape->eval_warps = sh.cw;
    shape->shared_entries = sh.se;
    shape->records = sh.rec + 1;
    return OKR_OK;
}

okr_status okr_get_decisions(const okr_ctx *ctx, int32_t cap, int32_t *s, int32_t *r, double *smice,
                             double *max_error, double *gap, int32_t *ncand) {
    if (!ctx || cap < 0) return OKR_EINVAL;
    if (!ctx->have_result) return OKR_ENOTREADY;
    const int t = ctx->last.t < cap ? ctx->last.t : cap;
    if (t == 0) return OKR_OK;
    const Search &X = ctx->fb.X;
    if (s && cudaMemcpy(s, X.dec_s, sizeof(int) * t, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    if (r && cudaMemcpy(r, X.dec_r, sizeof(int) * t, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    // objective 1 scores a network by its largest error, which is max_error
    const double *score = ctx->last.objective == 1 ? X.dec_maxerr : X.dec_score;
    if (smice && cudaMemcpy(smice, score, sizeof(double) * t, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    if (max_error && cudaMemcpy(max_error, X.dec_maxerr, sizeof(double) * t, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    if (gap && cudaMemcpy(gap, X.dec_gap, sizeof(double) * t, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    if (ncand && cudaMemcpy(ncand, X.dec_ncand, sizeof(int) * t, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    return OKR_OK;
}

okr_status okr_get_assignment(const okr_ctx *ctx, int32_t *super_of) {
    if (!ctx || !super_of) return OKR_EINVAL;
    if (!ctx->have_result) return OKR_ENOTREADY;
    if (cudaMemcpy(super_of, ctx->fb.super_out, sizeof(int) * ctx->n, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    return OKR_OK;
}

okr_status okr_get_voltages(const okr_ctx *ctx, double *vhat, double *vred) {
    if (!ctx) return OKR_EINVAL;
    if (!ctx->have_result) return OKR_ENOTREADY;
    const size_t bytes = sizeof(double) * 6 * ctx->L * ctx->n;
    if (vhat && cudaMemcpy(vhat, ctx->fb.vhat_out, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    if (vred && cudaMemcpy(vred, ctx->fb.vred_out, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    return OKR_OK;
}

}  // extern "C"

// A reduction's results copied out of its context (host memory, owned by the
// object): later calls on the context leave them alone.
struct okr_result {
    int n = 0, L = 0, t = 0, k_phi = -1;   // k_phi < 0: Y_Kron not taken
    okr_summary summary{};
    std::vector<int32_t> super_of, dec_s, dec_r, dec_ncand, phase_node;
    std::vector<double> dec_score, dec_maxerr, dec_gap, vhat, vred, ykron;
};

extern "C" {

okr_status okr_result_take(okr_ctx *ctx, int32_t with_ykron, okr_result **out) {
    if (!ctx || !out) return OKR_EINVAL;
    *out = nullptr;
    if (!ctx->have_result) return fail(ctx, OKR_ENOTREADY, "no reduction to take results from");
    okr_result *R = new (std::nothrow) okr_result;
    if (!R) return fail(ctx, OKR_ENOMEM, "result: out of host memory");
    okr_status s = OKR_OK;
    try {
        s = okr_get_summary(ctx, &R->summary);
        R->n = ctx->n;
        R->L = ctx->L;
        R->t = ctx->last.t;
        const size_t t = R->t > 0 ? (size_t)R->t : 1, nv = (size_t)6 * R->L * R->n;
        R->super_of.assign(R->n, 0);
        R->dec_s.assign(t, 0);
        R->dec_r.assign(t, 0);
        R->dec_ncand.assign(t, 0);
        R->dec_score.assign(t, 0.0);
        R->dec_maxerr.assign(t, 0.0);
        R->dec_gap.assign(t, 0.0);
        R->vhat.assign(nv, 0.0);
        R->vred.assign(nv, 0.0);
        if (s == OKR_OK) s = okr_get_assignment(ctx, R->super_of.data());
        if (s == OKR_OK)
            s = okr_get_decisions(ctx, R->t, R->dec_s.data(), R->dec_r.data(), R->dec_score.data(),
                                  R->dec_maxerr.data(), R->dec_gap.data(), R->dec_ncand.data());
        if (s == OKR_OK) s = okr_get_voltages(ctx, R->vhat.data(), R->vred.data());
        if (s == OKR_OK && with_ykron) {
            int32_t k = 0;
            s = okr_kron(ctx, nullptr, 0, nullptr, nullptr, &k);
            if (s == OKR_OK) {
                R->ykron.assign((size_t)2 * k * k, 0.0);
                R->phase_node.assign(k > 0 ? k : 1, 0);
                s = okr_kron(ctx, nullptr, k, R->ykron.data(), R->phase_node.data(), &k);
                R->k_phi = k;
                R->summary.kron_ms = ctx->kron_ms;
            }
        }
    } catch (const std::bad_alloc &) {
        s = fail(ctx, OKR_ENOMEM, "result: out of host memory");
    }
    if (s != OKR_OK) {
        delete R;
        return s;
    }
    *out = R;
    return OKR_OK;
}

void okr_result_free(okr_result *res) { delete res; }

okr_status okr_result_summary(const okr_result *res, okr_summary *out) {
    if (!res || !out) return OKR_EINVAL;
    *out = res->summary;
    return OKR_OK;
}

okr_status okr_result_assignment(const okr_result *res, int32_t *super_of, int32_t *n_bus, int32_t *n_kept) {
    if (!res) return OKR_EINVAL;
    if (n_bus) *n_bus = res->n;
    if (n_kept) *n_kept = res->n - res->t;
    if (super_of) std::memcpy(super_of, res->super_of.data(), sizeof(int32_t) * res->n);
    return OKR_OK;
}

okr_status okr_result_decisions(const okr_result *res, int32_t cap, int32_t *s, int32_t *r, double *smice,
                                double *max_error, double *gap, int32_t *ncand, int32_t *count) {
    if (!res || cap < 0) return OKR_EINVAL;
    if (count) *count = res->t;
    const size_t k = (size_t)(res->t < cap ? res->t : cap);
    if (k == 0) return OKR_OK;
    if (s) std::memcpy(s, res->dec_s.data(), sizeof(int32_t) * k);
    if (r) std::memcpy(r, res->dec_r.data(), sizeof(int32_t) * k);
    if (smice) std::memcpy(smice, res->dec_score.data(), sizeof(double) * k);
    if (max_error) std::memcpy(max_error, res->dec_maxerr.data(), sizeof(double) * k);
    if (gap) std::memcpy(gap, res->dec_gap.data(), sizeof(double) * k);
    if (ncand) std::memcpy(ncand, res->dec_ncand.data(), sizeof(int32_t) * k);
    return OKR_OK;
}

okr_status okr_result_errors(const okr_result *res, double *max_error, double *smice, double *vhat, double *vred,
                             int32_t *n_scen, int32_t *n_bus) {
    if (!res) return OKR_EINVAL;
    if (max_error) *max_error = res->summary.max_error;
    if (smice) *smice = res->summary.smice;
    if (n_scen) *n_scen = res->L;
    if (n_bus) *n_bus = res->n;
    const size_t nv = (size_t)6 * res->L * res->n;
    if (vhat) std::memcpy(vhat, res->vhat.data(), sizeof(double) * nv);
    if (vred) std::memcpy(vred, res->vred.data(), sizeof(double) * nv);
    return OKR_OK;
}

okr_status okr_result_ykron(const okr_result *res, int32_t cap, double *y, int32_t *phase_node, int32_t *k_phi) {
    if (!res || !k_phi) return OKR_EINVAL;
    if (res->k_phi < 0) return OKR_ENOTREADY;
    *k_phi = res->k_phi;
    if (!y && !phase_node) return OKR_OK;
    if (cap < res->k_phi) return OKR_EINVAL;
    const size_t K = res->k_phi;
    if (y && K) std::memcpy(y, res->ykron.data(), sizeof(double) * 2 * K * K);
    if (phase_node && K) std::memcpy(phase_node, res->phase_node.data(), sizeof(int32_t) * K);
    return OKR_OK;
}

okr_status okr_result_stats(const okr_result *res, int64_t *candidates, int32_t *iterations, double *seconds) {
    if (!res) return OKR_EINVAL;
    if (candidates) *candidates = res->summary.candidates;
    if (iterations) *iterations = res->summary.n_iter;
    if (seconds) *seconds = 1e-3 * res->summary.search_ms;
    return OKR_OK;
}

okr_status okr_get_recorded_features(const okr_ctx *ctx, int32_t iter, int32_t cap, float *features, int32_t *count) {
    if (!ctx || !count || cap < 0) return OKR_EINVAL;
    if (!ctx->have_result) return OKR_ENOTREADY;
    if (iter < 0 || iter >= ctx->rec_iters) return OKR_EINVAL;
    int c = 0;
    if (cudaMemcpy(&c, ctx->fb.X.rec_count + iter, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    *count = c;
    const int k = c < cap ? c : cap;
    const size_t off = (size_t)iter * 2 * ctx->n * kScorerFeatures;
    if (k > 0 && features &&
        cudaMemcpy(features, ctx->fb.X.rec_feat + off, sizeof(float) * k * kScorerFeatures, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return OKR_ECUDA;
    return OKR_OK;
}

okr_status okr_get_recorded(const okr_ctx *ctx, int32_t iter, int32_t cap, int32_t *s, int32_t *r, double *smice,
                            double *bound, int32_t *count) {
    if (!ctx || !count || cap < 0) return OKR_EINVAL;
    if (!ctx->have_result) return OKR_ENOTREADY;
    if (iter < 0 || iter >= ctx->rec_iters) return OKR_EINVAL;
    int c = 0;
    if (cudaMemcpy(&c, ctx->fb.X.rec_count + iter, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    *count = c;
    const int k = c < cap ? c : cap;
    const size_t off = (size_t)iter * 2 * ctx->n;
    if (k > 0) {
        if (s && cudaMemcpy(s, ctx->fb.X.rec_s + off, sizeof(int) * k, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
        if (r && cudaMemcpy(r, ctx->fb.X.rec_r + off, sizeof(int) * k, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
        if (smice && cudaMemcpy(smice, ctx->fb.X.rec_score + off, sizeof(double) * k, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
        if (bound && cudaMemcpy(bound, ctx->fb.X.rec_bound + off, sizeof(double) * k, cudaMemcpyDeviceToHost) != cudaSuccess) return OKR_ECUDA;
    }
    return OKR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- learned scorer
namespace {

template <typename T>
cudaError_t grab(okr_ctx *ctx, std::vector<void *> &list, T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = dev_alloc(ctx, &q, sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) { list.push_back(q); *p = static_cast<T *>(q); }
    return e;
}

okr_status mlp_ensure_work(okr_ctx *ctx, int N) {
    if (N <= ctx->mw.cap) return OKR_OK;
    free_list(ctx, ctx->mlp_work_allocs);
    ctx->mw = MlpWork{};
    MlpWork &w = ctx->mw;
    const size_t NH = (size_t)N * kMlpHidden;
    CK(grab(ctx, ctx->mlp_work_allocs, &w.h1, NH));
    CK(grab(ctx, ctx->mlp_work_allocs, &w.h2, NH));
    CK(grab(ctx, ctx->mlp_work_allocs, &w.h3, NH));
    CK(grab(ctx, ctx->mlp_work_allocs, &w.d1, NH));
    CK(grab(ctx, ctx->mlp_work_allocs, &w.d2, NH));
    CK(grab(ctx, ctx->mlp_work_allocs, &w.d3, NH));
    CK(grab(ctx, ctx->mlp_work_allocs, &w.y, (size_t)N));
    CK(grab(ctx, ctx->mlp_work_allocs, &w.dy, (size_t)N));
    CK(grab(ctx, ctx->mlp_work_allocs, &w.part, (size_t)mlp_segments(N) * (kMlpHidden + 1) * kMlpHidden));
    w.cap = N;
    return OKR_OK;
}

okr_status mlp_upload(okr_ctx *ctx, const float *x, const float *t, long long N) {
    const int F = ctx->mb.F;
    if (N > ctx->mlp_data_cap) {
        free_list(ctx, ctx->mlp_data_allocs);
        ctx->mlp_data_cap = 0;
        CK(grab(ctx, ctx->mlp_data_allocs, &ctx->mlp_x, (size_t)N * F));
        CK(grab(ctx, ctx->mlp_data_allocs, &ctx->mlp_t, (size_t)N));
        ctx->mlp_data_cap = N;
    }
    CK(cudaMemcpyAsync(ctx->mlp_x, x, sizeof(float) * (size_t)N * F, cudaMemcpyHostToDevice, ctx->stream));
    if (t) CK(cudaMemcpyAsync(ctx->mlp_t, t, sizeof(float) * (size_t)N, cudaMemcpyHostToDevice, ctx->stream));
    return OKR_OK;
}

okr_status mlp_batch_loss(okr_ctx *ctx, const float *y, const float *t, int N, double *sum) {
    const int nseg = mlp_segments(N);
    CK(mlp_sqerr(y, t, N, ctx->mw.part, ctx->stream));
    std::vector<float> part(nseg);
    CK(cudaMemcpyAsync(part.data(), ctx->mw.part, sizeof(float) * nseg, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double acc = 0.0;
    for (float v : part) acc += v;
    *sum = acc;
    return OKR_OK;
}

}  // namespace

extern "C" {

okr_status okr_scorer_init(okr_ctx *ctx, int32_t n_features, const float *theta) {
    if (!ctx) return OKR_EINVAL;
    if (n_features < 1 || n_features > kMlpMaxF) return fail(ctx, OKR_EINVAL, "n_features %d outside [1, %d]", n_features, kMlpMaxF);
    CK(cudaSetDevice(ctx->device));
    free_mlp(ctx);
    MlpBufs &b = ctx->mb;
    b.F = n_features;
    const int P = mlp_param_count(n_features);
    CK(grab(ctx, ctx->mlp_allocs, &b.theta, (size_t)P));
    CK(grab(ctx, ctx->mlp_allocs, &b.grad, (size_t)P));
    CK(grab(ctx, ctx->mlp_allocs, &b.m, (size_t)P));
    CK(grab(ctx, ctx->mlp_allocs, &b.v, (size_t)P));
    CK(grab(ctx, ctx->mlp_allocs, &b.w1, (size_t)kMlpMaxF * kMlpHidden));
    CK(grab(ctx, ctx->mlp_allocs, &b.w2, (size_t)kMlpHidden * kMlpHidden));
    CK(grab(ctx, ctx->mlp_allocs, &b.w3, (size_t)kMlpHidden * kMlpHidden));
    CK(grab(ctx, ctx->mlp_allocs, &b.w4, (size_t)kMlpHidden));
    cudaStream_t st = ctx->stream;
    if (theta) CK(cudaMemcpyAsync(b.theta, theta, sizeof(float) * P, cudaMemcpyHostToDevice, st));
    else CK(cudaMemsetAsync(b.theta, 0, sizeof(float) * P, st));
    CK(cudaMemsetAsync(b.m, 0, sizeof(float) * P, st));
    CK(cudaMemsetAsync(b.v, 0, sizeof(float) * P, st));
    CK(cudaMemsetAsync(b.grad, 0, sizeof(float) * P, st));
    CK(mlp_sync_bf16(b, st));
    CK(cudaStreamSynchronize(st));
    ctx->mlp_step = 0;
    return OKR_OK;
}

okr_status okr_scorer_params(okr_ctx *ctx, float *theta, int32_t *n_params) {
    if (!ctx || !n_params) return OKR_EINVAL;
    if (!ctx->mb.theta) return fail(ctx, OKR_ENOTREADY, "scorer not initialised");
    const int P = mlp_param_count(ctx->mb.F);
    *n_params = P;
    if (theta) CK(cudaMemcpy(theta, ctx->mb.theta, sizeof(float) * P, cudaMemcpyDeviceToHost));
    return OKR_OK;
}

okr_status okr_scorer_gradient(okr_ctx *ctx, const float *x, const float *t, int32_t n, float *grad, double *loss) {
    if (!ctx || !x || !t || n < 1) return OKR_EINVAL;
    if (!ctx->mb.theta) return fail(ctx, OKR_ENOTREADY, "scorer not initialised");
    CK(cudaSetDevice(ctx->device));
    okr_status s = mlp_ensure_work(ctx, n);
    if (s == OKR_OK) s = mlp_upload(ctx, x, t, n);
    if (s != OKR_OK) return s;
    CK(mlp_gradient(ctx->mb, ctx->mw, ctx->mlp_x, ctx->mlp_t, n, ctx->num_sms, ctx->stream));
    double sum = 0.0;
    s = mlp_batch_loss(ctx, ctx->mw.y, ctx->mlp_t, n, &sum);
    if (s != OKR_OK) return s;
    if (loss) *loss = sum / n;
    const int P = mlp_param_count(ctx->mb.F);
    if (grad) CK(cudaMemcpy(grad, ctx->mb.grad, sizeof(float) * P, cudaMemcpyDeviceToHost));
    return OKR_OK;
}

okr_status okr_scorer_train(okr_ctx *ctx, const float *x, const float *t, int64_t n, int32_t batch, int32_t epochs,
                            float lr, double *epoch_loss) {
    if (!ctx || !x || !t || n < 1 || batch < 1 || epochs < 0 || !(lr > 0.0f)) return OKR_EINVAL;
    if (!ctx->mb.theta) return fail(ctx, OKR_ENOTREADY, "scorer not initialised");
    CK(cudaSetDevice(ctx->device));
    const int B = (int)std::min<int64_t>(batch, n);
    okr_status s = mlp_ensure_work(ctx, B);
    if (s == OKR_OK) s = mlp_upload(ctx, x, t, n);
    if (s != OKR_OK) return s;
    const int F = ctx->mb.F;
    for (int e = 0; e < epochs; ++e) {
        double sum = 0.0;
        for (int64_t b0 = 0; b0 < n; b0 += B) {
            const int nb = (int)std::min<int64_t>(B, n - b0);
            const float *xb = ctx->mlp_x + (size_t)b0 * F;
            const float *tb = ctx->mlp_t + b0;
            CK(mlp_gradient(ctx->mb, ctx->mw, xb, tb, nb, ctx->num_sms, ctx->stream));
            double bs = 0.0;
            s = mlp_batch_loss(ctx, ctx->mw.y, tb, nb, &bs);
            if (s != OKR_OK) return s;
            sum += bs;
            CK(mlp_adam(ctx->mb, lr, ++ctx->mlp_step, ctx->stream));
        }
        if (epoch_loss) epoch_loss[e] = sum / (double)n;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return OKR_OK;
}

okr_status okr_scorer_predict_tc(okr_ctx *ctx, const float *x, int64_t n, float *y) {
    if (!ctx || !x || !y || n < 1) return OKR_EINVAL;
    if (!ctx->mb.theta) return fail(ctx, OKR_ENOTREADY, "scorer not initialised");
    if (n > INT32_MAX) return fail(ctx, OKR_EINVAL, "too many samples");
    CK(cudaSetDevice(ctx->device));
    okr_status s = mlp_upload(ctx, x, nullptr, n);
    if (s != OKR_OK) return s;
    float *yd = ctx->mlp_t;                     // the targets' buffer holds the predictions
    if (!ctx->mlp_err) CK(dev_alloc(ctx, (void **)&ctx->mlp_err, sizeof(int)));
    int *err = ctx->mlp_err;
    okr_status out = OKR_OK;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = mlp_forward_tc(ctx->mb, ctx->mlp_x, (int)n, yd, err, ctx->num_sms, ctx->stream);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, yd, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) out = fail(ctx, OKR_ECUDA, "tensor-core inference: %s", cudaGetErrorString(e));
    else if (herr) out = fail(ctx, OKR_ETIMEOUT, "tensor-core inference: a wait for the products gave up");
    return out;
}

okr_status okr_scorer_predict(okr_ctx *ctx, const float *x, int64_t n, float *y) {
    if (!ctx || !x || !y || n < 1) return OKR_EINVAL;
    if (!ctx->mb.theta) return fail(ctx, OKR_ENOTREADY, "scorer not initialised");
    if (n > INT32_MAX) return fail(ctx, OKR_EINVAL, "too many samples");
    CK(cudaSetDevice(ctx->device));
    okr_status s = mlp_upload(ctx, x, nullptr, n);
    if (s != OKR_OK) return s;
    float *yd = ctx->mlp_t;                     // the targets' buffer holds the predictions
    CK(mlp_forward(ctx->mb, ctx->mlp_x, (int)n, nullptr, nullptr, nullptr, yd, ctx->num_sms, ctx->stream));
    CK(cudaMemcpyAsync(y, yd, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return OKR_OK;
}

}  // extern "C"
