// okr_kernels.cuh -- kernel declarations shared between translation units.
#pragma once

#include "okr_internal.cuh"

#include <cuda_bf16.h>

namespace okr {

// okr_setup.cu
__global__ void __launch_bounds__(1024) k_topology(int n, const int *__restrict__ parent_in, const uint8_t *__restrict__ ph_in,
                           Topo T, int *dep, int *anc, int *anc2, int *d2, int *size, int *ccount,
                           int *coff_c, int *child_c, int *err);
__global__ void __launch_bounds__(1024) k_child_offsets(int n, Topo T, const int *__restrict__ coff_c, const int *__restrict__ child_c);
__global__ void k_rmq_level(int n, int j, const int *__restrict__ depth, uint16_t *st);
__global__ void __launch_bounds__(1024) k_rmq_all(int n, int nlev, const int *__restrict__ depth, uint16_t *st);
__global__ void k_lca_fill(int n, const int *__restrict__ parent, const int *__restrict__ sz,
                           const int *__restrict__ depth, const uint16_t *__restrict__ st, uint16_t *lca);
// line inverses (grid) and path impedances (one CTA)
cudaError_t launch_lines(int n, Topo T, const double *z_in, int *err, int num_sms, cudaStream_t st);
cudaError_t launch_line_inverses(int n, Topo T, const double *z_in, int *err, int num_sms, cudaStream_t st);
cudaError_t launch_path_impedance(int n, Topo T, cudaStream_t st);
// load flow of every scenario (cooperative launch).  J: [L*3n] line currents,
// W: [L*3n] work (its contents are overwritten), red: [3L+1] doubles of
// reduction slots and barrier counter (cleared by the launch), iters: [L].
// Each grid barrier polls at most max_spins times (> 0), then sets err = 6.
cudaError_t launch_power_flow(int n, int L, Topo T, const double *s_in, double tol, int max_iter, double2 *J,
                              double2 *W, double *red, int *iters, int *err, int num_sms, cudaStream_t st,
                              long long max_spins);
__global__ void k_line_currents(int n, int L, Topo T, double2 *J);
__global__ void k_injections(int n, int L, Topo T, const double2 *__restrict__ J);
__global__ void k_import_ops(int n, int L, Topo T, const double *__restrict__ vh, const double *__restrict__ ih);
__global__ void k_state_init(int n, int L, Topo T, State S);

// Per-feeder setup descriptor of a batch (every pointer into that feeder's buffers).
struct BatchSetup {
    int n, L, nlev;
    const int *parent_in;
    const uint8_t *ph_in;
    const double *z_in, *s_in;
    Topo T;
    State S;
    int *dep, *anc, *anc2, *d2, *size, *ccount, *coff_c, *child_c;
    uint16_t *rmq;
    double2 *J;
    int *pf_iters;
    int *err;                   // setup error of this feeder (0 = none)
    double *dec_maxerr, *mrank, *bmax;
    int *arrive;
};
// Setup of many feeders in four launches (CTA per feeder, per feeder x scenario):
// the LCA tables run on `side` (forked from st after the per-feeder prep by
// ev_fork, joined back into st by ev_join before the call returns), the load
// flows on st.
cudaError_t launch_batch_setup(int nf, int max_L, long long max_nn, const BatchSetup *bs, double tol, int max_iter,
                               int num_sms, cudaStream_t st, cudaStream_t side, cudaEvent_t ev_fork,
                               cudaEvent_t ev_join);

// The reduced network of a caller assignment (one CTA per scenario).
__global__ void __launch_bounds__(1024) k_eval_reduced(Topo T, const int *__restrict__ sup, const int *__restrict__ moff,
                                                      const int *__restrict__ mem, double2 *W, double2 *V, double *vred,
                                                      double *err);

// okr_kron.cu
constexpr int kKronShared = 64;     // groups up to this many phase-nodes are inverted in shared memory
constexpr int kKronMaxGroup = 1024; // larger groups are refused (dense inverse per group)
struct KronHdr {
    int n_groups, k_phi, max_d, err;
    long long big_total;            // double2 elements of global scratch for large groups
};
// Work arrays of the Y_Kron build (preorder ids unless noted).
struct KronWork {
    uint8_t *keptp;                 // [n] kept flag
    int *g;                         // [n] component top of a reduced bus
    int *key;                       // [n] group key of a kept non-root bus
    int *cnt, *dsum, *fill, *goff;  // [n] per key: ports, phase-nodes, fill counter, port offset
    int *ports;                     // [n] ports grouped by key
    int *out_off;                   // [n+1] output row offset per CALLER bus id
    int *pn;                        // [3n] output row -> caller bus * 3 + phase
    int *gkey, *gp, *gd;            // [n] per group: key, reference bus p, phase-nodes d
    int *gport, *grow;              // [n+1] per group: first port, first row
    int *rows;                      // [3n] per group rows: preorder bus * 4 + phase
    long long *gbig;                // [n] per group offset into the global scratch
    KronHdr *hdr;
};
__global__ void __launch_bounds__(1024) k_kron_groups(Topo T, const int *label, const uint8_t *kept_in, KronWork W);
__global__ void k_kron_diag(KronWork W, double2 *Y, int K);
__global__ void __launch_bounds__(1024) k_radial_critical(Topo T, const int *label, const uint8_t *kept_in, KronWork W,
                                                          uint8_t *crit, int *count);
cudaError_t launch_kron_solve(int n_groups, Topo T, KronWork W, double2 *big, double2 *Y, int K, cudaStream_t st);

// okr_mlp.cu -- the learned candidate scorer
constexpr int kMlpHidden = 128;     // units per hidden layer
constexpr int kMlpMaxF = 16;        // longest feature vector
struct MlpBufs {
    int F = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // FP32 [P]
    __nv_bfloat16 *w1 = nullptr, *w2 = nullptr, *w3 = nullptr, *w4 = nullptr;  // bf16 copies
};
struct MlpWork {
    int cap = 0;                    // samples the buffers hold
    float *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *d1 = nullptr, *d2 = nullptr, *d3 = nullptr;  // [cap][H]
    float *y = nullptr, *dy = nullptr;                                   // [cap]
    float *part = nullptr;                                               // [segments][(H+1) x H]
};
int mlp_param_count(int F);
int mlp_segments(int N);
cudaError_t mlp_sync_bf16(const MlpBufs &b, cudaStream_t st);
cudaError_t mlp_forward(const MlpBufs &b, const float *x, int N, float *h1, float *h2, float *h3, float *y, int num_sms,
                        cudaStream_t st);
cudaError_t mlp_gradient(const MlpBufs &b, const MlpWork &w, const float *x, const float *t, int N, int num_sms,
                         cudaStream_t st);
cudaError_t mlp_adam(const MlpBufs &b, float lr, int step, cudaStream_t st);
cudaError_t mlp_sqerr(const float *y, const float *t, int N, float *part, cudaStream_t st);
// okr_mlp_tc.cu: inference on the tensor cores (bfloat16 operands, FP32
// accumulators in tensor memory); *err (device) is set to 1 when a wait gave up.
cudaError_t mlp_forward_tc(const MlpBufs &b, const float *x, int N, float *y, int *err, int num_sms, cudaStream_t st);

// okr_persist.cu
// One feeder of a batched search launch.
struct BatchFeeder {
    Topo T;
    State S;
    Search X;
    Inc I;
    Ctrl *C;
    int *setup_err;             // nonzero: the setup failed, the search is skipped
    int *super_out;             // [n] assignment in caller numbering
    double *max_err;            // largest per-phase error of the final network
};
// Per-team state of a batched search: the team's barrier, its control block
// (spin limit, error flag) and the queue slot its leader fetched.
struct BatchTeam {
    GridBar bar;
    Ctrl ctrl;
    int slot;
    int pad;
};
// Batched search with teams of `team` CTAs (cooperative launch of `grid` CTAs,
// a multiple of `team`).
cudaError_t launch_search_batch(int precision, int team, int grid, const BatchFeeder *fd, const int *order, int nf,
                                int *queue, BatchTeam *teams, cudaStream_t st);
int search_batch_blocks_per_sm(int precision);
cudaError_t launch_search(int precision, int grid, Topo T, State S, Search X, Ctrl *C, GridBar *gb, cudaStream_t st);
int search_blocks_per_sm();     // CTAs of the search kernel that fit one SM (0 on error)
__global__ void k_export(Topo T, State S, double *super_vred, int *super_of, double *vhat_out);

// okr_incr.cu -- the search with scores carried across iterations: one CTA per
// feeder (verify = 1: every merge also re-evaluates every candidate and counts
// mismatches of the carried scores in C->inc_mismatch).
//
// Launch shape of that CTA: threads (256, 384 or 512), warps that evaluate the
// merge beside the changed-set scan (cw, 1 .. threads/32 - 1), work entries in
// shared memory (se, 1 .. 256; the rest in device memory) and where the
// selection records live (rec: -1 automatic, 0 device memory, 1 shared memory,
// 2 shared memory with the largest MICE per super-node; batches take 0 or 1).
// Every shape gives the same results.
struct IncShape {
    int threads, cw, se, rec;
};
constexpr int kIncDefaultThreads = 384;
constexpr int kIncInitPairs = 8;        // slot pairs per CTA of one feeder's first evaluation (at most all SMs)
constexpr int kIncInitCtasMax = 256;    // CTAs of one feeder's first evaluation, at most
constexpr int kIncInitBatchBuses = 64;  // buses per CTA of a batch's first evaluation
// CTAs of one feeder's first evaluation in a batch (its positions split
// evenly over them; the work buffer holds 2n + kIncInitCtasMax entries).
inline int inc_init_batch_ctas(int n) {
    const int c = (n + kIncInitBatchBuses - 1) / kIncInitBatchBuses;
    return c < 1 ? 1 : (c > kIncInitCtasMax ? kIncInitCtasMax : c);
}
// Out-of-range fields replaced by the defaults (384 threads, 2 evaluation
// warps (4 with 512 threads), 256 shared entries, automatic records).
IncShape inc_shape_resolve(IncShape sh);
// Dynamic shared memory and record placement of one search; false when a
// forced placement does not fit.
bool inc_smem(int n, bool maxm, const IncShape &sh, int *rec_mode, size_t *bytes);
// cudaErrorInvalidValue when the shape's forced record placement does not fit;
// *rec_used (may be NULL): the placement that ran.
cudaError_t launch_search_inc(int precision, Topo T, State S, Search X, Inc I, Ctrl *C, int verify, IncShape sh,
                              int *rec_used, cudaStream_t st);
// Many feeders: one CTA each, in the order given (prepare_search_inc_batch with
// the same precision, shape and at least the same largest feeder first: it
// sets the kernel's shared-memory attribute, which a stream capture must not
// see).
cudaError_t prepare_search_inc_batch(int precision, int max_n, IncShape sh);
cudaError_t launch_search_inc_batch(int precision, int max_n, const BatchFeeder *fd, const int *order, int nf,
                                    IncShape sh, cudaStream_t st);
// The batch's first evaluation on many CTAs, before launch_search_inc_batch
// (which then takes it as done): cta_off[i] = the first CTA of order[i]
// (inc_init_batch_ctas(n) each), ctas = their total; it first zeroes the
// feeders' carried sums.  prepare_inc_init_batch sets the kernel's
// shared-memory attribute (before any stream capture).
cudaError_t prepare_inc_init_batch(int precision, int max_n);
cudaError_t launch_inc_init_batch(int precision, int max_n, const BatchFeeder *fd, const int *order,
                                  const int *cta_off, int nf, int ctas, cudaStream_t st);

}  // namespace okr
