// okr_internal.cuh -- device data layout and small helpers shared by the
// library's translation units (not part of the public C ABI).
//
// Numbering.  The caller's buses (bus 0 = slack, parent[i] < i) are renumbered
// in depth-first preorder, children visited in increasing caller id.  In this
// numbering every subtree is the contiguous range [v, v + sz[v]).
//
// Per-bus three-phase quantities are stored structure-of-arrays with the bus
// index fastest: x[(l * 3 + p) * n + k] for scenario l, phase p, bus k, so that
// a warp reading 32 consecutive buses issues coalesced loads.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace okr {

constexpr int kChunk = 32;          // candidate positions per warp work item
constexpr int kMaxScen = 4;         // scenarios held in registers by the sweep
constexpr int kMaxBus = 32768;      // LCA table uses 16-bit entries
constexpr int kScorerFeatures = 14; // features of one candidate for the learned scorer

// ---------------------------------------------------------------- complex helpers
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double cmag(double2 a) {
    // |v| = sqrt(re*re + im*im), products rounded separately (no contraction).
    return sqrt(__dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)));
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// Load current of a constant-power load s at voltage v, conj(s / v), as
// conj(s) v / |v|^2 with one reciprocal.  Every operation is explicitly
// rounded, so the single-feeder and the batched load flows, which both call
// it, give the same bits.
__device__ __forceinline__ double2 load_current(double2 s, double2 v) {
    const double inv = __drcp_rn(__fma_rn(v.x, v.x, __dmul_rn(v.y, v.y)));
    return make_double2(__dmul_rn(__fma_rn(s.x, v.x, __dmul_rn(s.y, v.y)), inv),
                        __dmul_rn(__fma_rn(s.x, v.y, -__dmul_rn(s.y, v.x)), inv));
}
// |a|^2, explicitly rounded (the load flows' convergence test compares the
// largest squared voltage change with tol^2: no square root per element).
__device__ __forceinline__ double cmag2(double2 a) { return __fma_rn(a.x, a.x, __dmul_rn(a.y, a.y)); }

// (32-bit arithmetic: L * 3 * n < 2^31 for every feeder the library accepts)
__host__ __device__ __forceinline__ size_t sidx(int l, int p, int k, int n) { return (size_t)(unsigned)((l * 3 + p) * n + k); }

// ---------------------------------------------------------------- device structures
// Static description of one feeder (preorder numbering), built once per call.
struct Topo {
    int n, L;
    int *maxd;          // [2] deepest level, sum of subtree sizes (written on the device)
    int *parent;        // [n], parent[0] = -1
    int *orig;          // [n] preorder -> caller id
    int *pre;           // [n] caller id -> preorder
    int *sz;            // [n] subtree size
    int *depth;         // [n]
    int *child_off;     // [n+1] children (preorder ids, increasing)
    int *child;         // [n]
    int *level_off;     // [max_depth+2] buses grouped by depth
    int *level_bus;     // [n]
    uint8_t *ph;        // [n] phase masks
    uint16_t *lca;      // [n*n] lowest common ancestor (preorder ids)
    double2 *zl;        // [n*9] line impedance parent(k)->k, row-major 3x3
    double2 *yl;        // [n*9] line admittance on the phases of k
    double2 *zc;        // [n*9] path impedance root->k
    float2 *zh, *zlo;   // [n*9] zc split into two floats: zc ~ zh + zlo
    double2 *vhat;      // [L*3*n] scenario voltages
    double2 *ihat;      // [L*3*n] scenario injections, Y vhat
    double *amag;       // [L*3*n] |vhat|
    double2 *vslack;    // [3]
};

// One candidate (s, r) of the current iteration, in a compact list.  Its work
// positions are the super-nodes of the two affected preorder ranges, listed in
// the compact super-node order (s side first, then r side), plus one position
// for the merged cluster of s when s is the common ancestor (its voltage does
// not move, only its cluster grows).
struct Cand {
    int s, r, a;        // super-nodes and their lowest common ancestor (preorder ids)
    int dir;            // 0: s's cluster above r's, 1: r's above s's
    int js, ns;         // s side: super-node list range [js, js + ns)
    int jr, nr;         // r side
    int fixed;          // 1: extra position for the merged cluster of s (s == a)
    int pad;
    unsigned long long key;   // (caller r, caller s) for the tie rule
};

// Reduction state (super-node quantities live at the super-node's bus index).
struct State {
    int *label;         // [n] super-node of each bus
    int *top;           // [n] topmost bus of each cluster
    int *ptop;          // [n] parent bus of that topmost bus (-1 for the slack's cluster)
    int *sn_list[2];    // [n] super-nodes in increasing preorder id after t merges: buffer t & 1
    int *sn_rank;       // [n+1] number of super-nodes with a smaller preorder id
    double2 *vcur;      // [L*3*n] super-node voltages for the current injections
    double2 *icur;      // [L*3*n] aggregated injections
    double *hi, *lo;    // [L*3*n] max / min of |vhat| over the cluster (per phase)
    double *mice;       // [L*n] current MICE of each cluster
    double *mcur;       // [L*3*n] |vcur|
    // single-precision copies for the screening sweep
    float2 *v32;        // [L*3*n] vcur
    float *hr32, *lr32; // [L*3*n] hi - |vcur|, lo - |vcur| (differences taken in FP64)
    float *mice32;      // [L*n]
    float2 *icur32;     // [L*3*n]
};

struct Ctrl {
    int t;                  // merges committed
    int max_merges;
    int done;               // 1 once the search has stopped
    int stop_reason;        // 0 target reached, 1 no feasible candidate
    int n_cand;             // candidates of the current iteration
    int total_pos;          // work positions of the current iteration
    int total_chunks;
    int n_super;            // super-nodes left
    int err;                // device-side error code (0 = none)
    int profile;            // 1: count arithmetic and time the sweep phase
    int iters;              // sweeps run
    int precision;          // 0 FP64 sweep, 1 FP32 screen + FP64 recheck
    int rechecks;           // iterations that needed an FP64 recheck
    int recheck_cands;      // candidates rechecked in FP64 over the run
    int objective;          // 0 SMICE (Algorithm 1), 1 largest error of the candidate network
    int scorer_fallbacks;   // learned pruning: iterations re-evaluated exhaustively
    double margin;          // voltage-error bound (p.u.)
    double tau;             // tie band
    double s_cur;           // SMICE of the current state
    long long candidates;   // candidates evaluated over the run
    int inc_mismatch;       // incremental search, verification mode: slots whose carried score differs
    int pad2;
    long long pad3[2];
    long long pruned;       // certified pruning: candidates the bound excluded over the run
    long long max_spins;    // limit of a device-side wait
    double sweep_flops;     // algorithmic flops of the sweeps (profile mode)
    unsigned long long sweep_ns;   // time in the sweep phase (profile mode, device timer)
    unsigned long long phase_ns[16];  // profile mode, CTA 0: time per step of an iteration
};

// Grid-wide barrier of the persistent search kernel.
struct GridBar {
    unsigned int count;     // arrivals since launch; barrier k completes at k * grid
    unsigned int pad;
};

// Incremental search (okr_incr.cu).  One work entry: the (candidate, cluster)
// terms of one candidate slot that an iteration evaluates, as ranges of
// super-node ranks.
constexpr int kIncMaxSeg = 7;
// Doubles per scenario of one position's scratch in Inc::cbuf: 10 FP64 values
// (voltage x, y and magnitude per phase, the MICE), then 8 doubles' room for
// their FP32 copies (a 16-byte (v.x, v.y, hr, lr) per phase, the MICE).
constexpr int kIncCbStride = 18;
struct IncWork {
    int slot;           // candidate slot 2 w + d (w = the lower super-node of the quotient edge)
    int mode;           // 0: terms of changed clusters, ranks before the merge; 1: every term, ranks after
    int nseg;
    int pad;
    int2 seg[kIncMaxSeg];   // rank ranges [x, y)
    int s, r, a, js, ns, jr, nr, fixed;     // the candidate's geometry (as in Cand)
};

// Per-feeder buffers of the incremental search.
struct Inc {
    unsigned long long *acc;    // [2n][2] carried D(c) of each candidate slot, fixed point (low, high word)
    unsigned long long *bnd;    // [2n][2] precision 1: carried bound on |D32 - D64|, fixed point
    int *viol;                  // [2n] precision 0: terms above the margin; precision 1: terms surely
                                //      above it; kIncDead: no candidate in the slot
    int *vmay;                  // [2n] precision 1: terms not surely within the margin
    int *qpar;                  // [n] super-node holding the parent of the cluster's top (-1: slack's cluster)
    int *fpair;                 // [n] slot pairs whose candidates are rebuilt after the merge
    IncWork *work;              // [2n] work entries of one iteration
    double *cbuf;               // [n * kIncCbStride L] the merge's new values per position (okr_incr.cu)
    unsigned long long *vacc;   // [2n][2] FP64 rescoring (precision-1 recheck, verification)
    int *vviol;                 // [2n]
    int *rlist;                 // [2n] slots rescored in FP64 in one iteration
    unsigned char *recbuf;      // [48 n + 64] selection records when they do not fit shared memory
    double *maxm;               // [n] largest MICE of each super-node over the scenarios (0 when absorbed)
};
constexpr int kIncDead = 1 << 30;

struct Search {
    const int *setup_err;   // the setup's error flag: the incremental search does nothing when it is set (null: none)
    Cand *cand;             // [2n] compact candidate list
    unsigned long long *ckey;   // [2n] tie key of each compact candidate
    Cand *slot;             // [2n] candidates by super-node slot (s < 0: none)
    int *base;              // [2n+1] first work position of each candidate
    int *arrive;            // [2n] pieces written so far (reset by the last writer)
    int2 *block_tot;        // [grid] per-CTA (candidates, positions)
    int *chunk_first;       // [max_chunks] candidate holding the first position of a chunk
    double2 *partial;       // [max_chunks + 2n] (sum of score changes, max new MICE), slot g + c
    double *score;          // [2n] score change D(c) (FP64 sweep, or FP64 recheck of R)
    int *feas;              // [2n]
    float4 *scr;            // [2n] screen: (D32, bound of D, max new MICE, bound of it)
    double *wsum;           // [grid*warps] per-warp FP64 score change of the committed merge
    double *mrank;          // [n] objective 1: largest MICE over scenarios, by super-node rank
    double *bmax;           // [n/32+1] objective 1: max of mrank over each block of 32 ranks
    int max_chunks;
    // per-iteration record
    int *dec_s, *dec_r;     // caller ids
    double *dec_score, *dec_maxerr, *dec_gap;
    int *dec_ncand;
    int rec_iters;
    int *rec_s, *rec_r;     // [rec_iters][2n]
    double *rec_score;
    double *rec_bound;      // [rec_iters][2n] bound of the recorded score (0 for FP64)
    float *rec_feat;        // [rec_iters][2n][kScorerFeatures] scorer features of the recorded candidates
    // learned pruning (topk > 0): the scorer's parameters (FP32 biases in mlp_theta,
    // bfloat16 bit patterns of the weight matrices) and a prediction per candidate slot
    int topk;
    const float *mlp_theta;
    const uint16_t *mlp_w1, *mlp_w2, *mlp_w3, *mlp_w4;
    float *pred;            // [2n] by slot
    // kept predictions, by candidate (2 * the slot pair's super-node + direction):
    // the prediction, the key of the candidate it was made for (~0: none), and per
    // super-node the merge count after which its state last changed (-1: never)
    float *pcache;          // [2n]
    unsigned long long *pkey;   // [2n]
    int *moved;             // [n]
    // certified pruning (prune_exact = 1, with topk > 0): per compact candidate the
    // part of its lower bound that depends on it (lbp; +inf: surely infeasible);
    // per super-node rank floor(g_k 2^56) summed within its block of 32 ranks
    // (gpre, inclusive), per block the total (gblk) and the sum of the blocks
    // before it (gbp, one past the last block included)
    int prune_exact;
    double *lbp;            // [2n]
    long long *gpre;        // [n]
    long long *gblk;        // [n / 32 + 2]
    long long *gbp;         // [n / 32 + 2]
    double *lbc;            // [2n] lbp kept by candidate (as pcache), with its key
    unsigned long long *lbkey;  // [2n]
    int *rec_count;
};

}  // namespace okr
