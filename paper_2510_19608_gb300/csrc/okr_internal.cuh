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

__host__ __device__ __forceinline__ size_t sidx(int l, int p, int k, int n) { return ((size_t)l * 3 + p) * n + k; }

// ---------------------------------------------------------------- device structures
// Static description of one feeder (preorder numbering), built once per call.
struct Topo {
    int n, L;
    int *maxd;          // [1] deepest level (written on the device)
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
    double2 *vhat;      // [L*3*n] scenario voltages
    double2 *ihat;      // [L*3*n] scenario injections, Y vhat
    double *amag;       // [L*3*n] |vhat|
    double2 *vslack;    // [3]
};

// Candidate slot 2*w + d for the quotient edge above cluster w (d = 0: w's
// cluster joins its parent cluster x; d = 1: x's cluster joins w).
struct Cand {
    int s, r, a;        // super-nodes and their lowest common ancestor
    int dir;            // 0: s above r, 1: r above s
    int lo_s, len_s;    // buses whose path to s leaves the s-r path below a
    int lo_r, len_r;    // same on the r side
    unsigned long long key;   // (caller r, caller s) for the tie rule
};

// Reduction state (super-node quantities live at the super-node's index).
struct State {
    int *label;         // [n] super-node of each bus
    int *top;           // [n] topmost bus of each cluster
    double2 *vcur;      // [L*3*n] super-node voltages for the current injections
    double2 *icur;      // [L*3*n] aggregated injections
    double *hi, *lo;    // [L*3*n] max / min of |vhat| over the cluster (per phase)
    double *mice;       // [L*n] current MICE of each cluster
};

struct Ctrl {
    int t;                  // merges committed
    int max_merges;
    int done;               // 1 once the search has stopped
    int stop_reason;        // 0 target reached, 1 no feasible candidate
    int total_chunks;
    int win;                // winning slot of the last iteration
    int commit;             // 1 between a selection and its commit
    int n_valid;            // candidates of the last iteration
    int err;                // device-side error code (0 = none)
    double margin;          // voltage-error bound (p.u.)
    double tau;             // tie band
    double s_cur;           // SMICE of the current state
    double win_d;           // score change of the winner
    double gap;             // distance of the next score above the tie band
    long long candidates;   // candidates evaluated over the run
    int profile;            // 1: the sweep counts its arithmetic
    int sweeps_run;         // sweep launches that found work (profile mode)
    double sweep_flops;     // algorithmic flops of those sweeps (profile mode)
};

struct Search {
    Cand *cand;             // [2n]
    int *nchunk;            // [2n]
    int *base;              // [2n+1]
    int *chunk_cand;        // [max_chunks]
    double2 *partial;       // [max_chunks] (sum of score changes, max new MICE)
    double *score;          // [2n] score change D(c)
    int *feas;              // [2n]
    int max_chunks;
    // per-iteration record
    int *dec_s, *dec_r;     // caller ids
    double *dec_score, *dec_maxerr, *dec_gap;
    int *dec_ncand;
    int rec_iters;
    int *rec_s, *rec_r;     // [rec_iters][2n]
    double *rec_score;
    int *rec_count;
};

}  // namespace okr
