// okr_layout.cuh -- device buffers of one feeder and their layout inside one
// allocation.  The single-feeder context and the multi-feeder batch lay out
// every feeder the same way.
#pragma once

#include "okr_internal.cuh"

namespace okr {

struct FeederBufs {
    int n = 0, L = 0, rec = 0;
    // inputs (caller numbering)
    int *parent_in = nullptr;
    uint8_t *ph_in = nullptr;
    double *z_in = nullptr, *s_in = nullptr, *vh_in = nullptr, *ih_in = nullptr;
    // topology scratch
    int *dep = nullptr, *anc = nullptr, *anc2 = nullptr, *d2 = nullptr, *size = nullptr, *ccount = nullptr;
    int *coff_c = nullptr, *child_c = nullptr;
    uint16_t *rmq = nullptr;
    double2 *J = nullptr;
    int *pf_iters = nullptr, *err_dev = nullptr;
    GridBar *gb = nullptr;
    // outputs (caller numbering)
    int *super_out = nullptr;
    double *vred_out = nullptr, *vhat_out = nullptr;
    Topo T{};
    State S{};
    Search X{};
    Inc I{};
    Ctrl *C = nullptr;
};

// Measures (base == nullptr) or assigns (base != nullptr) 256-byte aligned pieces.
struct Carver {
    unsigned char *base = nullptr;
    size_t used = 0;
    template <typename T>
    void take(T *&p, size_t count) {
        const size_t bytes = (sizeof(T) * (count ? count : 1) + 255) / 256 * 256;
        p = base ? reinterpret_cast<T *>(base + used) : nullptr;
        used += bytes;
    }
};

inline int log2_ceil_i(int n) {
    int j = 0;
    while ((1 << j) < n) ++j;
    return j;
}

// Every per-feeder buffer for n buses, L scenarios, `rec` recorded iterations,
// a search grid of `grid` CTAs (per-warp sums) and, if chunks > 0, the chunk
// map and partial sums of `chunks` chunks (otherwise left for the caller).
inline void layout_feeder(Carver &c, int n, int L, int rec, int grid, long long chunks, FeederBufs &f) {
    const size_t N = n, NL3 = (size_t)3 * L * n;
    const int LOG = log2_ceil_i(n) + 1;
    f.n = n;
    f.L = L;
    f.rec = rec;
    c.take(f.parent_in, N);
    c.take(f.ph_in, N);
    c.take(f.z_in, N * 18);
    c.take(f.s_in, (size_t)L * N * 6);
    c.take(f.vh_in, (size_t)L * N * 6);
    c.take(f.ih_in, (size_t)L * N * 6);
    c.take(f.dep, N);
    c.take(f.anc, N);
    c.take(f.anc2, N);
    c.take(f.d2, N);
    c.take(f.size, N);
    c.take(f.ccount, N + 2);
    c.take(f.coff_c, N + 1);
    c.take(f.child_c, N);
    c.take(f.rmq, (size_t)LOG * N);
    c.take(f.J, NL3);
    c.take(f.pf_iters, (size_t)L);
    c.take(f.err_dev, 1);
    c.take(f.super_out, N);
    c.take(f.vred_out, (size_t)L * N * 6);
    c.take(f.vhat_out, (size_t)L * N * 6);

    Topo &T = f.T;
    T.n = n;
    T.L = L;
    c.take(T.maxd, 2);
    c.take(T.parent, N);
    c.take(T.orig, N);
    c.take(T.pre, N);
    c.take(T.sz, N);
    c.take(T.depth, N);
    c.take(T.child_off, N + 1);
    c.take(T.child, N);
    c.take(T.level_off, N + 2);
    c.take(T.level_bus, N);
    c.take(T.ph, N);
    c.take(T.lca, N * N);
    c.take(T.zl, N * 9);
    c.take(T.yl, N * 9);
    c.take(T.zc, N * 9);
    c.take(T.zh, N * 9);
    c.take(T.zlo, N * 9);
    c.take(T.vhat, NL3);
    c.take(T.ihat, NL3);
    c.take(T.amag, NL3);
    c.take(T.vslack, 3);

    State &S = f.S;
    c.take(S.label, N);
    c.take(S.top, N);
    c.take(S.ptop, N);
    c.take(S.sn_list[0], N);
    c.take(S.sn_list[1], N);
    c.take(S.sn_rank, N + 1);
    c.take(S.vcur, NL3);
    c.take(S.icur, NL3);
    c.take(S.hi, NL3);
    c.take(S.lo, NL3);
    c.take(S.mice, (size_t)L * N);
    c.take(S.mcur, NL3);
    c.take(S.v32, NL3);
    c.take(S.hr32, NL3);
    c.take(S.lr32, NL3);
    c.take(S.mice32, (size_t)L * N);
    c.take(S.icur32, NL3);

    Search &X = f.X;
    c.take(X.cand, 2 * N);
    c.take(X.slot, 2 * N);
    c.take(X.ckey, 2 * N);
    c.take(X.base, 2 * N + 1);
    c.take(X.arrive, 2 * N);
    c.take(X.block_tot, (size_t)grid);
    c.take(X.score, 2 * N);
    c.take(X.feas, 2 * N);
    c.take(X.scr, 2 * N);
    c.take(X.wsum, (size_t)grid * 32);
    c.take(X.mrank, N);
    c.take(X.bmax, N / 32 + 2);
    c.take(f.gb, 1);
    c.take(X.dec_s, N);
    c.take(X.dec_r, N);
    c.take(X.dec_score, N);
    c.take(X.dec_maxerr, N);
    c.take(X.dec_gap, N);
    c.take(X.dec_ncand, N);
    const size_t R = rec > 0 ? (size_t)rec : 1;
    c.take(X.rec_s, R * 2 * N);
    c.take(X.rec_r, R * 2 * N);
    c.take(X.rec_score, R * 2 * N);
    c.take(X.rec_bound, R * 2 * N);
    c.take(X.rec_count, R);
    c.take(X.rec_feat, R * 2 * N * kScorerFeatures);
    c.take(X.pred, 2 * N);
    c.take(X.pcache, 2 * N);
    c.take(X.pkey, 2 * N);
    c.take(X.moved, N);
    c.take(X.lbp, 2 * N);
    c.take(X.gpre, N);
    c.take(X.gblk, N / 32 + 2);
    c.take(X.gbp, N / 32 + 2);
    c.take(X.lbc, 2 * N);
    c.take(X.lbkey, 2 * N);
    X.setup_err = nullptr;
    X.topk = 0;
    X.prune_exact = 0;
    X.mlp_theta = nullptr;
    X.mlp_w1 = X.mlp_w2 = X.mlp_w3 = X.mlp_w4 = nullptr;
    c.take(f.C, 1);
    Inc &I = f.I;
    c.take(I.acc, 4 * N);
    c.take(I.bnd, 4 * N);
    c.take(I.viol, 2 * N);
    c.take(I.vmay, 2 * N);
    c.take(I.rlist, 2 * N);
    c.take(I.recbuf, 48 * N + 64);
    c.take(I.maxm, N);
    c.take(I.qpar, N);
    c.take(I.fpair, N);
    c.take(I.work, 2 * N + kIncInitCtasMax);      // (+ the first evaluation's candidates cut between CTAs)
    c.take(I.cbuf, N * (size_t)kIncCbStride * L);
    c.take(I.vacc, 4 * N);
    c.take(I.vviol, 2 * N);
    if (chunks > 0) {
        c.take(X.chunk_first, (size_t)chunks);
        c.take(X.partial, (size_t)chunks + 2 * N);
        X.max_chunks = (int)chunks;
    } else {
        X.chunk_first = nullptr;
        X.partial = nullptr;
        X.max_chunks = 0;
    }
}

}  // namespace okr
