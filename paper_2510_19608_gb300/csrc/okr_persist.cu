// okr_persist.cu -- the exhaustive search (Algorithm 1, Sec. IV) as one
// persistent cooperative kernel, one CTA per SM, three grid barriers per
// iteration:
//
//   phase 1  select + commit of the last sweep (argmin with the tie band, then
//            the merge), fused with the candidate setup of the next sweep
//   phase 2  candidate compaction, work positions, chunk map, super-node list
//   phase 3  sweep: the score change of every candidate
//
// Candidate evaluation.  The paper evaluates a candidate (s, r) by moving the
// aggregated injection of r onto s and solving the full network (Y fixed), which
// gives the Kron-reduced super-node voltages (Sec. IV).  By linearity the new
// voltages are V + (Z_{:,s} - Z_{:,r}) I_r, and for a radial network
// Z_{k,j} = Zc(lca(k, j)) with Zc the path impedance from the slack.  With
// a = lca(s, r), the change at bus k is zero unless k hangs below the s-r path
// strictly under a:
//   k in subtree(child of a toward s):  dV_k = (Zc(lca(k,s)) - Zc(a)) I_r
//   k in subtree(child of a toward r):  dV_k = (Zc(a) - Zc(lca(k,r))) I_r
// Both sets are contiguous preorder ranges, hence contiguous ranges of the
// preorder-sorted super-node list.  Clusters outside them keep their voltages and
// their MICE, so a candidate's SMICE differs from the current one by
// D(c) = sum over affected clusters of (new MICE - current MICE), the merged
// cluster of s and r counted once (post-merge clusters).  Unaffected clusters
// already satisfy the margin, so feasibility is decided on the affected ones.
//
// MICE of a cluster for a candidate voltage m = |V^c_k|: with hi/lo the largest
// and smallest |Vhat| of the members on phase p, max_i | |Vhat_i| - m | =
// max(hi - m, m - lo); the MICE is the largest of these over phases.
//
// Work layout.  The (candidate, affected super-node) pairs of an iteration form
// one dense position space, candidates back to back.  Each position spreads over
// a group of SP = 4 * Lp lanes, one lane per (scenario, phase) (Lp = scenarios
// rounded up to a power of two; the fourth phase lane idles): on this GPU the
// FP64 pipe issues a warp instruction every few dozen cycles, so a lane's FP64
// chain sets the latency and short chains matter more than idle lanes.
// Per-candidate sums are reduced in a fixed order (group shuffles, a segmented
// warp scan, then the pieces of a candidate in chunk order), so results do not
// depend on timing.
//
// Memory written by other CTAs during the kernel is read with L2-coherent loads
// (ld.global.cg); the static feeder description with ordinary loads.
#include "okr_internal.cuh"
#include "okr_kernels.cuh"

namespace okr {

constexpr int kThreads = 512;

// ---------------------------------------------------------------- loads
__device__ __forceinline__ int ldi(const int *p) { return __ldcg(p); }
__device__ __forceinline__ double ldd(const double *p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldz(const double2 *p) { return __ldcg(p); }
__device__ __forceinline__ Cand ldcand(const Cand *p) {
    Cand c;
    const int4 *q = reinterpret_cast<const int4 *>(p);
    int4 a = __ldcg(q), b = __ldcg(q + 1), d = __ldcg(q + 2);
    c.s = a.x; c.r = a.y; c.a = a.z; c.dir = a.w;
    c.js = b.x; c.ns = b.y; c.jr = b.z; c.nr = b.w;
    c.fixed = d.x; c.pad = d.y;
    c.key = ((unsigned long long)(unsigned)d.w << 32) | (unsigned)d.z;
    return c;
}
static_assert(sizeof(Cand) == 48, "Cand layout");

// ---------------------------------------------------------------- grid barrier
// Sense by generation: thread 0 of each CTA arrives on the counter; the last
// arrival resets it and bumps the generation; the others wait for the bump.
// Every wait is bounded: after max_spins polls the CTA records err = 6 and the
// kernel unwinds (all CTAs leave at their next barrier or error check).
__device__ bool grid_barrier(GridBar *gb, Ctrl *C, unsigned nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &gb->gen;
        const unsigned my = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&gb->count, 1u);
        int ok = 1;
        if (arrived == nblocks - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            long long spins = 0;
            const long long lim = C->max_spins;
            while (*gen == my) {
                if (++spins > lim || *(volatile int *)&C->err) { ok = 0; break; }
                __nanosleep(32);
            }
            if (!ok) atomicCAS(&C->err, 0, 6);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok;
}

// ---------------------------------------------------------------- small helpers
__device__ __forceinline__ int child_toward(const Topo &T, int a, int v) {
    // children of a have increasing preorder ids; v's branch is the last one <= v
    int lo = T.child_off[a], hi = T.child_off[a + 1] - 1;
    if (hi < lo) return v;          // a has no children (cannot happen for a proper ancestor)
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (T.child[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return T.child[lo];
}

__device__ __forceinline__ unsigned long long tie_key(const Topo &T, int s, int r) {
    return ((unsigned long long)(unsigned)T.orig[r] << 32) | (unsigned)T.orig[s];
}

__device__ __forceinline__ int cand_positions(const Cand &c) { return c.ns + c.nr + c.fixed; }

// Position p of candidate c: the super-node it evaluates (list = the super-node
// list the candidate was built on) and its side; -1 for the merged-cluster
// position (s == a).
__device__ __forceinline__ int position_bus(const int *list, const Cand &c, int p, bool &sside) {
    if (p < c.ns) { sside = true; return ldi(list + c.js + p); }
    p -= c.ns;
    sside = false;
    if (p < c.nr) return ldi(list + c.jr + p);
    return -1;
}

template <typename Tv, typename Op>
__device__ Tv block_reduce(Tv v, Op op, Tv *smem) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) smem[wid] = v;
    __syncthreads();
    Tv r = smem[0];
    for (int w = 1; w < nw; ++w) r = op(r, smem[w]);
    return r;
}

struct MinD { __device__ double operator()(double a, double b) const { return fmin(a, b); } };
struct MaxD { __device__ double operator()(double a, double b) const { return fmax(a, b); } };
struct MinU { __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a < b ? a : b; } };
struct MinI { __device__ int operator()(int a, int b) const { return a < b ? a : b; } };

// Exclusive scan of (x, y) over the block; *tot receives the block totals.
__device__ int2 block_scan2(int2 v, int2 *smem, int2 *tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int2 inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int yx = __shfl_up_sync(0xffffffffu, inc.x, o);
        const int yy = __shfl_up_sync(0xffffffffu, inc.y, o);
        if (lane >= o) { inc.x += yx; inc.y += yy; }
    }
    __syncthreads();
    if (lane == 31) smem[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int2 w = lane < nw ? smem[lane] : make_int2(0, 0);
        int2 wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int yx = __shfl_up_sync(0xffffffffu, wi.x, o);
            const int yy = __shfl_up_sync(0xffffffffu, wi.y, o);
            if (lane >= o) { wi.x += yx; wi.y += yy; }
        }
        __syncwarp();
        if (lane < nw) smem[lane] = make_int2(wi.x - w.x, wi.y - w.y);
        if (lane == nw - 1) smem[32] = wi;
    }
    __syncthreads();
    *tot = smem[32];
    return make_int2(smem[wid].x + inc.x - v.x, smem[wid].y + inc.y - v.y);
}

// ---------------------------------------------------------------- one work item
// Scenario l, phase p of the cluster of super-node k for candidate cd: the
// cluster's new voltage on that phase and its largest member error
// max(hi - |V|, |V| - lo) (merged extremes when the cluster is s's).  k < 0
// stands for s's cluster when s is the common ancestor (no voltage change).
struct ItemOut {
    double e;
    double2 v;
    bool on;
};

__device__ __forceinline__ ItemOut eval_item(const Topo &T, const State &S, int n, const Cand &cd, int k, bool sside,
                                             int l, int p, const double2 *Ir, unsigned phr) {
    ItemOut o;
    o.e = 0.0;
    o.v = make_double2(0.0, 0.0);
    o.on = false;
    const int kk = k < 0 ? cd.s : k;
    if (!(T.ph[kk] >> p & 1u)) return o;
    double2 v = ldz(S.vcur + sidx(l, p, kk, n));
    if (k >= 0) {
        const int y = T.lca[(size_t)(sside ? cd.s : cd.r) * n + k];
        const double2 *zy = T.zc + (size_t)y * 9 + p * 3;
        const double2 *za = T.zc + (size_t)cd.a * 9 + p * 3;
        double2 dv = make_double2(0.0, 0.0);
        for (int q = 0; q < 3; ++q) {
            if (!(phr >> q & 1u)) continue;
            const double2 g = sside ? csub(zy[q], za[q]) : csub(za[q], zy[q]);
            dv = cadd(dv, cmul(g, Ir[q]));
        }
        v = cadd(v, dv);
    }
    const double mag = cmag(v);
    double h = ldd(S.hi + sidx(l, p, kk, n)), lo = ldd(S.lo + sidx(l, p, kk, n));
    if (kk == cd.s) {
        h = fmax(h, ldd(S.hi + sidx(l, p, cd.r, n)));
        lo = fmin(lo, ldd(S.lo + sidx(l, p, cd.r, n)));
    }
    o.e = fmax(h - mag, mag - lo);
    o.v = v;
    o.on = true;
    return o;
}

__device__ __forceinline__ double item_flops(const Topo &T, const Cand &cd, int k, unsigned phr) {
    // per (scenario, phase): per phase of r a complex subtraction and a complex
    // multiply-add; the voltage update, |V|, two differences, two maxima
    return k < 0 ? 8.0 : 10.0 * __popc(phr) + 10.0;
}

// ---------------------------------------------------------------- the kernel
__global__ void __launch_bounds__(kThreads, 1) k_search(Topo T, State S, Search X, Ctrl *C, GridBar *gb) {
    __shared__ double smd[32];
    __shared__ unsigned long long smu[32];
    __shared__ int smi[32];
    __shared__ int2 sm2[33];
    __shared__ int2 s_pref, s_tot;
    const int n = T.n, L = T.L;
    const int Lp = L <= 1 ? 1 : (L <= 2 ? 2 : 4);
    const int SP = 4 * Lp, PPW = 32 / SP;
    const unsigned G = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int gt = blockIdx.x * kThreads + tid, gs = (int)G * kThreads;
    const int warp = gt >> 5, nwarps = gs >> 5;
    const double margin = C->margin, tau = C->tau;
    const int max_merges = C->max_merges;
    const bool prof = C->profile != 0;
    const bool lead = (blockIdx.x == 0 && tid == 0);
    int t = C->t, ns = C->n_super;
    double s_cur = C->s_cur;
    bool have = false;                     // a sweep's scores wait for selection
    int nc = 0, P = 0, nchunks = 0;        // current candidate list
    int2 my_ex = make_int2(0, 0);          // this thread's offsets inside its CTA
    double flops = 0.0;
    if (t >= max_merges || C->done) return;

    for (;;) {
        // ============================================================ phase 1
        const int told = t;
        const int *list_old = S.sn_list[told & 1];
        bool committed = false;
        int r0 = -1, s0 = -1, dir0 = 0, jr0 = 0;
        if (have) {
            // ---- selection (identical in every CTA)
            double best = INFINITY;
            for (int c = tid; c < nc; c += kThreads)
                if (ldi(X.feas + c)) best = fmin(best, ldd(X.score + c));
            best = block_reduce(best, MinD(), smd);
            const bool rec = lead && t < X.rec_iters;
            if (best == INFINITY) {
                if (blockIdx.x == 0 && t < X.rec_iters) {
                    for (int c = tid; c < nc; c += kThreads) {
                        const Cand cd = ldcand(X.cand + c);
                        X.rec_s[(size_t)t * 2 * n + c] = T.orig[cd.s];
                        X.rec_r[(size_t)t * 2 * n + c] = T.orig[cd.r];
                        X.rec_score[(size_t)t * 2 * n + c] = INFINITY;
                    }
                }
                if (lead) {
                    if (t < X.rec_iters) X.rec_count[t] = nc;
                    C->done = 1; C->stop_reason = 1; C->t = t; C->s_cur = s_cur; C->n_super = ns;
                }
                break;
            }
            const double edge = best + tau;
            unsigned long long key = ~0ull;
            double gap = INFINITY;
            for (int c = tid; c < nc; c += kThreads) {
                if (!ldi(X.feas + c)) continue;
                const double d = ldd(X.score + c);
                if (d <= edge) {
                    const unsigned long long k = ldcand(X.cand + c).key;
                    if (k < key) key = k;
                } else {
                    gap = fmin(gap, d - edge);
                }
            }
            key = block_reduce(key, MinU(), smu);
            gap = block_reduce(gap, MinD(), smd);
            int w = 0x7fffffff;
            for (int c = tid; c < nc; c += kThreads)
                if (ldi(X.feas + c) && ldd(X.score + c) <= edge && ldcand(X.cand + c).key == key) w = min(w, c);
            w = block_reduce(w, MinI(), smi);
            if (w >= nc) {                              // unreachable: the minimum lies in the band
                if (lead) { C->err = 5; C->done = 1; }
                break;
            }
            const Cand cd = ldcand(X.cand + w);
            const double dw = ldd(X.score + w);
            if (blockIdx.x == 0 && t < X.rec_iters) {
                for (int c = tid; c < nc; c += kThreads) {
                    const Cand cc = ldcand(X.cand + c);
                    X.rec_s[(size_t)t * 2 * n + c] = T.orig[cc.s];
                    X.rec_r[(size_t)t * 2 * n + c] = T.orig[cc.r];
                    X.rec_score[(size_t)t * 2 * n + c] = ldi(X.feas + c) ? s_cur + ldd(X.score + c) : INFINITY;
                }
            }
            // ---- commit: r's cluster joins s
            const unsigned phr = T.ph[cd.r];
            for (int i = gt; i < n; i += gs)
                if (ldi(S.label + i) == cd.r) S.label[i] = cd.s;
            const int nitems = cand_positions(cd) * SP;
            for (int i0 = warp * 32; i0 < nitems; i0 += nwarps * 32) {
                const int item = i0 + lane;
                const int q = item / SP, sub = item % SP, l = sub >> 2, p = sub & 3;
                bool sside = false;
                const int k = item < nitems ? position_bus(list_old, cd, q, sside) : cd.r;
                const bool live = item < nitems && l < L && p < 3 && k != cd.r;
                ItemOut o;
                o.e = 0.0; o.on = false;
                if (live) {
                    double2 Ir[3];
                    for (int qq = 0; qq < 3; ++qq) Ir[qq] = ldz(S.icur + sidx(l, qq, cd.r, n));
                    o = eval_item(T, S, n, cd, k, sside, l, p, Ir, phr);
                }
                double m = o.e;
                m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 1));
                m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 2));
                if (live) {
                    const int kk = k < 0 ? cd.s : k;
                    if (o.on) {
                        S.vcur[sidx(l, p, kk, n)] = o.v;
                        if (kk == cd.s) {
                            S.hi[sidx(l, p, kk, n)] = fmax(ldd(S.hi + sidx(l, p, kk, n)), ldd(S.hi + sidx(l, p, cd.r, n)));
                            S.lo[sidx(l, p, kk, n)] = fmin(ldd(S.lo + sidx(l, p, kk, n)), ldd(S.lo + sidx(l, p, cd.r, n)));
                        }
                    }
                    if (p == 0) S.mice[(size_t)l * n + kk] = m;
                }
            }
            if (lead) {
                for (int l = 0; l < L; ++l) {
                    for (int q = 0; q < 3; ++q)
                        if (phr >> q & 1u)
                            S.icur[sidx(l, q, cd.s, n)] = cadd(ldz(S.icur + sidx(l, q, cd.s, n)), ldz(S.icur + sidx(l, q, cd.r, n)));
                    S.mice[(size_t)l * n + cd.r] = 0.0;
                }
                if (cd.dir == 1) S.top[cd.s] = ldi(S.top + cd.r);
                X.dec_s[t] = T.orig[cd.s];
                X.dec_r[t] = T.orig[cd.r];
                X.dec_score[t] = s_cur + dw;
                X.dec_gap[t] = gap;
                X.dec_ncand[t] = nc;
                if (rec) X.rec_count[t] = nc;
            }
            committed = true;
            r0 = cd.r; s0 = cd.s; dir0 = cd.dir;
            jr0 = ldi(S.sn_rank + r0);
            t += 1;
            s_cur += dw;
            ns -= 1;
            if (lead) { C->t = t; C->s_cur = s_cur; C->n_super = ns; }
            if (t >= max_merges) {
                if (lead) { C->done = 1; C->stop_reason = 0; }
                break;
            }
        }

        // ---- candidate setup for the next sweep (reads adjusted for the merge
        // committed above: label r -> s, rank drops past r, s's top)
        {
            int2 mine = make_int2(0, 0);
            const int j = gt;
            Cand c0, c1;
            c0.s = -1;
            c1.s = -1;
            if (j >= 1 && j < ns) {
                const int w = ldi(list_old + j + (committed && j >= jr0 ? 1 : 0));
                const int tw = (committed && w == s0 && dir0 == 1) ? ldi(S.top + r0) : ldi(S.top + w);
                int x = ldi(S.label + T.parent[tw]);
                if (committed && x == r0) x = s0;
                const int a = T.lca[(size_t)x * n + w];
                const int cw = child_toward(T, a, w);
                auto rank = [&](int b) { return ldi(S.sn_rank + b) - ((committed && b > r0) ? 1 : 0); };
                const int jw = rank(cw), nw = rank(cw + T.sz[cw]) - jw;
                int jx = 0, nx = 0;
                if (x != a) {
                    const int cx = child_toward(T, a, x);
                    jx = rank(cx);
                    nx = rank(cx + T.sz[cx]) - jx;
                }
                const unsigned pw = T.ph[w], px = T.ph[x];
                if ((pw & px) == pw) {                          // w's cluster joins x
                    c0.s = x; c0.r = w; c0.a = a; c0.dir = 0;
                    c0.js = jx; c0.ns = nx; c0.jr = jw; c0.nr = nw; c0.fixed = (x == a); c0.pad = 0;
                    c0.key = tie_key(T, x, w);
                    mine.x += 1;
                    mine.y += cand_positions(c0);
                }
                if (x != 0 && (px & pw) == px) {                // x's cluster joins w
                    c1.s = w; c1.r = x; c1.a = a; c1.dir = 1;
                    c1.js = jw; c1.ns = nw; c1.jr = jx; c1.nr = nx; c1.fixed = 0; c1.pad = 0;
                    c1.key = tie_key(T, w, x);
                    mine.x += 1;
                    mine.y += cand_positions(c1);
                }
            }
            if (j < ns) {
                X.slot[2 * j] = c0;
                X.slot[2 * j + 1] = c1;
            }
            int2 tot;
            my_ex = block_scan2(mine, sm2, &tot);
            if (tid == 0) X.block_tot[blockIdx.x] = tot;
        }
        if (!grid_barrier(gb, C, G)) return;

        // ============================================================ phase 2
        if (tid < 32) {
            int2 acc = make_int2(0, 0), all = make_int2(0, 0);
            for (int b = lane; b < (int)G; b += 32) {
                const int2 v = __ldcg(X.block_tot + b);
                if (b < (int)blockIdx.x) { acc.x += v.x; acc.y += v.y; }
                all.x += v.x;
                all.y += v.y;
            }
            for (int o = 16; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                all.x += __shfl_xor_sync(0xffffffffu, all.x, o);
                all.y += __shfl_xor_sync(0xffffffffu, all.y, o);
            }
            if (lane == 0) { s_pref = acc; s_tot = all; }
        }
        __syncthreads();
        const int2 pref = s_pref, tot = s_tot;
        nc = tot.x;
        P = tot.y;
        nchunks = (P + PPW - 1) / PPW;
        if (committed) {
            // super-node list after the merge (other buffer), ranks, largest MICE
            int *list_new = S.sn_list[t & 1];
            double m = 0.0;
            for (int j = gt; j < ns; j += gs) {
                const int k = ldi(list_old + j + (j >= jr0 ? 1 : 0));
                list_new[j] = k;
                for (int l = 0; l < L; ++l) m = fmax(m, ldd(S.mice + (size_t)l * n + k));
            }
            for (int b = r0 + 1 + gt; b <= n; b += gs) S.sn_rank[b] = ldi(S.sn_rank + b) - 1;
            m = block_reduce(m, MaxD(), smd);
            if (tid == 0 && m > 0.0)
                atomicMax((unsigned long long *)&X.dec_maxerr[told], (unsigned long long)__double_as_longlong(m));
        }
        if (nc == 0) {                                  // no candidate at all: nothing is feasible
            if (lead) { C->done = 1; C->stop_reason = 1; C->t = t; C->s_cur = s_cur; C->n_super = ns; }
            break;
        }
        if (nchunks > X.max_chunks) {                   // grow the work buffers and relaunch
            if (lead) { C->err = 7; C->total_pos = P; C->t = t; C->s_cur = s_cur; C->n_super = ns; }
            break;
        }
        if (gt >= 1 && gt < ns) {
            int ci = pref.x + my_ex.x, pos = pref.y + my_ex.y;
            for (int d = 0; d < 2; ++d) {
                const Cand c = X.slot[2 * gt + d];
                if (c.s < 0) continue;
                const int cnt = cand_positions(c);
                X.cand[ci] = c;
                X.base[ci] = pos;
                for (int g = (pos + PPW - 1) / PPW; g * PPW < pos + cnt; ++g) X.chunk_first[g] = ci;
                ++ci;
                pos += cnt;
            }
        }
        if (lead) {
            X.base[nc] = P;
            C->n_cand = nc;
            C->total_pos = P;
            C->candidates += nc;
            C->iters += 1;
        }
        if (!grid_barrier(gb, C, G)) return;

        // ============================================================ phase 3
        {
            const int *list_new = S.sn_list[t & 1];
            unsigned long long t_start = 0;
            if (prof && lead) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
            const int sub = lane % SP, l = sub >> 2, p = sub & 3;
            for (int g = warp; g < nchunks; g += nwarps) {
                const int c0 = ldi(X.chunk_first + g);
                const int q = g * PPW + lane / SP;
                const bool active = q < P;
                const int cb = (c0 + lane <= nc) ? ldi(X.base + c0 + lane) : 0x7fffffff;    // base[nc] = P
                int off = 0;
                for (int j = 1; j < 32; ++j) off += (__shfl_sync(0xffffffffu, cb, j) <= q);
                const int cbase = __shfl_sync(0xffffffffu, cb, off);
                const int c = c0 + off;
                Cand cd;
                cd.r = -1;
                int k = -1;
                bool sside = false;
                if (active) {
                    cd = ldcand(X.cand + c);
                    k = position_bus(list_new, cd, q - cbase, sside);
                }
                const bool valid = active && k != cd.r;
                const bool live = valid && l < L && p < 3;
                ItemOut o;
                o.e = 0.0;
                o.on = false;
                if (live) {
                    double2 Ir[3];
                    for (int qq = 0; qq < 3; ++qq) Ir[qq] = ldz(S.icur + sidx(l, qq, cd.r, n));
                    o = eval_item(T, S, n, cd, k, sside, l, p, Ir, T.ph[cd.r]);
                    if (prof && o.on) flops += item_flops(T, cd, k, T.ph[cd.r]);
                }
                double m = o.e;
                m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 1));
                m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 2));
                double dl = 0.0, ml = 0.0;
                if (valid && p == 0 && l < L) {
                    const int kk = k < 0 ? cd.s : k;
                    dl = m - ldd(S.mice + (size_t)l * n + kk);
                    if (kk == cd.s) dl -= ldd(S.mice + (size_t)l * n + cd.r);
                    ml = m;
                }
                for (int o2 = 4; o2 < SP; o2 <<= 1) {
                    dl += __shfl_xor_sync(0xffffffffu, dl, o2);
                    ml = fmax(ml, __shfl_xor_sync(0xffffffffu, ml, o2));
                }
                if (sub != 0) { dl = 0.0; ml = 0.0; }
                // segmented inclusive scan over the lanes of one candidate
                const int cseg = active ? c : -1 - lane;
                const int prev = __shfl_up_sync(0xffffffffu, cseg, 1);
                const bool head = (lane == 0) || (prev != cseg);
                const unsigned heads = __ballot_sync(0xffffffffu, head);
                const int seg_start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
                for (int o2 = 1; o2 < 32; o2 <<= 1) {
                    const double y = __shfl_up_sync(0xffffffffu, dl, o2);
                    const double z = __shfl_up_sync(0xffffffffu, ml, o2);
                    if (lane - o2 >= seg_start) { dl += y; ml = fmax(ml, z); }
                }
                const bool last = (lane == 31) || ((heads >> (lane + 1)) & 1u);
                if (active && last) {
                    const int first = cbase / PPW;
                    const int np = (cbase + cand_positions(cd) - 1) / PPW - first + 1;
                    X.partial[g + c] = make_double2(dl, ml);
                    __threadfence();
                    if (atomicAdd(X.arrive + c, 1) == np - 1) {
                        __threadfence();
                        double sum = 0.0, mx = 0.0;
                        for (int j = 0; j < np; ++j) {
                            const double2 pj = ldz(X.partial + first + c + j);
                            sum += pj.x;
                            mx = fmax(mx, pj.y);
                        }
                        X.score[c] = sum;
                        X.feas[c] = (mx <= margin);
                        X.arrive[c] = 0;
                    }
                }
            }
            if (!grid_barrier(gb, C, G)) return;
            if (prof && lead) {
                unsigned long long t_end;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
                C->sweep_ns += t_end - t_start;
            }
        }
        have = true;
    }
    if (prof) {
        for (int o2 = 16; o2 > 0; o2 >>= 1) flops += __shfl_xor_sync(0xffffffffu, flops, o2);
        if (lane == 0 && flops > 0.0) atomicAdd(&C->sweep_flops, flops);
    }
}

// Largest MICE of the final state into the record of the last merge (the
// search records every earlier merge itself).
__global__ void k_final_maxerr(Topo T, State S, Search X, const Ctrl *C) {
    const int n = T.n, L = T.L, t = C->t;
    if (t < 1) return;
    double m = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        if (S.label[k] == k)
            for (int l = 0; l < L; ++l) m = fmax(m, S.mice[(size_t)l * n + k]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax((unsigned long long *)&X.dec_maxerr[t - 1], (unsigned long long)__double_as_longlong(m));
}

// Results in caller numbering: super-node of each bus, reduced-network voltage
// of each bus (its super-node's), and the scenario voltages ([L][n][3][2]).
__global__ void k_export(Topo T, State S, double *vred, int *super_of, double *vhat_out) {
    const int n = T.n, L = T.L;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L * n; e += gridDim.x * blockDim.x) {
        const int l = e / n, i = e % n;
        const int v = T.pre[i];
        const int k = S.label[v];
        if (l == 0 && super_of) super_of[i] = T.orig[k];
        for (int p = 0; p < 3; ++p) {
            const bool on = T.ph[v] >> p & 1u;
            const size_t o = (((size_t)l * n + i) * 3 + p) * 2;
            double2 vr = on ? S.vcur[sidx(l, p, k, n)] : make_double2(0.0, 0.0);
            double2 vh = on ? T.vhat[sidx(l, p, v, n)] : make_double2(0.0, 0.0);
            if (vred) { vred[o] = vr.x; vred[o + 1] = vr.y; }
            if (vhat_out) { vhat_out[o] = vh.x; vhat_out[o + 1] = vh.y; }
        }
    }
}

}  // namespace okr
