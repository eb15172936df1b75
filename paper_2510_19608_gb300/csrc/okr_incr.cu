// okr_incr.cu -- the exhaustive search (Algorithm 1, Sec. IV) with every
// candidate's score carried from one iteration to the next.
//
// Why scores can be carried.  As in okr_persist.cu, candidate c = (s, r) with
// a = lca(s, r) moves voltages only in two preorder ranges (the subtrees of the
// children of a toward s and toward r), and its SMICE is s_cur + D(c) with
//   D(c) = sum over its positions k and scenarios l of
//          (new MICE of k) - MICE_k  [- MICE_r when k = s: the merged cluster],
// the positions being the super-nodes of the two ranges (r excluded) and s.
// One term reads only: k's voltage, extremes and MICE; r's aggregated
// injection; the geometry (s, r, a); and, for k = s, r's extremes and MICE.
// A merge (s*, r*) changes those inputs only for the clusters whose voltage
// moves (the merge's own two ranges), for s* (extremes, MICE, injection) and
// for r* (removed); the quotient edges change only around s* and r*.  So after
// a merge only the terms that read a changed input are evaluated again:
//   - candidates next to s* or r* (slot pairs of s* and of the children of s*
//     and r* in the quotient tree) are rebuilt and every term evaluated;
//   - every other candidate evaluates the terms of its positions inside the
//     changed set, once on the state before the merge (subtracted) and once
//     on the state after it (added), plus its s term when r's MICE changed.
// On a 1,000-bus feeder that is about 0.2 % of the terms a full sweep
// evaluates.
//
// Exactness.  D(c) is held as a 128-bit fixed-point integer (units of 2^-100
// p.u.).  A term is computed in FP64 and converted by a fixed function of its
// bits; integer addition is associative, so removing a term's old value and
// adding its new one gives exactly the sum a fresh evaluation of every term
// gives, in any order.  The old value is recomputed from the unchanged inputs
// by the same compiled function (term(), not inlined), so it is bit-identical
// to the value added earlier.  Feasibility is carried the same way: the count of
// (cluster, scenario) terms whose new MICE exceeds the margin.  Engine 3 checks
// both against a full re-evaluation after every merge.
//
// Selection compares the fixed-point D(c) exactly: the minimum m over feasible
// candidates, the tie band D <= m + tau, and the smallest (r, s) key in it.
//
// Execution.  One CTA runs one feeder's whole search; its steps are separated
// by __syncthreads only (no grid barrier, no device-side wait).  A batch runs
// one CTA per feeder.
#include "okr_internal.cuh"
#include "okr_kernels.cuh"

namespace okr {

namespace {

typedef unsigned __int128 u128;

constexpr int kFxShift = 100;               // fixed point: value * 2^100
constexpr u128 kSignBit = (u128)1 << 127;

__device__ __forceinline__ unsigned long long gtimer_inc() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// d * 2^100 truncated toward zero, modulo 2^128 (|d| < 2^27 is represented
// exactly up to the truncation; larger values wrap, which subtraction of the
// same value undoes).  Non-finite d counts as 0 (its term is infeasible anyway).
__device__ __forceinline__ u128 to_fx(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    int e = (int)((b >> 52) & 0x7ff);
    if (e == 0x7ff) return 0;
    unsigned long long m = b & 0xfffffffffffffull;
    if (e == 0) e = 1;
    else m |= 1ull << 52;
    // d = m * 2^(e - 1075), so d * 2^100 = m * 2^(e - 975)
    const int sh = e - 1075 + kFxShift;
    u128 v;
    if (sh >= 0) v = sh >= 128 ? (u128)0 : ((u128)m << sh);
    else v = sh <= -64 ? (u128)0 : (u128)(m >> (-sh));
    return (b >> 63) ? (u128)0 - v : v;
}

__device__ __forceinline__ double fx_to_d(u128 v) {
    const bool neg = (v & kSignBit) != 0;
    const u128 a = neg ? (u128)0 - v : v;
    const double r = (double)(unsigned long long)(a >> 64) * 18446744073709551616.0 + (double)(unsigned long long)a;
    const double x = r * 7.8886090522101180541e-31;     // 2^-100
    return neg ? -x : x;
}

__device__ __forceinline__ u128 ld128(const unsigned long long *p) {
    return ((u128)p[1] << 64) | (u128)p[0];
}
__device__ __forceinline__ void st128(unsigned long long *p, u128 v) {
    p[0] = (unsigned long long)v;
    p[1] = (unsigned long long)(v >> 64);
}
// signed order as unsigned order
__device__ __forceinline__ u128 okey(u128 v) { return v ^ kSignBit; }

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int o) {
    const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
    const unsigned long long hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
    return ((u128)hi << 64) | lo;
}

// Exact 128-bit accumulation into shared memory from many threads: the low
// words add modulo 2^64 and every addition that wraps carries one into the high
// word, so the pair ends as the exact sum modulo 2^128 in any order.
__device__ __forceinline__ void sadd128(unsigned long long *lo, unsigned long long *hi, u128 v) {
    const unsigned long long vl = (unsigned long long)v, vh = (unsigned long long)(v >> 64);
    const unsigned long long old = atomicAdd(lo, vl);
    atomicAdd(hi, vh + ((old + vl < old) ? 1ull : 0ull));
}

// ---------------------------------------------------------------- block primitives
template <int NT>
__device__ __forceinline__ int block_sum_int(int v, int *sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < NT / 32; ++w) t += sm[w];
    return t;
}

template <int NT>
__device__ __forceinline__ double block_max_d(double v, double *sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    double t = sm[0];
    for (int w = 1; w < NT / 32; ++w) t = fmax(t, sm[w]);
    return t;
}

// Exclusive prefix sum of one int per thread; *total = the block's sum.
template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int *total, int *sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sm[wid] = x;
    __syncthreads();
    int before = 0, tot = 0;
    for (int w = 0; w < NT / 32; ++w) {
        const int s = sm[w];
        if (w < wid) before += s;
        tot += s;
    }
    *total = tot;
    return before + x - v;
}

// Block minima of two 128-bit keys and one 64-bit key at once.
struct Min3 {
    u128 a, b;
    unsigned long long c;
};
template <int NT>
__device__ __forceinline__ void block_min3(u128 &a, u128 &b, unsigned long long &c, Min3 *sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const u128 ya = shfl_xor_u128(a, o), yb = shfl_xor_u128(b, o);
        const unsigned long long yc = __shfl_xor_sync(0xffffffffu, c, o);
        a = ya < a ? ya : a;
        b = yb < b ? yb : b;
        c = yc < c ? yc : c;
    }
    __syncthreads();
    if (lane == 0) sm[wid] = Min3{a, b, c};
    __syncthreads();
    a = sm[0].a;
    b = sm[0].b;
    c = sm[0].c;
    for (int w = 1; w < NT / 32; ++w) {
        a = sm[w].a < a ? sm[w].a : a;
        b = sm[w].b < b ? sm[w].b : b;
        c = sm[w].c < c ? sm[w].c : c;
    }
}

// ---------------------------------------------------------------- geometry
__device__ __forceinline__ int child_toward_inc(const Topo &T, int a, int v) {
    // children of a have increasing preorder ids; v's branch is the last one <= v
    int lo = T.child_off[a], hi = T.child_off[a + 1] - 1;
    if (hi < lo) return v;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.child[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return T.child[lo];
}

// The two candidates of the quotient edge above super-node w, from the current
// clusters: x = super-node holding the parent of w's top, a = lca(x, w), cw and
// cx the children of a toward w and x.  Slot 2w: w's cluster joins x (s = x,
// r = w); slot 2w + 1: x's cluster joins w (s = w, r = x; never the slack's
// cluster).  js/ns and jr/nr hold the s-side and r-side subtrees as BUS
// ranges [j, j + size) (preorder ids); fixed = 1 when s is the common ancestor.
// Returns x (-1 for the slack's cluster, which has no edge above it).
__device__ int slot_geometry(const Topo &T, const State &S, int n, int w, Cand &c0, Cand &c1) {
    c0.s = -1;
    c1.s = -1;
    const int pb = S.ptop[w];
    if (pb < 0 || S.label[w] != w) return -1;
    const int tw = S.top[w];
    const int x = S.label[pb];
    const bool direct = (x == pb);
    const int a = direct ? x : (int)T.lca[(size_t)x * n + w];
    const int cw = direct ? tw : child_toward_inc(T, a, w);
    const int cx = (x != a) ? child_toward_inc(T, a, x) : -1;
    const int szw = T.sz[cw], szx = cx >= 0 ? T.sz[cx] : 0;
    const unsigned pw = T.ph[w], px = T.ph[x];
    const unsigned long long ow = (unsigned)T.orig[w], ox = (unsigned)T.orig[x];
    if ((pw & px) == pw) {
        c0.s = x; c0.r = w; c0.a = a; c0.dir = 0;
        c0.js = cx >= 0 ? cx : 0; c0.ns = szx; c0.jr = cw; c0.nr = szw;
        c0.fixed = (x == a) ? 1 : 0; c0.pad = 0;
        c0.key = (ow << 15) | ox;                   // (caller r, caller s)
    }
    if (x != 0 && (px & pw) == px) {
        c1.s = w; c1.r = x; c1.a = a; c1.dir = 1;
        c1.js = cw; c1.ns = szw; c1.jr = cx >= 0 ? cx : 0; c1.nr = szx;
        c1.fixed = 0; c1.pad = 0;
        c1.key = (ox << 15) | ow;
    }
    return x;
}

// ---------------------------------------------------------------- one term
// Term of position k (a super-node, k != c.r) of candidate c over every
// scenario: fx = sum over l of fixed(new MICE - MICE_k [- MICE_r if k = s]),
// nv = scenarios whose new MICE exceeds the margin.  With out != nullptr it
// also writes the new voltage and magnitude per (l, p) and the new MICE per l
// (the merge of the winner).  Not inlined: every evaluation of a term runs the
// same instructions, so equal inputs give bit-equal terms.
__device__ __noinline__ void term(const Topo &T, const State &S, int n, int L, const Cand &c, int k, double margin,
                                  u128 *fx_out, int *nv_out, double *out) {
    const bool fixed = (k == c.s) && c.fixed;
    const bool sside = (k >= c.js && k < c.js + c.ns);
    const unsigned phk = T.ph[k], phr = T.ph[c.r];
    const int y = fixed ? 0 : (int)T.lca[(size_t)(sside ? c.s : c.r) * n + k];
    const double2 *zy = T.zc + (size_t)y * 9, *za = T.zc + (size_t)c.a * 9;
    u128 fx = 0;
    int nv = 0;
    for (int l = 0; l < L; ++l) {
        double2 Ir[3];
        for (int q = 0; q < 3; ++q) Ir[q] = S.icur[sidx(l, q, c.r, n)];
        double m = 0.0;
        for (int p = 0; p < 3; ++p) {
            if (!(phk >> p & 1u)) continue;
            double2 v = S.vcur[sidx(l, p, k, n)];
            if (!fixed) {
                double2 dv = make_double2(0.0, 0.0);
                for (int q = 0; q < 3; ++q) {
                    if (!(phr >> q & 1u)) continue;
                    const double2 g = sside ? csub(zy[p * 3 + q], za[p * 3 + q]) : csub(za[p * 3 + q], zy[p * 3 + q]);
                    dv = cadd(dv, cmul(g, Ir[q]));
                }
                v = cadd(v, dv);
            }
            const double mag = cmag(v);
            double h = S.hi[sidx(l, p, k, n)], lo = S.lo[sidx(l, p, k, n)];
            if (k == c.s) {
                h = fmax(h, S.hi[sidx(l, p, c.r, n)]);
                lo = fmin(lo, S.lo[sidx(l, p, c.r, n)]);
            }
            m = fmax(m, fmax(h - mag, mag - lo));
            if (out) {
                out[(l * 3 + p) * 3 + 0] = v.x;
                out[(l * 3 + p) * 3 + 1] = v.y;
                out[(l * 3 + p) * 3 + 2] = mag;
            }
        }
        double d = m - S.mice[(size_t)l * n + k];
        if (k == c.s) d -= S.mice[(size_t)l * n + c.r];
        fx += to_fx(d);
        nv += (m > margin) ? 1 : 0;
        if (out) out[9 * L + l] = m;
    }
    *fx_out = fx;
    *nv_out = nv;
}

// ---------------------------------------------------------------- the changed set of a merge
struct Win {
    int slot, s, r, a, dir, fixed;
    int w1lo, w1hi, w2lo, w2hi;     // bus ranges whose voltages move
    int rtop, rtop_end;             // r's cluster lies inside [rtop, rtop_end)
    int jr;                         // rank of r before the merge
    int npos;                       // positions of the merge (ranks of the two ranges, r excluded, + fixed s)
    int q1lo, q1hi, q2lo, q2hi;     // their rank ranges before the merge
};

__device__ __forceinline__ bool in_range(int b, int lo, int hi) { return b >= lo && b < hi; }

// Rank ranges of the terms of candidate c that read an input the merge h
// changes (c is not next to s* or r*).  Returns their number (0: c unchanged).
__device__ int changed_segments(const Cand &c, const Win &h, const int *sn_rank, int2 *seg) {
    int k = 0;
    const int clo[2] = {c.js, c.jr}, chi[2] = {c.js + c.ns, c.jr + c.nr};
    const int wlo[2] = {h.w1lo, h.w2lo}, whi[2] = {h.w1hi, h.w2hi};
    for (int i = 0; i < 2; ++i) {
        if (clo[i] >= chi[i]) continue;
        for (int j = 0; j < 2; ++j) {
            if (wlo[j] >= whi[j]) continue;
            const int lo = max(clo[i], wlo[j]), hi = min(chi[i], whi[j]);
            if (lo < hi) {
                const int a = sn_rank[lo], b = sn_rank[hi];
                if (a < b) seg[k++] = make_int2(a, b);
            }
        }
    }
    // points: s* and r* where a range of c holds them outside the moved ranges,
    // and s when its term changes (it is not inside the ranges when fixed)
    auto in_cr = [&](int b) { return in_range(b, c.js, c.js + c.ns) || in_range(b, c.jr, c.jr + c.nr); };
    auto in_w = [&](int b) { return in_range(b, h.w1lo, h.w1hi) || in_range(b, h.w2lo, h.w2hi); };
    auto point = [&](int b) { const int a = sn_rank[b]; seg[k++] = make_int2(a, a + 1); };
    if (h.s != c.r && in_cr(h.s) && !in_w(h.s)) point(h.s);
    if (h.r != c.r && in_cr(h.r) && !in_w(h.r)) point(h.r);
    // the s term also reads r's MICE
    const bool r_changed = in_w(c.r) || c.r == h.s || c.r == h.r;
    if (c.fixed) {
        if (in_w(c.s) || c.s == h.s || c.s == h.r || r_changed) point(c.s);
    } else if (r_changed && !in_w(c.s) && c.s != h.s && c.s != h.r) {
        point(c.s);
    }
    return k;
}

// Every term of candidate c: its two ranges and the fixed s, as ranks.
__device__ int full_segments(const Cand &c, const int *sn_rank, int2 *seg) {
    int k = 0;
    if (c.ns > 0) {
        const int a = sn_rank[c.js], b = sn_rank[c.js + c.ns];
        if (a < b) seg[k++] = make_int2(a, b);
    }
    if (c.nr > 0) {
        const int a = sn_rank[c.jr], b = sn_rank[c.jr + c.nr];
        if (a < b) seg[k++] = make_int2(a, b);
    }
    if (c.fixed) { const int a = sn_rank[c.s]; seg[k++] = make_int2(a, a + 1); }
    return k;
}

__device__ __forceinline__ void write_entry(IncWork *w, int slot, int mode, int nseg, const int2 *seg) {
    w->slot = slot;
    w->mode = mode;
    w->nseg = nseg;
    w->pad = 0;
    for (int i = 0; i < nseg; ++i) w->seg[i] = seg[i];
}

// ---------------------------------------------------------------- evaluation of work entries
struct EvalSmem {
    unsigned long long lo[1024], hi[1024];
    int nv[1024];
    int off[1025];
};

// Evaluates the terms of entries [e0, e1) of I.work and applies them to the
// accumulators (acc, viol): sub = subtract (terms before the merge); entries
// of mode 1 are set (every term), the others added.  Mode-0 entries take
// positions from list_old and skip r* after the merge; mode-1 entries from
// list_new.  Returns the number of terms evaluated (thread 0's count is exact).
template <int NT>
__device__ long long eval_entries(const Topo &T, const State &S, const Search &X, const Inc &I, int n, int L,
                                  double margin, int e0, int e1, bool sub, int rstar, const int *list_old,
                                  const int *list_new, unsigned long long *acc, int *viol, EvalSmem *E, int *smi) {
    const int tid = threadIdx.x;
    long long terms = 0;
    for (int t0 = e0; t0 < e1; t0 += NT) {
        const int e = t0 + tid;
        int cnt = 0;
        if (e < e1) {
            const IncWork &w = I.work[e];
            for (int i = 0; i < w.nseg; ++i) cnt += w.seg[i].y - w.seg[i].x;
        }
        int tot = 0;
        const int off = block_excl_scan<NT>(cnt, &tot, smi);
        E->off[tid] = off;
        if (tid == NT - 1) E->off[NT] = tot;
        E->lo[tid] = 0ull;
        E->hi[tid] = 0ull;
        E->nv[tid] = 0;
        terms += tot;
        const int ne = min(NT, e1 - t0);
        __syncthreads();
        for (int q = tid; q < tot; q += NT) {
            int lo = 0, hi = ne - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (E->off[mid] <= q) lo = mid;
                else hi = mid - 1;
            }
            const IncWork &w = I.work[t0 + lo];
            int rem = q - E->off[lo], j = -1;
            for (int i = 0; i < w.nseg; ++i) {
                const int len = w.seg[i].y - w.seg[i].x;
                if (rem < len) { j = w.seg[i].x + rem; break; }
                rem -= len;
            }
            if (j < 0) continue;
            const int k = (w.mode == 0 ? list_old : list_new)[j];
            const Cand &c = X.slot[w.slot];
            if (k == c.r || (!sub && w.mode == 0 && k == rstar)) continue;
            u128 fx;
            int nv;
            term(T, S, n, L, c, k, margin, &fx, &nv, nullptr);
            if (sub) { fx = (u128)0 - fx; nv = -nv; }
            sadd128(&E->lo[lo], &E->hi[lo], fx);
            if (nv) atomicAdd(&E->nv[lo], nv);
        }
        __syncthreads();
        if (e < e1) {
            const IncWork &w = I.work[e];
            const u128 add = ((u128)E->hi[tid] << 64) | (u128)E->lo[tid];
            unsigned long long *a = acc + 2 * (size_t)w.slot;
            if (w.mode == 1 && !sub) {
                st128(a, add);
                viol[w.slot] = E->nv[tid];
            } else {
                st128(a, ld128(a) + add);
                viol[w.slot] += E->nv[tid];
            }
        }
        __syncthreads();
    }
    return terms;
}

// Slot pairs w handled by this thread: [w_b, w_e), consecutive.
template <int NT>
__device__ __forceinline__ void my_pairs(int n, int &wb, int &we) {
    const int per = (n + NT - 1) / NT;
    wb = min(n, (int)threadIdx.x * per);
    we = min(n, wb + per);
}

// Rebuilds the slot pairs listed in fp[0, nf) from the current clusters and
// appends a full work entry for each valid candidate at I.work[base...).
// Returns the number of entries appended.
template <int NT>
__device__ int rebuild_pairs(const Topo &T, const State &S, const Search &X, const Inc &I, int n, const int *fp, int nf,
                             int base, int *smi) {
    int added = 0;
    for (int i0 = 0; i0 < nf; i0 += NT) {
        const int i = i0 + threadIdx.x;
        Cand c[2];
        c[0].s = c[1].s = -1;
        int cnt = 0;
        if (i < nf) {
            const int w = fp[i];
            I.qpar[w] = slot_geometry(T, S, n, w, c[0], c[1]);
            for (int d = 0; d < 2; ++d) {
                X.slot[2 * w + d] = c[d];
                if (c[d].s >= 0) ++cnt;
                else {
                    I.viol[2 * w + d] = kIncDead;
                    st128(I.acc + 4 * (size_t)w + 2 * d, 0);
                }
            }
        }
        int tot = 0;
        int off = block_excl_scan<NT>(cnt, &tot, smi);
        if (i < nf) {
            const int w = fp[i];
            for (int d = 0; d < 2; ++d) {
                if (c[d].s < 0) continue;
                int2 seg[kIncMaxSeg];
                const int ns = full_segments(c[d], S.sn_rank, seg);
                write_entry(I.work + base + added + off, 2 * w + d, 1, ns, seg);
                ++off;
            }
        }
        added += tot;
    }
    return added;
}

}  // namespace

// ---------------------------------------------------------------- the search
template <int NT>
__device__ void inc_run(const Topo &T, const State &S, const Search &X, const Inc &I, Ctrl *C, bool verify) {
    __shared__ __align__(16) EvalSmem E;
    __shared__ __align__(16) Min3 sm3[NT / 32];
    __shared__ int smi[NT / 32];
    __shared__ double smd[NT / 32];
    __shared__ Win h;
    __shared__ unsigned long long s_sfx[2];     // SMICE of the committed state, fixed point
    const int n = T.n, L = T.L, tid = threadIdx.x;
    const double margin = C->margin;
    const int max_merges = C->max_merges;
    const bool prof = C->profile != 0;
    const u128 tau_fx = to_fx(C->tau);
    if (C->done || C->t >= max_merges) return;
    int t = 0, ns = n;
    if (tid == 0) { s_sfx[0] = 0ull; s_sfx[1] = 0ull; }     // every MICE starts at 0
    unsigned long long tp = 0;
    auto stamp = [&](int i) {
        if (prof && tid == 0) { const unsigned long long now = gtimer_inc(); C->phase_ns[i] += now - tp; tp = now; }
    };
    long long terms = 0;

    // ---- every slot pair from the initial clusters (all singletons), every term
    for (int w = tid; w < n; w += NT) I.fpair[w] = w;
    __syncthreads();
    {
        const int ne = rebuild_pairs<NT>(T, S, X, I, n, I.fpair, n, 0, smi);
        __syncthreads();
        terms += eval_entries<NT>(T, S, X, I, n, L, margin, 0, ne, false, -1, S.sn_list[0], S.sn_list[0], I.acc,
                                  I.viol, &E, smi);
    }
    if (prof && tid == 0) tp = gtimer_inc();

    for (;;) {
        if (t >= max_merges) {
            if (tid == 0) { C->done = 1; C->stop_reason = 0; }
            break;
        }
        const int *list_old = S.sn_list[t & 1];
        int *list_new = S.sn_list[(t + 1) & 1];
        // ============================================================ selection
        u128 best = ~(u128)0, dummy = ~(u128)0;
        unsigned long long dmy = ~0ull;
        int nvalid = 0;
        for (int c = tid; c < 2 * n; c += NT) {
            const int v = I.viol[c];
            if (v >= kIncDead) continue;
            ++nvalid;
            if (v == 0) {
                const u128 k = okey(ld128(I.acc + 2 * (size_t)c));
                best = k < best ? k : best;
            }
        }
        nvalid = block_sum_int<NT>(nvalid, smi);
        block_min3<NT>(best, dummy, dmy, sm3);
        if (tid == 0) {
            C->candidates += nvalid;
            C->iters += 1;
            X.dec_ncand[t] = nvalid;
        }
        const double s_cur = fx_to_d(ld128(s_sfx));
        if (t < X.rec_iters) {
            // every candidate's SMICE (+inf when infeasible), compacted in slot order
            int base = 0;
            for (int c0 = 0; c0 < 2 * n; c0 += NT) {
                const int c = c0 + tid;
                const int v = c < 2 * n ? I.viol[c] : kIncDead;
                const int f = v < kIncDead ? 1 : 0;
                int tot = 0;
                const int o = block_excl_scan<NT>(f, &tot, smi) + base;
                if (f) {
                    const Cand &cc = X.slot[c];
                    const size_t at = (size_t)t * 2 * n + o;
                    X.rec_s[at] = T.orig[cc.s];
                    X.rec_r[at] = T.orig[cc.r];
                    X.rec_score[at] = v == 0 ? s_cur + fx_to_d(ld128(I.acc + 2 * (size_t)c)) : INFINITY;
                    X.rec_bound[at] = 0.0;
                }
                base += tot;
            }
            if (tid == 0) X.rec_count[t] = nvalid;
        }
        if (best == ~(u128)0) {                          // nothing feasible
            if (tid == 0) { C->done = 1; C->stop_reason = 1; }
            break;
        }
        const u128 m = best ^ kSignBit;
        const u128 edge = m + tau_fx;
        const u128 ek = okey(edge);
        // band: smallest (r, s) key with its slot; gap: smallest score above the band
        u128 kp = ~(u128)0, gk = ~(u128)0;
        for (int c = tid; c < 2 * n; c += NT) {
            if (I.viol[c] != 0) continue;
            const u128 k = okey(ld128(I.acc + 2 * (size_t)c));
            if (k <= ek) {
                const u128 key = ((u128)X.slot[c].key << 32) | (u128)(unsigned)c;
                kp = key < kp ? key : kp;
            } else {
                gk = k < gk ? k : gk;
            }
        }
        block_min3<NT>(kp, gk, dmy, sm3);
        stamp(0);
        const int ws = (int)(unsigned)(kp & 0xffffffffu);
        // ============================================================ the merge's changed set
        if (tid == 0) {
            const Cand w = X.slot[ws];
            h.slot = ws; h.s = w.s; h.r = w.r; h.a = w.a; h.dir = w.dir; h.fixed = w.fixed;
            h.w1lo = w.js; h.w1hi = w.js + w.ns; h.w2lo = w.jr; h.w2hi = w.jr + w.nr;
            h.rtop = S.top[w.r];
            h.rtop_end = h.rtop + T.sz[h.rtop];
            h.jr = S.sn_rank[w.r];
            h.q1lo = w.ns > 0 ? S.sn_rank[w.js] : 0;
            h.q1hi = w.ns > 0 ? S.sn_rank[w.js + w.ns] : 0;
            h.q2lo = w.nr > 0 ? S.sn_rank[w.jr] : 0;
            h.q2hi = w.nr > 0 ? S.sn_rank[w.jr + w.nr] : 0;
            h.npos = (h.q1hi - h.q1lo) + (h.q2hi - h.q2lo) + w.fixed;
            X.dec_s[t] = T.orig[w.s];
            X.dec_r[t] = T.orig[w.r];
            X.dec_gap[t] = (gk == ~(u128)0) ? INFINITY : fx_to_d((gk ^ kSignBit) - edge);
        }
        __syncthreads();
        const Win hw = h;
        // ---- which candidates change: rebuilt pairs (next to s* or r*) and changed terms
        int wb, we;
        my_pairs<NT>(n, wb, we);
        int nf_mine = 0, np_mine = 0;
        for (int w = wb; w < we; ++w) {
            if (w == hw.r) continue;
            const int qp = I.qpar[w];
            if (w == hw.s || qp == hw.r || qp == hw.s) { ++nf_mine; continue; }
            for (int d = 0; d < 2; ++d) {
                const Cand &c = X.slot[2 * w + d];
                if (c.s < 0) continue;
                int2 seg[kIncMaxSeg];
                if (changed_segments(c, hw, S.sn_rank, seg) > 0) ++np_mine;
            }
        }
        int nf_tot = 0, np_tot = 0;
        int fo = block_excl_scan<NT>(nf_mine, &nf_tot, smi);
        int po = block_excl_scan<NT>(np_mine, &np_tot, smi);
        for (int w = wb; w < we; ++w) {
            if (w == hw.r) continue;
            const int qp = I.qpar[w];
            if (w == hw.s || qp == hw.r || qp == hw.s) { I.fpair[fo++] = w; continue; }
            for (int d = 0; d < 2; ++d) {
                const Cand &c = X.slot[2 * w + d];
                if (c.s < 0) continue;
                int2 seg[kIncMaxSeg];
                const int k = changed_segments(c, hw, S.sn_rank, seg);
                if (k > 0) write_entry(I.work + po++, 2 * w + d, 0, k, seg);
            }
        }
        __syncthreads();
        stamp(1);
        // ============================================================ terms before the merge
        // the merge's own new values (state before the merge) into the scratch
        {
            const Cand wc = X.slot[ws];
            const int n1 = hw.q1hi - hw.q1lo, n2 = hw.q2hi - hw.q2lo;
            for (int j = tid; j < hw.npos; j += NT) {
                const int k = j < n1 ? list_old[hw.q1lo + j] : (j < n1 + n2 ? list_old[hw.q2lo + j - n1] : wc.s);
                if (k == wc.r) continue;
                u128 fx;
                int nv;
                term(T, S, n, L, wc, k, margin, &fx, &nv, I.cbuf + (size_t)j * 10 * L);
            }
        }
        terms += eval_entries<NT>(T, S, X, I, n, L, margin, 0, np_tot, true, hw.r, list_old, list_new, I.acc, I.viol,
                                  &E, smi);
        stamp(2);
        // ============================================================ the merge (FP64)
        {
            const int n1 = hw.q1hi - hw.q1lo, n2 = hw.q2hi - hw.q2lo;
            for (int j = tid; j < hw.npos; j += NT) {
                const bool fx = j >= n1 + n2;
                const int k = j < n1 ? list_old[hw.q1lo + j] : (j < n1 + n2 ? list_old[hw.q2lo + j - n1] : hw.s);
                if (k == hw.r) continue;
                const double *cb = I.cbuf + (size_t)j * 10 * L;
                const unsigned phk = T.ph[k];
                for (int l = 0; l < L; ++l) {
                    for (int p = 0; p < 3; ++p) {
                        if (!(phk >> p & 1u)) continue;
                        const size_t ik = sidx(l, p, k, n);
                        if (!fx) {
                            S.vcur[ik] = make_double2(cb[(l * 3 + p) * 3 + 0], cb[(l * 3 + p) * 3 + 1]);
                            S.mcur[ik] = cb[(l * 3 + p) * 3 + 2];
                        }
                        if (k == hw.s) {
                            const size_t ir = sidx(l, p, hw.r, n);
                            S.hi[ik] = fmax(S.hi[ik], S.hi[ir]);
                            S.lo[ik] = fmin(S.lo[ik], S.lo[ir]);
                        }
                    }
                    S.mice[(size_t)l * n + k] = cb[9 * L + l];
                }
            }
            // r's members join s; ranks past r drop by one; the new super-node list
            for (int b = hw.rtop + tid; b < hw.rtop_end; b += NT)
                if (S.label[b] == hw.r) S.label[b] = hw.s;
            for (int b = hw.r + 1 + tid; b <= n; b += NT) S.sn_rank[b] -= 1;
            for (int j = tid; j < ns - 1; j += NT) list_new[j] = list_old[j + (j >= hw.jr ? 1 : 0)];
            if (tid == 0) {
                const unsigned phr = T.ph[hw.r];
                for (int l = 0; l < L; ++l) {
                    for (int q = 0; q < 3; ++q)
                        if (phr >> q & 1u) {
                            const size_t is = sidx(l, q, hw.s, n), ir = sidx(l, q, hw.r, n);
                            S.icur[is] = cadd(S.icur[is], S.icur[ir]);
                        }
                    S.mice[(size_t)l * n + hw.r] = 0.0;
                }
                if (hw.dir == 1) {
                    S.top[hw.s] = S.top[hw.r];
                    S.ptop[hw.s] = S.ptop[hw.r];
                }
                const u128 sfx = ld128(s_sfx) + ld128(I.acc + 2 * (size_t)ws);
                st128(s_sfx, sfx);
                X.dec_score[t] = fx_to_d(sfx);
                I.qpar[hw.r] = -1;
            }
            if (tid < 2) {
                X.slot[2 * hw.r + tid].s = -1;
                I.viol[2 * hw.r + tid] = kIncDead;
            }
        }
        __syncthreads();
        ns -= 1;
        stamp(3);
        // ---- largest MICE of the reduced network
        {
            double mx = 0.0;
            for (int j = tid; j < ns; j += NT) {
                const int k = list_new[j];
                for (int l = 0; l < L; ++l) mx = fmax(mx, S.mice[(size_t)l * n + k]);
            }
            mx = block_max_d<NT>(mx, smd);
            if (tid == 0) X.dec_maxerr[t] = mx;
        }
        // ============================================================ terms after the merge
        const int nfe = rebuild_pairs<NT>(T, S, X, I, n, I.fpair, nf_tot, np_tot, smi);
        __syncthreads();
        stamp(4);
        terms += eval_entries<NT>(T, S, X, I, n, L, margin, 0, np_tot + nfe, false, hw.r, list_old, list_new,
                                  I.acc, I.viol, &E, smi);
        stamp(5);
        t += 1;
        if (verify) {
            // every candidate again from scratch; the carried scores must match bit for bit
            int cnt = 0;
            for (int w0 = 0; w0 < n; w0 += NT) {
                const int w = w0 + tid;
                int c2 = 0;
                if (w < n) c2 = (X.slot[2 * w].s >= 0) + (X.slot[2 * w + 1].s >= 0);
                int tot = 0;
                int o = block_excl_scan<NT>(c2, &tot, smi) + cnt;
                if (w < n)
                    for (int d = 0; d < 2; ++d) {
                        const Cand &c = X.slot[2 * w + d];
                        if (c.s < 0) continue;
                        int2 seg[kIncMaxSeg];
                        const int k = full_segments(c, S.sn_rank, seg);
                        write_entry(I.work + o++, 2 * w + d, 1, k, seg);
                    }
                cnt += tot;
            }
            __syncthreads();
            eval_entries<NT>(T, S, X, I, n, L, margin, 0, cnt, false, -1, list_new, list_new, I.vacc, I.vviol, &E,
                             smi);
            int bad = 0;
            for (int c = tid; c < 2 * n; c += NT) {
                if (X.slot[c].s < 0) continue;
                if (I.viol[c] != I.vviol[c] || ld128(I.acc + 2 * (size_t)c) != ld128(I.vacc + 2 * (size_t)c)) ++bad;
            }
            bad = block_sum_int<NT>(bad, smi);
            if (tid == 0 && bad) C->inc_mismatch += bad;
        }
    }
    if (tid == 0) {
        C->t = t;
        C->n_super = ns;
        C->s_cur = fx_to_d(ld128(s_sfx));
        if (prof) C->sweep_flops = (double)terms;     // terms evaluated (profile mode)
    }
}

template <int NT>
__global__ void __launch_bounds__(NT, 1) k_search_inc(Topo T, State S, Search X, Inc I, Ctrl *C, int verify) {
    inc_run<NT>(T, S, X, I, C, verify != 0);
}

// One CTA per feeder, feeders in the order given (largest first).
template <int NT>
__global__ void __launch_bounds__(NT) k_search_inc_batch(const BatchFeeder *fd, const int *order, int nf) {
    __shared__ Topo sT;
    __shared__ State sS;
    __shared__ Search sX;
    __shared__ Inc sI;
    const int q = blockIdx.x;
    if (q >= nf) return;
    const int f = order[q];
    if (threadIdx.x == 0) {
        sT = fd[f].T;
        sS = fd[f].S;
        sX = fd[f].X;
        sI = fd[f].I;
    }
    __syncthreads();
    Ctrl *C = fd[f].C;
    const bool ok = *fd[f].setup_err == 0;
    if (ok) inc_run<NT>(sT, sS, sX, sI, C, false);
    __syncthreads();
    for (int i = threadIdx.x; i < sT.n; i += NT) fd[f].super_out[i] = ok ? sT.orig[sS.label[sT.pre[i]]] : -1;
    if (threadIdx.x == 0) {
        const int t = ok ? C->t : 0;
        *fd[f].max_err = t > 0 ? sX.dec_maxerr[t - 1] : 0.0;
    }
}

constexpr int kIncThreads = 1024;           // one feeder on one SM
constexpr int kIncBatchThreads = 512;       // batches: several feeders per SM

cudaError_t launch_search_inc(Topo T, State S, Search X, Inc I, Ctrl *C, int verify, cudaStream_t st) {
    k_search_inc<kIncThreads><<<1, kIncThreads, 0, st>>>(T, S, X, I, C, verify);
    return cudaGetLastError();
}

cudaError_t launch_search_inc_batch(const BatchFeeder *fd, const int *order, int nf, cudaStream_t st) {
    if (nf <= 0) return cudaSuccess;
    k_search_inc_batch<kIncBatchThreads><<<nf, kIncBatchThreads, 0, st>>>(fd, order, nf);
    return cudaGetLastError();
}

}  // namespace okr
