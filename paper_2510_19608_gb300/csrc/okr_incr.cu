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
// Exactness.  Carried sums are 128-bit fixed-point integers (units of 2^-100
// p.u.).  A term is converted by a fixed function of its bits; integer
// addition is associative, so removing a term's old value and adding its new
// one gives exactly the sum a fresh evaluation of every term gives, in any
// order.  The old value is recomputed from the unchanged inputs by the same
// arithmetic, every operation of which is explicitly rounded (no contraction
// into fused multiply-adds, whose use could differ between inlined copies), so
// it is bit-identical to the value added earlier.  Counts of terms above the
// margin are carried the same way.
// Engine 3 checks the carried values against a fresh evaluation after every
// merge.
//
// Precision 0 carries FP64 terms and selects on them exactly: the minimum m
// over feasible candidates, the tie band D <= m + tau, the smallest (r, s) key
// in it.  Precision 1 (GB300's FP64 rate is a small fraction of its FP32 rate)
// carries FP32 terms of the same quantities with the rigorous per-term bound
// of okr_persist.cu, summed into a bound B(c) >= |D32 - D64|, and counts of
// terms surely / possibly above the margin.  The selection of okr_persist.cu's
// screen then decides the FP64 winner, or names the few candidates whose FP64
// score it needs; those are evaluated in FP64 from scratch.  Merges are always
// applied in FP64.
//
// Execution.  One CTA runs one feeder's whole search; its steps are separated
// by __syncthreads only (no grid barrier, no device-side wait).  A term is
// evaluated by a group of lanes, one per (scenario, phase).  A batch runs one
// CTA per feeder.  Each merge takes four steps: selection; the changed set
// (beside it, the merge's own FP64 evaluation into a scratch, and a map of its
// positions); the merge's score change and topology, and beside it the
// rebuilt candidates (which read the clusters through the merge's view); one
// pass over the changed terms, which evaluates each term before the merge (the
// state as stored) and after it (the stored state overlaid with the scratch's
// new values) in the same lane group and adds the difference.  The new values
// and ranks are written back to the state at the end of that pass.
#include "okr_internal.cuh"
#include "okr_kernels.cuh"

namespace okr {

namespace {

typedef unsigned __int128 u128;

constexpr int kFxShift = 100;               // fixed point: value * 2^100
constexpr u128 kSignBit = (u128)1 << 127;
constexpr u128 kNone = ~(u128)0;
constexpr float kU32 = 5.9604645e-08f;      // 2^-24

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

// The same truncation for a float, with integer operations only (FP64
// instructions are scarce on this GPU): equal to to_fx((double)f).
__device__ __forceinline__ u128 to_fx32(float f) {
    const unsigned b = __float_as_uint(f);
    int e = (int)((b >> 23) & 0xff);
    if (e == 0xff) return 0;
    unsigned m = b & 0x7fffffu;
    if (e == 0) e = 1;
    else m |= 1u << 23;
    // f = m * 2^(e - 150), so f * 2^100 = m * 2^(e - 50)
    const int sh = e - 150 + kFxShift;
    u128 v;
    if (sh >= 0) v = sh >= 128 ? (u128)0 : ((u128)m << sh);
    else v = sh <= -32 ? (u128)0 : (u128)(m >> (-sh));
    return (b >> 31) ? (u128)0 - v : v;
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
__device__ __forceinline__ u128 umin(u128 a, u128 b) { return a < b ? a : b; }

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
// Every reduction: warps reduce with shuffles, warp 0 reduces the warps'
// partials and publishes the result; two barriers.
struct Red {
    u128 a, b, c;
    int i;
};

__device__ __forceinline__ Red red_op(Red x, Red y) {
    Red r;
    r.a = umin(x.a, y.a);
    r.b = umin(x.b, y.b);
    r.c = umin(x.c, y.c);
    r.i = x.i + y.i;
    return r;
}
__device__ __forceinline__ Red red_shfl(Red x, int o) {
    Red r;
    r.a = shfl_xor_u128(x.a, o);
    r.b = shfl_xor_u128(x.b, o);
    r.c = shfl_xor_u128(x.c, o);
    r.i = __shfl_xor_sync(0xffffffffu, x.i, o);
    return r;
}

// Three 128-bit minima and one int sum over the block.
template <int NT>
__device__ __forceinline__ Red block_red(Red v, Red *sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = red_op(v, red_shfl(v, o));
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    if (wid == 0) {
        Red x;
        x.a = x.b = x.c = kNone;
        x.i = 0;
        if (lane < NT / 32) x = sm[lane];
        for (int o = 16; o > 0; o >>= 1) x = red_op(x, red_shfl(x, o));
        if (lane == 0) sm[32] = x;
    }
    __syncthreads();
    return sm[32];
}

// The same with 64-bit minima (precision 1: every key fits 64 bits).
struct Red64 {
    unsigned long long a, b, c;
    int i;
};

template <int NT>
__device__ __forceinline__ Red64 block_red64(Red64 v, Red64 *sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    auto op = [](Red64 x, Red64 y) {
        Red64 r;
        r.a = x.a < y.a ? x.a : y.a;
        r.b = x.b < y.b ? x.b : y.b;
        r.c = x.c < y.c ? x.c : y.c;
        r.i = x.i + y.i;
        return r;
    };
    auto shfl = [](Red64 x, int o) {
        Red64 r;
        r.a = __shfl_xor_sync(0xffffffffu, x.a, o);
        r.b = __shfl_xor_sync(0xffffffffu, x.b, o);
        r.c = __shfl_xor_sync(0xffffffffu, x.c, o);
        r.i = __shfl_xor_sync(0xffffffffu, x.i, o);
        return r;
    };
    for (int o = 16; o > 0; o >>= 1) v = op(v, shfl(v, o));
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    if (wid == 0) {
        Red64 x;
        x.a = x.b = x.c = ~0ull;
        x.i = 0;
        if (lane < NT / 32) x = sm[lane];
        for (int o = 16; o > 0; o >>= 1) x = op(x, shfl(x, o));
        if (lane == 0) sm[32] = x;
    }
    __syncthreads();
    return sm[32];
}

// Selection reductions of precision 1 in one barrier: each warp reduces with
// redux.sync (a 64-bit minimum as the minimum of the high words, then of the
// low words among the lanes that hold it), lane 0 folds the warp's result
// into the shared accumulator with atomics, one barrier, every thread reads
// it.  The accumulator must hold the identity (reset_sel) before the first
// atomic; the caller resets it only after a later barrier.
__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
    const unsigned hi = (unsigned)(v >> 32);
    const unsigned mh = __reduce_min_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_min_sync(0xffffffffu, hi == mh ? (unsigned)v : 0xffffffffu);
    return ((unsigned long long)mh << 32) | ml;
}
__device__ __forceinline__ void reset_sel(Red64 *acc) {
    acc->a = acc->b = acc->c = ~0ull;
    acc->i = 0;
}
__device__ __forceinline__ Red64 block_sel64(Red64 v, Red64 *acc) {
    Red64 w;
    w.a = warp_min64(v.a);
    w.b = warp_min64(v.b);
    w.c = warp_min64(v.c);
    w.i = (int)__reduce_add_sync(0xffffffffu, (unsigned)v.i);
    if ((threadIdx.x & 31) == 0) {
        if (w.a != ~0ull) atomicMin(&acc->a, w.a);
        if (w.b != ~0ull) atomicMin(&acc->b, w.b);
        if (w.c != ~0ull) atomicMin(&acc->c, w.c);
        if (w.i) atomicAdd(&acc->i, w.i);
    }
    __syncthreads();
    return *acc;
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
    if (lane == 31) sm[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int y = lane < NT / 32 ? sm[lane] : 0;
        const int y0 = y;
        for (int o = 1; o < 32; o <<= 1) {
            const int z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        if (lane < NT / 32) sm[lane] = y - y0;      // exclusive offsets of the warps
        if (lane == 31) sm[32] = y;                 // total
    }
    __syncthreads();
    *total = sm[32];
    return sm[wid] + x - v;
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

// The clusters as a merge (s*, r*) leaves them, read while that merge is being
// written: r*'s members belong to s*; with dir = 1 s* takes r*'s top; ranks
// past r* drop by one.  Either value of an entry the merge is rewriting reads
// the same through the view, and the ranks are rewritten only after the
// rebuild.  With no merge (s = -1) the state as stored.
struct View {
    int s, r, dir;
    __device__ __forceinline__ int label(const State &S, int b) const {
        const int l = S.label[b];
        return l == r ? s : l;
    }
    __device__ __forceinline__ int top(const State &S, int w) const {
        return (w == s && dir == 1) ? S.top[r] : S.top[w];
    }
    __device__ __forceinline__ int ptop(const State &S, int w) const {
        return (w == s && dir == 1) ? S.ptop[r] : S.ptop[w];
    }
};
__device__ __forceinline__ View no_view() {
    View v;
    v.s = v.r = -1;
    v.dir = 0;
    return v;
}

// The two candidates of the quotient edge above super-node w, from the current
// clusters: x = super-node holding the parent of w's top, a = lca(x, w), cw and
// cx the children of a toward w and x.  Slot 2w: w's cluster joins x (s = x,
// r = w); slot 2w + 1: x's cluster joins w (s = w, r = x; never the slack's
// cluster).  js/ns and jr/nr hold the s-side and r-side subtrees as BUS
// ranges [j, j + size) (preorder ids); fixed = 1 when s is the common ancestor.
// Returns x (-1 for the slack's cluster, which has no edge above it).
__device__ int slot_geometry(const Topo &T, const State &S, const View &V, int n, int w, Cand &c0, Cand &c1) {
    c0.s = -1;
    c1.s = -1;
    const int pb = V.ptop(S, w);
    if (pb < 0 || V.label(S, w) != w) return -1;
    const int tw = V.top(S, w);
    const int x = V.label(S, pb);
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

// ---------------------------------------------------------------- term groups
// A term (candidate c, position k) is evaluated by a group of G = 4 Lp lanes
// (Lp = scenarios rounded up to a power of two): lane gl takes scenario
// l = gl / 4 and phase p = gl % 4 (p = 3 idles).  Every lane of the warp calls
// the group function (it shuffles); the results are the group's sums over its
// scenarios (every lane holds them).
//
// A group evaluates its term on one or two states, e in [e_lo, e_hi) (the
// same range for every group of a warp): e = 0, the state as stored; e = 1,
// the state after the merge in progress, whose new values (voltage,
// magnitude, extremes, MICE of the merge's positions) are not yet written
// back and are read through the overlay.  With both, the result is the term
// on state 1 minus the term on state 0.  v_old / v_new say whether the group
// has a term on state 0 / 1.  The geometry (the voltage change the candidate
// causes) is the same on both states and is computed once.  The arithmetic of
// a term on one state's inputs (term_arith32, term_arith64) rounds every
// operation explicitly, so equal inputs give bit-equal results in every
// inlined copy.

// The merge in progress, as the terms after it see it: map[x] = 1 + the index
// of super-node x among the merge's positions (0: unchanged), whose new values
// the merge's own evaluation left in cbuf (per position: per (l, p) the new
// voltage x, y and magnitude; per l the new MICE).  Positions from nfree on
// are the fixed s (its voltage does not move).  s* takes r*'s extremes.
struct Ovl {
    const unsigned short *map;
    const double *cbuf;
    int s, r, nfree;
};

// A position's FP32 copies in its scratch (after the 10 L FP64 values): per
// (l, p) the voltage, and the extremes relative to the magnitude; per l the MICE.
__device__ __forceinline__ float4 *cb_f4(const double *cb_pos, int L, int l, int p) {
    return reinterpret_cast<float4 *>(const_cast<double *>(cb_pos) + 10 * L) + (l * 3 + p);
}
__device__ __forceinline__ float *cb_mice32(const double *cb_pos, int L, int l) {
    return reinterpret_cast<float *>(const_cast<double *>(cb_pos) + 10 * L) + 12 * L + l;
}

// FP64 state of super-node x, phase p, scenario l on state e (0 stored, 1 overlay).
__device__ __forceinline__ void at64(const State &S, const Ovl &O, int e, int x, int l, int p, int n, int L,
                                     bool need_v, double2 *v, double *hh, double *ll) {
    const size_t ix = sidx(l, p, x, n);
    const int j = e ? (int)O.map[x] - 1 : -1;
    double h = S.hi[ix], lo = S.lo[ix];
    if (j >= 0 && x == O.s) {
        const size_t irs = sidx(l, p, O.r, n);
        h = fmax(h, S.hi[irs]);
        lo = fmin(lo, S.lo[irs]);
    }
    *hh = h;
    *ll = lo;
    if (need_v) {
        if (j >= 0 && j < O.nfree) {
            const double *cb = O.cbuf + (size_t)j * kIncCbStride * L + (l * 3 + p) * 3;
            *v = make_double2(cb[0], cb[1]);
        } else {
            *v = S.vcur[ix];
        }
    }
}
__device__ __forceinline__ double mice64(const State &S, const Ovl &O, int e, int x, int l, int n, int L) {
    const int j = e ? (int)O.map[x] - 1 : -1;
    return j >= 0 ? O.cbuf[(size_t)j * kIncCbStride * L + 9 * L + l] : S.mice[(size_t)l * n + x];
}

// FP32 copies (voltage, extremes relative to the magnitude) and the FP64
// magnitude of super-node x on state e: the values the write-back stores.
__device__ __forceinline__ void at32(const State &S, const Ovl &O, int e, int x, int l, int p, int n, int L,
                                     bool need_v, bool need_mc, float2 *v, float *hr, float *lr, double *mc) {
    const size_t ix = sidx(l, p, x, n);
    const int j = e ? (int)O.map[x] - 1 : -1;
    if (j < 0) {
        *hr = S.hr32[ix];
        *lr = S.lr32[ix];
        if (need_v) *v = S.v32[ix];
        if (need_mc) *mc = S.mcur[ix];
        return;
    }
    // the FP32 copies the merge's evaluation derived (the write-back stores the same)
    const double *cbp = O.cbuf + (size_t)j * kIncCbStride * L;
    const float4 f = *cb_f4(cbp, L, l, p);
    *hr = f.z;
    *lr = f.w;
    if (need_v) *v = make_float2(f.x, f.y);
    if (need_mc) *mc = j >= O.nfree ? S.mcur[ix] : cbp[(l * 3 + p) * 3 + 2];
}
__device__ __forceinline__ float mice32(const State &S, const Ovl &O, int e, int x, int l, int n, int L) {
    const int j = e ? (int)O.map[x] - 1 : -1;
    return j >= 0 ? *cb_mice32(O.cbuf + (size_t)j * kIncCbStride * L, L, l) : S.mice32[(size_t)l * n + x];
}

// The arithmetic of one FP64 term on one state's inputs (every lane of the
// warp calls it: it shuffles).  Explicitly rounded operations: equal inputs
// give bit-equal results wherever it is inlined.
struct In64 {
    double2 v;
    double h, lo, hr, lr, mo, mr;
};
struct Out64 {
    u128 t;
    int tv;
};
__device__ __forceinline__ Out64 term_arith64(In64 x, double2 dv, bool one, bool moves, bool is_s, bool lvp0,
                                              double margin, double *out, int l, int p, int L) {
    // every operation explicitly rounded (no contraction): each inlined copy
    // gives the same bits for the same inputs
    double em = 0.0;
    if (one) {
        double2 v = x.v;
        if (moves) v = make_double2(__dadd_rn(v.x, dv.x), __dadd_rn(v.y, dv.y));
        const double mag = cmag(v);
        double h = x.h, lo = x.lo;
        if (is_s) {
            h = fmax(h, x.hr);
            lo = fmin(lo, x.lr);
        }
        em = fmax(__dsub_rn(h, mag), __dsub_rn(mag, lo));
        if (out) {
            out[(l * 3 + p) * 3 + 0] = v.x;
            out[(l * 3 + p) * 3 + 1] = v.y;
            out[(l * 3 + p) * 3 + 2] = mag;
        }
    }
    double m = fmax(em, __shfl_xor_sync(0xffffffffu, em, 1));
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 2));
    Out64 r;
    r.t = 0;
    r.tv = 0;
    if (lvp0) {
        if (out) out[9 * L + l] = m;
        double dd = __dsub_rn(m, x.mo);
        if (is_s) dd = __dsub_rn(dd, x.mr);
        r.t = to_fx(dd);
        r.tv = (m > margin) ? 1 : 0;
    }
    return r;
}

// FP64 term.  d = sum over l of fixed(new MICE - MICE_k [- MICE_r]); nv = scenarios
// whose new MICE exceeds the margin.  out != nullptr (state 0 only): the new
// voltage and magnitude per (l, p) and the new MICE per l (the merge).
__device__ __forceinline__ void group_term64(const Topo &T, const State &S, const uint8_t *ph, int n, int L, int G,
                                             const Cand &c, int k, int e_lo, int e_hi, bool v_old, bool v_new,
                                             const Ovl &O, int gl, double margin, double *out, u128 *d_out,
                                             int *nv_out) {
    const bool valid = v_old || v_new;
    const int l = gl >> 2, p = gl & 3;
    const bool lv = valid && l < L;
    const unsigned phk = valid ? ph[k] : 0u, phr = valid ? ph[c.r] : 0u;
    const bool on = lv && p < 3 && (phk >> p & 1u);
    const bool is_s = (k == c.s);
    const bool fixed = is_s && c.fixed;
    const bool sside = (k >= c.js && k < c.js + c.ns);
    const bool moves = on && !fixed;
    const int li = lv ? l : 0, pi = p < 3 ? p : 0;
    // the inputs of state e, loaded ahead of the arithmetic that uses them
    typedef In64 St;
    auto fetch = [&](int e, St &x) {
        const bool ve = e == 0 ? v_old : v_new;
        x.v = make_double2(0.0, 0.0);
        x.h = x.lo = x.mo = x.mr = 0.0;
        x.hr = -INFINITY;
        x.lr = INFINITY;
        if (on && ve) {
            at64(S, O, e, k, li, pi, n, L, true, &x.v, &x.h, &x.lo);
            if (is_s) at64(S, O, e, c.r, li, pi, n, L, false, nullptr, &x.hr, &x.lr);
        }
        if (lv && ve && p == 0) {
            x.mo = mice64(S, O, e, k, l, n, L);
            if (is_s) x.mr = mice64(S, O, e, c.r, l, n, L);
        }
    };
    St cur;
    fetch(e_lo, cur);
    // the voltage change at k (the same on both states)
    double2 dv = make_double2(0.0, 0.0);
    if (moves) {
        const int y = __ldg(T.lca + (size_t)(sside ? c.s : c.r) * n + k);
        double2 iq[3], za[3];
        for (int q = 0; q < 3; ++q) {
            iq[q] = (phr >> q & 1u) ? S.icur[sidx(li, q, c.r, n)] : make_double2(0.0, 0.0);
            za[q] = __ldg(T.zc + (size_t)c.a * 9 + pi * 3 + q);
        }
        const double2 *zy = T.zc + (size_t)y * 9 + pi * 3;
        for (int q = 0; q < 3; ++q) {
            if (!(phr >> q & 1u)) continue;
            const double2 zyq = __ldg(zy + q);
            const double2 g = sside ? csub(zyq, za[q]) : csub(za[q], zyq);
            dv = cadd(dv, cmul(g, iq[q]));
        }
    }
    u128 d = 0;
    int nv = 0;
#pragma unroll 1
    for (int e = e_lo; e < e_hi; ++e) {
        const bool ve = e == 0 ? v_old : v_new;
        const bool one = on && ve;
        St nxt = cur;
        if (e + 1 < e_hi) fetch(e + 1, nxt);
        const Out64 r = term_arith64(cur, dv, one, moves, is_s, lv && ve && p == 0, margin, out, l, p, L);
        cur = nxt;
        if (e == 1 || e_hi - e_lo == 1) { d += r.t; nv += r.tv; }
        else { d -= r.t; nv -= r.tv; }
    }
    for (int o = 4; o < G; o <<= 1) {            // the group's sum over its scenarios
        d += shfl_xor_u128(d, o);
        nv += __shfl_xor_sync(0xffffffffu, nv, o);
    }
    *d_out = d;
    *nv_out = nv;
}

// The arithmetic of one FP32 term with its bound on one state's inputs (every
// lane of the warp calls it: it shuffles).  Explicitly rounded operations:
// equal inputs give bit-equal results wherever it is inlined.
struct In32 {
    float hr, lr, hrr, lrr, mo, mr;
    float2 v;
    double mck, mcr;
};
struct Out32 {
    u128 td, tb;
    int ts, tm;
};
__device__ __forceinline__ Out32 term_arith32(In32 x, float2 dv, float sdv, bool one, bool moves, bool sterm,
                                              bool lvp0, float margin_lo, float margin_hi) {
    // every operation explicitly rounded (no contraction): each inlined copy
    // gives the same bits for the same inputs
    float em = 0.0f, b = 0.0f;
    if (one) {
        float hr = x.hr, lr = x.lr, hrr = x.hrr, lrr = x.lrr;
        float bx = 0.0f;
        if (sterm) {
            const float dr = (float)__dsub_rn(x.mcr, x.mck);
            hrr = __fadd_rn(hrr, dr);
            lrr = __fadd_rn(lrr, dr);
            hr = fmaxf(hr, hrr);
            lr = fminf(lr, lrr);
            bx = __fmul_rn(2.0f * kU32, __fadd_rn(__fadd_rn(fabsf(hrr), fabsf(lrr)), __fmul_rn(2.0f, fabsf(dr))));
        }
        float delta = 0.0f, bd = 0.0f;
        if (moves) {
            const float2 v = x.v;
            const float s1 = __fadd_rn(__fmul_rn(v.x, dv.x), __fmul_rn(v.y, dv.y));
            const float s2 = __fadd_rn(__fmul_rn(dv.x, dv.x), __fmul_rn(dv.y, dv.y));
            const float num = __fadd_rn(__fmul_rn(2.0f, s1), s2);
            const float wx = __fadd_rn(v.x, dv.x), wy = __fadd_rn(v.y, dv.y);
            const float mv = __fsqrt_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)));
            const float den = __fadd_rn(__fsqrt_rn(__fadd_rn(__fmul_rn(wx, wx), __fmul_rn(wy, wy))), mv);
            delta = __fdiv_rn(num, den);
            const float v1 = __fadd_rn(fabsf(v.x), fabsf(v.y));
            bd = __fmul_rn(kU32, __fadd_rn(__fdiv_rn(__fmul_rn(__fmul_rn(40.0f, __fadd_rn(v1, sdv)), sdv), den),
                                           __fmul_rn(8.0f, fabsf(delta))));
        }
        em = fmaxf(__fsub_rn(hr, delta), __fsub_rn(delta, lr));
        const float ab = __fadd_rn(__fadd_rn(fabsf(hr), fabsf(lr)), fabsf(em));
        b = __fadd_rn(__fadd_rn(__fmul_rn(1.5f, __fadd_rn(__fmul_rn(kU32, ab), bd)), bx), 4e-15f);
    }
    float m = fmaxf(em, __shfl_xor_sync(0xffffffffu, em, 1));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    float bm = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, 1));
    bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, 2));
    Out32 r;
    r.td = r.tb = 0;
    r.ts = r.tm = 0;
    if (lvp0) {
        const float dd = __fsub_rn(__fsub_rn(m, x.mo), x.mr);
        // rounding of MICE_k, MICE_r to FP32 and of the two subtractions; the
        // factor 1.001 covers the rounding of the bound's own arithmetic
        const float am = __fadd_rn(__fadd_rn(fabsf(x.mo), fabsf(x.mr)), fabsf(m));
        const float bl = __fmul_rn(1.001f, __fadd_rn(bm, __fmul_rn(3.0f * kU32, am)));
        r.td = to_fx32(dd);
        r.tb = to_fx32(bl) + 3;             // + the truncations of both terms to fixed point
        r.ts = (__fsub_rd(m, bm) > margin_hi) ? 1 : 0;
        r.tm = (__fadd_ru(m, bm) > margin_lo) ? 1 : 0;
    }
    return r;
}

// FP32 term with a rigorous bound (the screen of okr_persist.cu, per item
// e = max(hr - delta, delta - lr) relative to the cluster's present magnitude).
// d = sum over l of fixed(D32 term); b = sum over l of a fixed-point bound on
// |fixed(D32 term) - fixed(D64 term)|; n_sure = scenarios whose new MICE is
// surely above the margin; n_maybe = scenarios where it may be.  With two
// states each is state 1's minus state 0's.
__device__ __forceinline__ void group_term32(const Topo &T, const State &S, const uint8_t *ph, int n, int L, int G,
                                             const Cand &c, int k, int e_lo, int e_hi, bool v_old, bool v_new,
                                             const Ovl &O, int gl, float margin_lo, float margin_hi, u128 *d_out,
                                             u128 *b_out, int *ns_out, int *nm_out) {
    const bool valid = v_old || v_new;
    const int l = gl >> 2, p = gl & 3;
    const bool lv = valid && l < L;
    const unsigned phk = valid ? ph[k] : 0u, phr = valid ? ph[c.r] : 0u;
    const bool on = lv && p < 3 && (phk >> p & 1u);
    const bool is_s = (k == c.s);
    const bool fixed = is_s && c.fixed;
    const bool sside = (k >= c.js && k < c.js + c.ns);
    const bool sterm = on && is_s && (phr >> p & 1u);
    const bool moves = on && !fixed;
    const int li = lv ? l : 0, pi = p < 3 ? p : 0;
    // the inputs of state e, loaded ahead of the arithmetic that uses them
    typedef In32 St;
    auto fetch = [&](int e, St &x) {
        const bool ve = e == 0 ? v_old : v_new;
        x.hr = x.lr = x.hrr = x.lrr = x.mo = x.mr = 0.0f;
        x.v = make_float2(0.0f, 0.0f);
        x.mck = x.mcr = 0.0;
        if (on && ve) at32(S, O, e, k, li, pi, n, L, moves, sterm, &x.v, &x.hr, &x.lr, &x.mck);
        if (on && ve && sterm) {
            float2 vr;
            at32(S, O, e, c.r, li, pi, n, L, false, true, &vr, &x.hrr, &x.lrr, &x.mcr);
        }
        if (lv && ve && p == 0) {
            x.mo = mice32(S, O, e, k, l, n, L);
            if (is_s) x.mr = mice32(S, O, e, c.r, l, n, L);
        }
    };
    St cur;
    fetch(e_lo, cur);
    // the voltage change at k (the same on both states)
    float2 dv = make_float2(0.0f, 0.0f);
    float sdv = 0.0f;
    if (moves) {
        const int y = __ldg(T.lca + (size_t)(sside ? c.s : c.r) * n + k);
        float2 iq[3], ha[3], la[3];
        for (int q = 0; q < 3; ++q) {
            iq[q] = (phr >> q & 1u) ? S.icur32[sidx(li, q, c.r, n)] : make_float2(0.0f, 0.0f);
            ha[q] = __ldg(T.zh + (size_t)c.a * 9 + pi * 3 + q);
            la[q] = __ldg(T.zlo + (size_t)c.a * 9 + pi * 3 + q);
        }
        const float2 *zhy = T.zh + (size_t)y * 9 + pi * 3, *zly = T.zlo + (size_t)y * 9 + pi * 3;
        for (int q = 0; q < 3; ++q) {
            if (!(phr >> q & 1u)) continue;
            const float2 hy = __ldg(zhy + q), ly = __ldg(zly + q);
            float gx = (hy.x - ha[q].x) + (ly.x - la[q].x);
            float gy = (hy.y - ha[q].y) + (ly.y - la[q].y);
            if (!sside) { gx = -gx; gy = -gy; }
            dv.x = fmaf(gx, iq[q].x, fmaf(-gy, iq[q].y, dv.x));
            dv.y = fmaf(gx, iq[q].y, fmaf(gy, iq[q].x, dv.y));
            sdv = fmaf(fabsf(gx) + fabsf(gy), fabsf(iq[q].x) + fabsf(iq[q].y), sdv);
        }
    }
    u128 d = 0, bb = 0;
    int ns = 0, nm = 0;
#pragma unroll 1
    for (int e = e_lo; e < e_hi; ++e) {
        const bool ve = e == 0 ? v_old : v_new;
        const bool one = on && ve;
        St nxt = cur;
        if (e + 1 < e_hi) fetch(e + 1, nxt);
        const Out32 r = term_arith32(cur, dv, sdv, one, moves, sterm, lv && ve && p == 0, margin_lo, margin_hi);
        cur = nxt;
        if (e == 1 || e_hi - e_lo == 1) { d += r.td; bb += r.tb; ns += r.ts; nm += r.tm; }
        else { d -= r.td; bb -= r.tb; ns -= r.ts; nm -= r.tm; }
    }
    for (int o = 4; o < G; o <<= 1) {            // the group's sums over its scenarios
        d += shfl_xor_u128(d, o);
        bb += shfl_xor_u128(bb, o);
        ns += __shfl_xor_sync(0xffffffffu, ns, o);
        nm += __shfl_xor_sync(0xffffffffu, nm, o);
    }
    *d_out = d;
    *b_out = bb;
    *ns_out = ns;
    *nm_out = nm;
}

// ---------------------------------------------------------------- the changed set of a merge
struct Win {
    int slot, s, r, a, dir, fixed;
    int w1lo, w1hi, w2lo, w2hi;     // bus ranges whose voltages move
    int jr;                         // rank of r before the merge
    int npos;                       // positions of the merge (ranks of the two ranges, r excluded, + fixed s)
    int q1lo, q1hi, q2lo, q2hi;     // their rank ranges before the merge
};

__device__ __forceinline__ bool in_range(int b, int lo, int hi) { return b >= lo && b < hi; }

// The winner's record from its candidate (slot ws) and the super-node ranks.
__device__ __forceinline__ Win make_win(const Cand &w, int ws, const int *rank) {
    Win h;
    h.slot = ws; h.s = w.s; h.r = w.r; h.a = w.a; h.dir = w.dir; h.fixed = w.fixed;
    h.w1lo = w.js; h.w1hi = w.js + w.ns; h.w2lo = w.jr; h.w2hi = w.jr + w.nr;
    h.jr = rank[w.r];
    h.q1lo = w.ns > 0 ? rank[w.js] : 0;
    h.q1hi = w.ns > 0 ? rank[w.js + w.ns] : 0;
    h.q2lo = w.nr > 0 ? rank[w.jr] : 0;
    h.q2hi = w.nr > 0 ? rank[w.jr + w.nr] : 0;
    h.npos = (h.q1hi - h.q1lo) + (h.q2hi - h.q2lo) + w.fixed;
    return h;
}


// Whether candidate c (not next to s* or r*) has a term that reads an input
// the merge h changes: a position in the moved ranges or at s*, r*; its fixed
// s when that cluster changed; its s term when r's MICE changed.
__device__ __forceinline__ bool touched(const Cand &c, const Win &h) {
    auto in_cr = [&](int b) { return in_range(b, c.js, c.js + c.ns) || in_range(b, c.jr, c.jr + c.nr); };
    auto in_w = [&](int b) { return in_range(b, h.w1lo, h.w1hi) || in_range(b, h.w2lo, h.w2hi); };
    const int clo[2] = {c.js, c.jr}, chi[2] = {c.js + c.ns, c.jr + c.nr};
    const int wlo[2] = {h.w1lo, h.w2lo}, whi[2] = {h.w1hi, h.w2hi};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            if (max(clo[i], wlo[j]) < min(chi[i], whi[j])) return true;
    if (in_cr(h.s) || in_cr(h.r)) return true;
    if (c.fixed && (in_w(c.s) || c.s == h.s || c.s == h.r)) return true;
    return in_w(c.r) || c.r == h.s || c.r == h.r;
}

// Rank ranges of the terms of candidate c that read an input the merge h
// changes (c is not next to s* or r*).  Returns their number.
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
__device__ int full_segments(const Cand &c, const int *sn_rank, int2 *seg, int rdead = -1) {
    // rdead >= 0: ranks past bus rdead drop by one (the merge of r* = rdead)
    auto rk = [&](int b) { return sn_rank[b] - (rdead >= 0 && b > rdead ? 1 : 0); };
    int k = 0;
    if (c.ns > 0) {
        const int a = rk(c.js), b = rk(c.js + c.ns);
        if (a < b) seg[k++] = make_int2(a, b);
    }
    if (c.nr > 0) {
        const int a = rk(c.jr), b = rk(c.jr + c.nr);
        if (a < b) seg[k++] = make_int2(a, b);
    }
    if (c.fixed) { const int a = rk(c.s); seg[k++] = make_int2(a, a + 1); }
    return k;
}

__device__ __forceinline__ void write_entry(IncWork *w, int slot, int mode, int nseg, const int2 *seg, const Cand &c) {
    w->slot = slot;
    w->mode = mode;
    w->nseg = nseg;
    w->pad = 0;
    for (int i = 0; i < nseg; ++i) w->seg[i] = seg[i];
    w->s = c.s; w->r = c.r; w->a = c.a;
    w->js = c.js; w->ns = c.ns; w->jr = c.jr; w->nr = c.nr; w->fixed = c.fixed;
}

__device__ __forceinline__ Cand entry_cand(const IncWork &w) {
    Cand c;
    c.s = w.s; c.r = w.r; c.a = w.a; c.dir = 0;
    c.js = w.js; c.ns = w.ns; c.jr = w.jr; c.nr = w.nr;
    c.fixed = w.fixed; c.pad = 0; c.key = 0;
    return c;
}

// Where one search keeps its per-merge data: the first `se` work entries
// (at most kSEMax), the super-node lists (16-bit, by merge parity) and the
// phase masks in shared memory; further entries in global memory.
constexpr int kSEMax = 256;
struct Loc {
    IncWork *wsm, *wgl;
    int se;                     // work entries in shared memory
    unsigned short *lst[2];
    const uint8_t *ph;
    int *rank;                  // [n + 1] rank of each bus's super-node among the super-nodes
    __device__ __forceinline__ IncWork *ent(int i) const { return i < se ? wsm + i : wgl + (i - se); }
};

// ---------------------------------------------------------------- evaluation of work entries
enum Pass {
    kMerge = 0,     // after a merge: mode 0 adds (term after - term before), mode 1 sets every term after
    kInit = 1,      // the stored state, every term of the entries, set
    kFresh = 2,     // carried precision, every term after the merge in progress, into vacc / vviol
    kF64 = 3,       // FP64, every term on the stored state, into vacc / vviol
    kInitPart = 4   // the stored state, every term of the entries (parts of candidates): added to the carried
                    // sums with atomics, the records left to the search
};

// One tile of NT work entries (one per thread): their sums and offsets.
template <int NT>
struct EvalSmem {
    unsigned long long dlo[NT], dhi[NT], blo[NT], bhi[NT];
    int n1[NT], n2[NT];
    int off[NT + 1];
};

// Per-slot selection records (shared memory when they fit, else global):
//   r0 (precision 0): okey(D) of a feasible candidate, kNone otherwise;
//   r1 (precision 1): order-preserving keys of the lower and upper end of the
//       interval that holds the FP64 score, in units of 2^-56 p.u. (lower end
//       rounded down, upper end up); the lower key is ~0 when the candidate is
//       surely infeasible, the upper key when it is not surely feasible (or
//       the slot holds no candidate).  Integer keys keep the selection off the
//       FP64 pipe;
//   tkey: the tie key (caller r, caller s), ~0u for an empty slot;
//   maxm: per super-node, its largest MICE over the scenarios (0 when absorbed);
//   span: per slot pair, what the changed-set scan tests first.
struct Rec {
    u128 *r0;
    ulonglong2 *r1;
    unsigned *tkey;
    double *maxm;
    ushort4 *span;      // per slot pair: bus span [x, y) holding both candidates' ranges, s and r;
                        // z: the quotient parent (0xffff: none); w: empty pair when 0
    // Summaries of blocks of 32 slots (shared memory), so that a selection
    // reads the blocks, not every record: the smallest r0 (precision 0) or the
    // smallest lower and upper keys (precision 1), the slots holding a
    // candidate, and the largest maxm over the block's 16 super-nodes (bit
    // patterns: MICE >= 0 orders like its bits).  A block whose records
    // changed since the last selection is marked dirty and summarised again
    // before the next one.
    void *bsum;         // [nb] u128 (precision 0) or ulonglong2 (precision 1)
    int *bcnt;          // [nb]
    unsigned long long *bmx;    // [nb]
    unsigned char *dirty;       // [nb]
    int nb;
    // (dirty is null in the first evaluation on many CTAs: the search marks every block)
    __device__ __forceinline__ void touch(int sl) const { if (dirty) dirty[sl >> 5] = 1; }
    __device__ __forceinline__ void touch_sn(int k) const { if (dirty) dirty[k >> 4] = 1; }   // maxm of super-node k (slot 2k)
};

constexpr int kKeyShift = 44;                       // 2^-100 -> 2^-56 units
constexpr unsigned long long kKeyNone = ~0ull;

// floor(v / 2^44) of a signed fixed-point value, as an order-preserving key;
// *ok = false when it does not fit 64 bits.
__device__ __forceinline__ unsigned long long key_floor(u128 v, bool *ok) {
    const bool neg = (v & kSignBit) != 0;
    const u128 q = neg ? ~((~v) >> kKeyShift) : (v >> kKeyShift);      // arithmetic shift
    const u128 top = q >> 63;                                          // all sign bits above 63
    *ok = neg ? (top == ((u128)1 << 65) - 1) : (top == 0);
    return (unsigned long long)q ^ 0x8000000000000000ull;
}
__device__ __forceinline__ unsigned long long key_ceil(u128 v, bool *ok) {
    // ceil(v / 2^44) = -floor(-v / 2^44)
    const unsigned long long k = key_floor((u128)0 - v, ok);
    return (unsigned long long)(-(long long)(k ^ 0x8000000000000000ull)) ^ 0x8000000000000000ull;
}
__device__ __forceinline__ long long key_val(unsigned long long k) { return (long long)(k ^ 0x8000000000000000ull); }
__device__ __forceinline__ unsigned long long val_key(long long v) {
    return (unsigned long long)v ^ 0x8000000000000000ull;
}

__device__ __forceinline__ unsigned long long warp_max64(unsigned long long v) { return ~warp_min64(~v); }
__device__ __forceinline__ u128 warp_min128(u128 v) {
    for (int o = 16; o > 0; o >>= 1) v = umin(v, shfl_xor_u128(v, o));
    return v;
}

// Pass B of the selection reads every record when they are in shared memory
// and the feeder has at most this many buses (at most 8 records a thread of
// a 384-thread CTA; measured faster up to 1,000 buses, slower from 2,200);
// otherwise it reads the blocks that may hold a candidate of the tie band, one
// warp per block (or all warps each, when there are at most kFewBlocks).
constexpr int kFlatSelectMax = 1536;
constexpr int kFewBlocks = 8;

// The summaries of the dirty blocks, one warp per block, then a barrier.
template <int NT, int PREC>
__device__ __forceinline__ void refresh_blocks(const Rec &R, int n) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = wid; j < R.nb; j += NT / 32) {
        if (!R.dirty[j]) continue;                      // (the same for the whole warp)
        const int c = 32 * j + lane;
        const bool in = c < 2 * n;
        const unsigned long long mb =
            (in && (c & 1) == 0) ? (unsigned long long)__double_as_longlong(R.maxm[c >> 1]) : 0ull;
        const unsigned cnt = __popc(__ballot_sync(0xffffffffu, in && R.tkey[c] != ~0u));
        const unsigned long long mx = warp_max64(mb);
        if (PREC == 0) {
            const u128 k = warp_min128(in ? R.r0[c] : kNone);
            if (lane == 0) reinterpret_cast<u128 *>(R.bsum)[j] = k;
        } else {
            const ulonglong2 q = in ? R.r1[c] : make_ulonglong2(kKeyNone, kKeyNone);
            const unsigned long long lo = warp_min64(q.x), hi = warp_min64(q.y);
            if (lane == 0) reinterpret_cast<ulonglong2 *>(R.bsum)[j] = make_ulonglong2(lo, hi);
        }
        if (lane == 0) {
            R.bcnt[j] = (int)cnt;
            R.bmx[j] = mx;
            R.dirty[j] = 0;
        }
    }
    __syncthreads();
}

template <int PREC>
__device__ __forceinline__ void set_rec(const Rec &R, int sl, u128 d, u128 b, int viol, int vmay) {
    R.touch(sl);
    if (PREC == 0) {
        R.r0[sl] = (viol == 0) ? okey(d) : kNone;
    } else {
        unsigned long long lo = kKeyNone, hi = kKeyNone;
        if (viol == 0) {
            bool ok;
            lo = key_floor(d - b, &ok);
            if (!ok) lo = ((d - b) & kSignBit) ? 0ull : kKeyNone - 1;
            if (vmay == 0) {
                hi = key_ceil(d + b, &ok);
                if (!ok) hi = kKeyNone;
            }
        }
        R.r1[sl] = make_ulonglong2(lo, hi);
    }
}
template <int PREC>
__device__ __forceinline__ void kill_rec(const Rec &R, int sl) {
    R.touch(sl);
    if (PREC == 0) R.r0[sl] = kNone;
    else R.r1[sl] = make_ulonglong2(kKeyNone, kKeyNone);
    R.tkey[sl] = ~0u;
}

// The merge's own evaluation (FP64, state before the merge): new voltage,
// magnitude and MICE of each of its positions into the scratch.
struct Commit {
    const Win *h;
    Cand wc;
    const unsigned short *list;     // super-nodes before the merge
    const uint8_t *ph;
    Ovl O;                          // (not read: state 0)
    unsigned short *map;            // the overlay map, filled here
};

// Run by warps [warp0, warp0 + nw) only.
__device__ __forceinline__ long long commit_groups(const Topo &T, const State &S, const Inc &I, int n, int L, int G,
                                                   double margin, const Commit &cm, int warp0, int nw) {
    long long items = 0;
    const int lw = ((int)threadIdx.x >> 5) - warp0, gpw = 32 / G, gl = threadIdx.x % G;
    const int gi = lw * gpw + ((int)threadIdx.x & 31) / G, NG = nw * gpw;
    const Win &h = *cm.h;
    const int n1 = h.q1hi - h.q1lo, n2 = h.q2hi - h.q2lo;
    for (int r0 = 0; r0 < h.npos; r0 += NG) {
        if (r0 + lw * gpw >= h.npos) break;             // this warp's groups are all past the end
        const int q = r0 + gi;
        bool valid = q < h.npos;
        int k = cm.wc.s;
        if (valid) {
            k = q < n1 ? cm.list[h.q1lo + q] : (q < n1 + n2 ? cm.list[h.q2lo + q - n1] : cm.wc.s);
            if (k == cm.wc.r) { valid = false; k = cm.wc.s; }
        }
        u128 d;
        int nv;
        group_term64(T, S, cm.ph, n, L, G, cm.wc, k, 0, 1, valid, false, cm.O, gl, margin,
                     valid ? I.cbuf + (size_t)q * kIncCbStride * L : nullptr, &d, &nv);
        if (valid) {
            // the FP32 copies of the new values (what the write-back will store),
            // from the FP64 values this lane has just written
            const int l = gl >> 2, p = gl & 3;
            const double *cb = I.cbuf + (size_t)q * kIncCbStride * L;
            const bool fx = q >= n1 + n2;
            if (l < L && p < 3 && (cm.ph[k] >> p & 1u)) {
                const size_t ik = sidx(l, p, k, n);
                const double mc = fx ? S.mcur[ik] : cb[(l * 3 + p) * 3 + 2];
                double hh = S.hi[ik], ll = S.lo[ik];
                if (k == h.s) {
                    const size_t ir = sidx(l, p, h.r, n);
                    hh = fmax(hh, S.hi[ir]);
                    ll = fmin(ll, S.lo[ir]);
                }
                const float2 v32 =
                    fx ? S.v32[ik] : make_float2((float)cb[(l * 3 + p) * 3], (float)cb[(l * 3 + p) * 3 + 1]);
                *cb_f4(cb, L, l, p) = make_float4(v32.x, v32.y, (float)(hh - mc), (float)(ll - mc));
            }
            if (l < L && p == 0) *cb_mice32(cb, L, l) = (float)cb[9 * L + l];
            if (gl == 0) {
                items += __popc(cm.ph[k]) * L;
                cm.map[k] = (unsigned short)(q + 1);     // the terms after the merge read k's new values here
            }
        }
    }
    return items;
}

// Evaluates the terms of work entries [e0, e1) (tiles of NT entries) and applies
// them per the pass (without the barrier after the last tile's updates when
// !last_barrier).  kMerge: mode-0 entries take positions from list_pre and
// add, per term, its value after the merge (r* has none) minus its value before;
// mode-1 entries take positions from list_post and set every term after the
// merge.  kInit / kFresh / kF64: every term of the entries, positions from
// list_pre.  Returns the number of terms evaluated.
template <int NT, int PREC>
__device__ __forceinline__ long long run_entries(const Topo &T, const State &S, const Search &X, const Inc &I, int n, int L, int G,
                                 double margin, float mlo, float mhi, int e0, int e1, int pass,
                                 const unsigned short *list_pre, const unsigned short *list_post, int rstar,
                                 const Ovl O, EvalSmem<NT> &E, int *sscan, const Rec &R, const Loc &Lc,
                                 unsigned long long *prof = nullptr, bool last_barrier = true) {
    // the states every group evaluates (the same for the whole pass)
    const int st_lo = (pass == kFresh) ? 1 : 0, st_hi = (pass == kMerge || pass == kFresh) ? 2 : 1;
    const int tid = threadIdx.x, gl = tid % G, gi = tid / G, NG = NT / G;
    long long terms = 0;
    unsigned long long tq = (prof && tid == 0) ? gtimer_inc() : 0;
    auto sub = [&](int i) {             // profile mode: time of the pass's steps (thread 0, after barriers)
        if (prof && tid == 0) { const unsigned long long now = gtimer_inc(); prof[i] += now - tq; tq = now; }
    };
    for (int t0 = e0; t0 < e1; t0 += NT) {
        const int ne = min(NT, e1 - t0);
        int cnt = 0;
        if (tid < ne) {
            const IncWork &w = *Lc.ent(t0 + tid);
            for (int i = 0; i < w.nseg; ++i) cnt += w.seg[i].y - w.seg[i].x;
        }
        int tot = 0;
        const int off = block_excl_scan<NT>(cnt, &tot, sscan);
        E.off[tid] = off;
        {
            const int i = tid;
            E.dlo[i] = E.dhi[i] = E.blo[i] = E.bhi[i] = 0ull;
            E.n1[i] = E.n2[i] = 0;
        }
        __syncthreads();
        sub(0);
        unsigned long long cq = (prof && tid == 0) ? clock64() : 0;
        for (int r0 = 0; r0 < tot; r0 += NG) {
            if (r0 + (tid >> 5) * (32 / G) >= tot) break;     // this warp's groups are all past the end
            const int q = r0 + gi;
            bool valid = q < tot, v_old = false, v_new = false;
            int ei = 0, k = 0;
            Cand c;
            c.s = c.r = c.a = c.js = c.ns = c.jr = c.nr = c.fixed = 0;
            if (valid) {
                // the entry holding item q: the last one whose offset is <= q
                {
                    int lo = 0, hi = ne - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (E.off[mid] <= q) lo = mid;
                        else hi = mid - 1;
                    }
                    ei = lo;
                }
                const IncWork &w = *Lc.ent(t0 + ei);
                int rem = q - E.off[ei], j = 0;
                for (int i = 0; i < w.nseg; ++i) {
                    const int len = w.seg[i].y - w.seg[i].x;
                    if (rem < len) { j = w.seg[i].x + rem; break; }
                    rem -= len;
                }
                k = ((pass == kMerge && w.mode == 1) ? list_post : list_pre)[j];
                c = entry_cand(w);
                if (k == c.r) valid = false;
                if (pass == kMerge) {
                    v_old = valid && w.mode == 0;
                    v_new = valid && !(w.mode == 0 && k == rstar);
                } else {
                    v_old = v_new = valid;
                }
                valid = v_old || v_new;
            }
            if (gl == 0) {                                            // (phase-node, scenario) items
                const int it = (st_lo == 0 && v_old ? 1 : 0) + (st_hi == 2 && v_new ? 1 : 0);
                if (it) terms += it * __popc(Lc.ph[k]) * L;
            }
            const unsigned long long c0 = (prof && tid == 0) ? clock64() : 0;
            if (prof && tid == 0) { prof[3] += c0 - cq; prof[7] += 1; }     // lookup cycles, rounds
            if (PREC == 0 || pass == kF64) {
                u128 d;
                int nv;
                group_term64(T, S, Lc.ph, n, L, G, c, k, st_lo, st_hi, v_old, v_new, O, gl, margin, nullptr, &d, &nv);
                if (valid && gl == 0) {
                    sadd128(&E.dlo[ei], &E.dhi[ei], d);
                    if (nv) atomicAdd(&E.n1[ei], nv);
                }
            } else {
                u128 d, b;
                int ns, nm;
                group_term32(T, S, Lc.ph, n, L, G, c, k, st_lo, st_hi, v_old, v_new, O, gl, mlo, mhi, &d, &b, &ns, &nm);
                if (valid && gl == 0) {
                    sadd128(&E.dlo[ei], &E.dhi[ei], d);
                    sadd128(&E.blo[ei], &E.bhi[ei], b);
                    if (ns) atomicAdd(&E.n1[ei], ns);
                    if (nm) atomicAdd(&E.n2[ei], nm);
                }
            }
            if (prof && tid == 0) { cq = clock64(); prof[4] += cq - c0; }   // term cycles
        }
        __syncthreads();
        sub(1);
        if (tid < ne) {
            const IncWork &w = *Lc.ent(t0 + tid);
            const int sl = w.slot;
            const u128 d = ((u128)E.dhi[tid] << 64) | (u128)E.dlo[tid];
            const u128 b = ((u128)E.bhi[tid] << 64) | (u128)E.blo[tid];
            unsigned long long *a = I.acc + 2 * (size_t)sl, *bp = I.bnd + 2 * (size_t)sl;
            if (pass == kInitPart) {
                sadd128(a, a + 1, d);
                if (E.n1[tid]) atomicAdd(I.viol + sl, E.n1[tid]);
                if (PREC == 1) {
                    sadd128(bp, bp + 1, b);
                    if (E.n2[tid]) atomicAdd(I.vmay + sl, E.n2[tid]);
                }
            } else if (pass == kMerge || pass == kInit) {
                u128 na, nb = 0;
                int nv, nm = 0;
                if (w.mode == 1) {
                    na = d;
                    nv = E.n1[tid];
                    if (PREC == 1) { nb = b; nm = E.n2[tid]; }
                } else {
                    na = ld128(a) + d;
                    nv = I.viol[sl] + E.n1[tid];
                    if (PREC == 1) { nb = ld128(bp) + b; nm = I.vmay[sl] + E.n2[tid]; }
                }
                st128(a, na);
                I.viol[sl] = nv;
                if (PREC == 1) {
                    st128(bp, nb);
                    I.vmay[sl] = nm;
                }
                set_rec<PREC>(R, sl, na, nb, nv, nm);
            } else {
                st128(I.vacc + 2 * (size_t)sl, d);
                I.vviol[sl] = E.n1[tid];
            }
        }
        if (last_barrier || t0 + NT < e1) __syncthreads();    // else the caller synchronises
        sub(2);
    }
    return terms;
}

// Rebuilds slot pair w from the clusters as the view shows them and appends
// a full work entry for each valid candidate at entry base + *cnt (*cnt: a
// shared counter; the caller synchronises before reading it).
template <int NT, int PREC>
__device__ void rebuild_pair(const Topo &T, const State &S, const Search &X, const Inc &I, int n, int w, int *cnt,
                             int base, const Rec &R, const Loc &Lc, const View &V) {
    {
        Cand c[2];
        const int x = slot_geometry(T, S, V, n, w, c[0], c[1]);
        I.qpar[w] = x;
        {
            int lo = n, hi = 0;
            for (int d = 0; d < 2; ++d) {
                if (c[d].s < 0) continue;
                lo = min(lo, min(min(c[d].s, c[d].r), c[d].ns > 0 ? c[d].js : n));
                lo = min(lo, c[d].nr > 0 ? c[d].jr : n);
                hi = max(hi, max(max(c[d].s, c[d].r) + 1, max(c[d].js + c[d].ns, c[d].jr + c[d].nr)));
            }
            const bool any = c[0].s >= 0 || c[1].s >= 0;
            R.span[w] = make_ushort4((unsigned short)(any ? lo : 0), (unsigned short)(any ? hi : 0),
                                     (unsigned short)(x >= 0 ? x : 0xffff), (unsigned short)(any ? 1 : 0));
        }
        for (int d = 0; d < 2; ++d) {
            const int sl = 2 * w + d;
            X.slot[sl] = c[d];
            if (c[d].s >= 0) {
                int2 seg[kIncMaxSeg];
                const int ns = full_segments(c[d], Lc.rank, seg, V.r);
                write_entry(Lc.ent(base + atomicAdd(cnt, 1)), sl, 1, ns, seg, c[d]);
                R.tkey[sl] = (unsigned)c[d].key;
                R.touch(sl);
            } else {
                I.viol[sl] = kIncDead;
                st128(I.acc + 2 * (size_t)sl, 0);
                kill_rec<PREC>(R, sl);
            }
        }
    }
}

// The slot pairs listed in fp[0, nf), from the last thread down.
template <int NT, int PREC>
__device__ void rebuild_pairs(const Topo &T, const State &S, const Search &X, const Inc &I, int n, const int *fp, int nf,
                              int *cnt, int base, const Rec &R, const Loc &Lc, const View &V) {
    for (int i = NT - 1 - (int)threadIdx.x; i < nf; i += NT)
        rebuild_pair<NT, PREC>(T, S, X, I, n, fp[i], cnt, base, R, Lc, V);
}

}  // namespace

// Writes the merge hw's new values from its scratch into the state (the
// values the overlay gave the terms after it: FP64 voltage, magnitude, MICE,
// s*'s merged extremes, and their FP32 copies), clears its overlay map, and
// zeroes r*'s MICE.  `list`: the super-nodes before that merge.
template <int NT>
__device__ void write_back(const State &S, const Inc &I, const Win &hw, const unsigned short *list, const uint8_t *ph,
                           unsigned short *map, int n, int L, int G) {
    // lanes from the last thread down (no shuffles here), beside the first
    // threads' updates of the entries' sums
    const int tid = threadIdx.x, rt = NT - 1 - tid, gl = rt % G, gi = rt / G, NG = NT / G, l = gl >> 2, p = gl & 3;
    const int n1 = hw.q1hi - hw.q1lo, n2 = hw.q2hi - hw.q2lo;
    for (int j = gi; j < hw.npos; j += NG) {
        const int k = j < n1 ? list[hw.q1lo + j] : (j < n1 + n2 ? list[hw.q2lo + j - n1] : hw.s);
        if (k == hw.r) continue;
        const bool fx = j >= n1 + n2;
        const double *cb = I.cbuf + (size_t)j * kIncCbStride * L;
        if (l < L && p < 3 && (ph[k] >> p & 1u)) {
            const size_t ik = sidx(l, p, k, n);
            const float4 f = *cb_f4(cb, L, l, p);
            if (!fx) {
                S.vcur[ik] = make_double2(cb[(l * 3 + p) * 3 + 0], cb[(l * 3 + p) * 3 + 1]);
                S.mcur[ik] = cb[(l * 3 + p) * 3 + 2];
                S.v32[ik] = make_float2(f.x, f.y);
            }
            if (k == hw.s) {
                const size_t ir = sidx(l, p, hw.r, n);
                S.hi[ik] = fmax(S.hi[ik], S.hi[ir]);
                S.lo[ik] = fmin(S.lo[ik], S.lo[ir]);
            }
            S.hr32[ik] = f.z;
            S.lr32[ik] = f.w;
        }
        if (l < L && p == 0) {
            S.mice[(size_t)l * n + k] = cb[9 * L + l];
            S.mice32[(size_t)l * n + k] = *cb_mice32(cb, L, l);
        }
        if (gl == 0) map[k] = 0;
    }
    if (rt < L) {                           // r's cluster is gone
        S.mice[(size_t)rt * n + hw.r] = 0.0;
        S.mice32[(size_t)rt * n + hw.r] = 0.0f;
    }
}

// ---------------------------------------------------------------- the search
// Bytes of the selection records of an n-bus feeder.
__host__ __device__ constexpr size_t rec_bytes(int n) { return (size_t)48 * n + 64; }
// ... and with the per-super-node largest MICE after them (shared memory only).
__host__ __device__ constexpr size_t rec_maxm_bytes(int n) { return rec_bytes(n) + (size_t)8 * n; }

// Shared memory of one search: [work entries][two super-node lists][phase
// masks][overlay map][super-node ranks][block summaries of the selection
// records], then the selection records when they fit.
__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }
// Blocks of 32 selection slots, and the bytes of their summaries.
__host__ __device__ constexpr int sel_blocks(int n) { return (2 * n + 31) / 32; }
__host__ __device__ constexpr size_t sel_bytes(int n) {
    return align16((size_t)16 * sel_blocks(n)) + align16((size_t)4 * sel_blocks(n)) +
           align16((size_t)8 * sel_blocks(n)) + align16((size_t)sel_blocks(n));
}
// Every region is rounded up to 16 bytes: the block summaries and the
// selection records are 16-byte keys.
__host__ __device__ constexpr size_t base_bytes(int n, int se) {
    return align16((size_t)se * sizeof(IncWork)) + align16((size_t)4 * n) + align16((size_t)n) + align16((size_t)2 * n) +
           align16((size_t)4 * (n + 1)) + sel_bytes(n);
}

template <int NT, int PREC>
__device__ void inc_run(const Topo &T, const State &S, const Search &X, const Inc &I, Ctrl *C, bool verify,
                        unsigned char *dyn, int rec_mode, int se, int cw, bool pre_init) {
    static_assert(NT >= 128 && NT <= 1024 && NT % 32 == 0, "thread count");
    __shared__ __align__(16) EvalSmem<NT> E;
    __shared__ __align__(16) Red sred[33];
    __shared__ __align__(16) Red64 s_sel[2];   // precision-1 selection accumulators: pass A, pass B
    __shared__ int sscan[33];
    __shared__ unsigned long long s_sfx[2];     // SMICE of the committed state, fixed point
    __shared__ unsigned long long s_dsum[2];    // the last merge's change of it
    __shared__ int s_cnt[4];                    // append counters: rebuilt pairs, changed entries, entries, R
    const int n = T.n, L = T.L, tid = threadIdx.x;
    const int G = 4 * (L <= 1 ? 1 : (L <= 2 ? 2 : 4));
    const double margin = C->margin;
    const float mlo = __double2float_rd(margin), mhi = __double2float_ru(margin);
    const int max_merges = C->max_merges;
    const bool prof = C->profile != 0;
    const u128 tau_fx = to_fx(C->tau);
    if (C->done || C->t >= max_merges) return;
    // shared memory: entries, lists, phases; selection records: r0 or r1
    // (2n x 16 B), tkey (2n x 4 B), span (n x 8 B)
    Loc Lc;
    Lc.wsm = reinterpret_cast<IncWork *>(dyn);
    Lc.wgl = I.work;
    Lc.se = se;
    Lc.lst[0] = reinterpret_cast<unsigned short *>(dyn + align16((size_t)se * sizeof(IncWork)));
    Lc.lst[1] = Lc.lst[0] + n;
    uint8_t *phs = dyn + align16((size_t)se * sizeof(IncWork)) + align16((size_t)4 * n);
    Lc.ph = phs;
    unsigned short *ovl_map = reinterpret_cast<unsigned short *>(phs + align16((size_t)n));
    // the super-node ranks live in shared memory during the search (copied back at the end)
    int *rank = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(ovl_map) + align16((size_t)2 * n));
    Lc.rank = rank;
    Ovl O;
    O.map = ovl_map;
    O.cbuf = I.cbuf;
    O.s = O.r = -1;
    O.nfree = 0;
    unsigned char *recmem = rec_mode ? dyn + base_bytes(n, se) : I.recbuf;
    Rec R;
    R.r0 = reinterpret_cast<u128 *>(recmem);
    R.r1 = reinterpret_cast<ulonglong2 *>(recmem);
    R.tkey = reinterpret_cast<unsigned *>(recmem + (size_t)32 * n);
    R.maxm = rec_mode == 2 ? reinterpret_cast<double *>(recmem + rec_bytes(n)) : I.maxm;
    R.span = reinterpret_cast<ushort4 *>(recmem + (size_t)40 * n);
    {
        unsigned char *sm = reinterpret_cast<unsigned char *>(rank) + align16((size_t)4 * (n + 1));
        R.nb = sel_blocks(n);
        R.bsum = sm;
        sm += align16((size_t)16 * R.nb);
        R.bcnt = reinterpret_cast<int *>(sm);
        sm += align16((size_t)4 * R.nb);
        R.bmx = reinterpret_cast<unsigned long long *>(sm);
        sm += align16((size_t)8 * R.nb);
        R.dirty = sm;
    }
    int t = 0, ns = n;
    if (tid == 0) {
        s_sfx[0] = s_sfx[1] = 0ull;                 // every MICE starts at 0
        s_cnt[0] = s_cnt[1] = s_cnt[2] = s_cnt[3] = 0;
        reset_sel(&s_sel[0]);
        reset_sel(&s_sel[1]);
    }
    unsigned long long tp = 0;
    auto stamp = [&](int i) {
        if (prof && tid == 0) { const unsigned long long now = gtimer_inc(); C->phase_ns[i] += now - tp; tp = now; }
    };
    long long terms = 0, cands_run = 0;
    int rechecks = 0, recheck_cands = 0;
    bool maxerr_done = true;                // dec_maxerr of the last merge written

    // ---- every slot pair from the initial clusters (all singletons), every term
    for (int w = tid; w < n; w += NT) {
        I.fpair[w] = w;
        R.maxm[w] = 0.0;
        Lc.lst[0][w] = (unsigned short)w;
        phs[w] = __ldg(T.ph + w);
        ovl_map[w] = 0;
        rank[w] = S.sn_rank[w];
    }
    if (tid == 0) rank[n] = S.sn_rank[n];
    for (int j = tid; j < R.nb; j += NT) R.dirty[j] = 1;
    if (pre_init) {
        // the first evaluation ran on many CTAs (k_inc_init): its records are in
        // device memory in the same layout; bring them into shared memory
        if (rec_mode) {
            const uint4 *src = reinterpret_cast<const uint4 *>(I.recbuf);
            uint4 *dst = reinterpret_cast<uint4 *>(recmem);
            for (int i = tid; i < 3 * n; i += NT) dst[i] = src[i];       // 48 n bytes
        }
        __syncthreads();
        // the live candidates' keys from their carried sums (the first evaluation
        // may have summed a candidate's terms on several CTAs)
        for (int sl = tid; sl < 2 * n; sl += NT) {
            const int v = I.viol[sl];
            if (v == kIncDead) continue;
            set_rec<PREC>(R, sl, ld128(I.acc + 2 * (size_t)sl), PREC == 1 ? ld128(I.bnd + 2 * (size_t)sl) : (u128)0, v,
                          PREC == 1 ? I.vmay[sl] : 0);
        }
        __syncthreads();
    } else {
        __syncthreads();
        rebuild_pairs<NT, PREC>(T, S, X, I, n, I.fpair, n, &s_cnt[2], 0, R, Lc, no_view());
        __syncthreads();
        const int ne = s_cnt[2];
        terms += run_entries<NT, PREC>(T, S, X, I, n, L, G, margin, mlo, mhi, 0, ne, kInit, Lc.lst[0], Lc.lst[0],
                                       -1, O, E, sscan, R, Lc);
    }
    if (prof && tid == 0) tp = gtimer_inc();

    for (;;) {
        if (t >= max_merges) {
            if (tid == 0) { C->done = 1; C->stop_reason = 0; }
            break;
        }
        const unsigned short *list_old = Lc.lst[t & 1];
        unsigned short *list_new = Lc.lst[(t + 1) & 1];
        // ============================================================ selection
        // The blocks whose records changed are summarised again (one warp per
        // block; the append counters are cleared before that barrier).
        if (tid == 0) s_cnt[0] = s_cnt[1] = s_cnt[2] = s_cnt[3] = 0;
        refresh_blocks<NT, PREC>(R, n);
        // pass A, by every warp on its own from the block summaries (no
        // barrier): precision 0: the minimum over feasible candidates;
        // precision 1: the smallest lower end (m_lo) and the smallest upper end
        // (m_hi); the largest MICE after the last merge; the candidates.
        const int lane = tid & 31, wid = tid >> 5;
        Red ra;
        ra.a = ra.b = ra.c = kNone;
        ra.i = 0;
        {
            unsigned long long mx = 0;
            unsigned cnt = 0;
            if (PREC == 0) {
                const u128 *bs = reinterpret_cast<const u128 *>(R.bsum);
                u128 mn = kNone;
                for (int j = lane; j < R.nb; j += 32) {
                    mn = umin(mn, bs[j]);
                    cnt += (unsigned)R.bcnt[j];
                    mx = R.bmx[j] > mx ? R.bmx[j] : mx;
                }
                ra.a = warp_min128(mn);
            } else {
                const ulonglong2 *bs = reinterpret_cast<const ulonglong2 *>(R.bsum);
                unsigned long long lo = ~0ull, hi = ~0ull;
                for (int j = lane; j < R.nb; j += 32) {
                    const ulonglong2 b = bs[j];
                    lo = b.x < lo ? b.x : lo;
                    hi = b.y < hi ? b.y : hi;
                    cnt += (unsigned)R.bcnt[j];
                    mx = R.bmx[j] > mx ? R.bmx[j] : mx;
                }
                lo = warp_min64(lo);
                hi = warp_min64(hi);
                ra.a = lo == kKeyNone ? kNone : (u128)lo;
                ra.b = hi == kKeyNone ? kNone : (u128)hi;
            }
            ra.i = (int)__reduce_add_sync(0xffffffffu, cnt);
            ra.c = ~(u128)warp_max64(mx);               // kNone when every maxm is 0
        }
        const int nvalid = ra.i;
        stamp(11);                                      // profile: block summaries and pass A
        if (tid == 0) {
            cands_run += nvalid;
            X.dec_ncand[t] = nvalid;
            if (t > 0)
                X.dec_maxerr[t - 1] = ra.c == kNone ? 0.0 : __longlong_as_double((long long)(unsigned long long)~ra.c);
        }
        if (t < X.rec_iters) {
            const double s_cur = fx_to_d(ld128(s_sfx));
            // every candidate's SMICE (+inf when (surely) infeasible), compacted in slot order
            int base = 0;
            for (int c0 = 0; c0 < 2 * n; c0 += NT) {
                const int c = c0 + tid;
                const int v = c < 2 * n ? I.viol[c] : kIncDead;
                const int f = v < kIncDead ? 1 : 0;
                int tot = 0;
                const int o = block_excl_scan<NT>(f, &tot, sscan) + base;
                if (f) {
                    const Cand &cc = X.slot[c];
                    const size_t at = (size_t)t * 2 * n + o;
                    X.rec_s[at] = T.orig[cc.s];
                    X.rec_r[at] = T.orig[cc.r];
                    X.rec_score[at] = v == 0 ? s_cur + fx_to_d(ld128(I.acc + 2 * (size_t)c)) : INFINITY;
                    X.rec_bound[at] = (PREC == 1 && v == 0) ? fx_to_d(ld128(I.bnd + 2 * (size_t)c)) * (1.0 + 1e-12) : 0.0;
                }
                base += tot;
            }
            if (tid == 0) X.rec_count[t] = nvalid;
        }
        if (ra.a == kNone) {                             // nothing (possibly) feasible
            if (tid == 0) { C->done = 1; C->stop_reason = 1; }
            maxerr_done = true;
            break;
        }
        // pass B: the smallest (tie key, slot) in the tie band and the smallest
        // key above it (precision 0); in precision 1, the smallest (tie key,
        // slot) surely in the band, the smallest tie key of a candidate the
        // screen cannot place, and the smallest lower end surely out of it.
        // Records in shared memory, at most kFlatSelectMax buses: every record
        // once, each thread a strided share of the slots, then one block
        // reduction.  Otherwise only the blocks that may hold a candidate of the band are
        // read record by record (a block whose smallest key lies above the
        // band counts whole); with few such blocks every warp reads them all
        // and needs no barrier, with more they are spread over the warps.
        int ws = -1;
        double gap = INFINITY;
        const bool flat_b = rec_mode != 0 && n <= kFlatSelectMax;
        if (PREC == 0) {
            const u128 edge = (ra.a ^ kSignBit) + tau_fx, ek = okey(edge);
            u128 pa = kNone, pb = kNone;        // smallest (key, slot) in the band; smallest score above it
            if (flat_b) {
                for (int c = tid; c < 2 * n; c += NT) {
                    const u128 k = R.r0[c];
                    if (k == kNone) continue;
                    if (k <= ek) pa = umin(pa, ((u128)R.tkey[c] << 32) | (u128)(unsigned)c);
                    else pb = umin(pb, k);
                }
                {
                    Red rb;
                    rb.a = pa;
                    rb.b = pb;
                    rb.c = kNone;
                    rb.i = 0;
                    rb = block_red<NT>(rb, sred);
                    pa = rb.a;
                    pb = rb.b;
                }
            } else {
                const u128 *bs = reinterpret_cast<const u128 *>(R.bsum);
                auto relevant = [&](int j) {
                    const u128 bk = j < R.nb ? bs[j] : kNone;
                    return bk != kNone && bk <= ek;
                };
                int nrel = 0;
                for (int j0 = 0; j0 < R.nb; j0 += 32) {
                    const int j = j0 + lane;
                    const bool rel = relevant(j);
                    if (!rel && j < R.nb) pb = umin(pb, bs[j]);          // the whole block above the band
                    nrel += __popc(__ballot_sync(0xffffffffu, rel));
                }
                const bool few = nrel <= kFewBlocks;
                int kq = 0;
                for (int j0 = 0; j0 < R.nb; j0 += 32) {
                    unsigned mask = __ballot_sync(0xffffffffu, relevant(j0 + lane));
                    while (mask) {
                        const int b = __ffs(mask) - 1;
                        mask &= mask - 1;
                        if (few || kq % (NT / 32) == wid) {
                            const int c = 32 * (j0 + b) + lane;
                            if (c < 2 * n) {
                                const u128 k = R.r0[c];
                                if (k <= ek) pa = umin(pa, ((u128)R.tkey[c] << 32) | (u128)(unsigned)c);
                                else pb = umin(pb, k);
                            }
                        }
                        ++kq;
                    }
                }
                if (few) {
                    pa = warp_min128(pa);
                    pb = warp_min128(pb);
                } else {
                    Red rb;
                    rb.a = pa;
                    rb.b = pb;
                    rb.c = kNone;
                    rb.i = 0;
                    rb = block_red<NT>(rb, sred);
                    pa = rb.a;
                    pb = rb.b;
                }
            }
            ws = (int)(unsigned)(pa & 0xffffffffu);
            if (tid == 0 && pb != kNone) gap = fx_to_d((pb ^ kSignBit) - edge);
        } else {
            const bool has_hi = ra.b != kNone;
            bool ok;
            const long long tau_dn = key_val(key_floor(tau_fx, &ok)), tau_up = key_val(key_ceil(tau_fx, &ok));
            const long long m_lo = key_val((unsigned long long)ra.a);
            const long long m_hi = has_hi ? key_val((unsigned long long)ra.b) : 0;
            const unsigned long long ein = val_key(m_lo + tau_dn);
            const unsigned long long eout = has_hi ? val_key(m_hi + tau_up) : kKeyNone;
            unsigned long long pa = ~0ull, pb = ~0ull, pc = ~0ull;
            if (flat_b) {
                for (int c = tid; c < 2 * n; c += NT) {
                    const ulonglong2 q = R.r1[c];
                    if (q.x == kKeyNone) continue;
                    const bool in_sure = q.y <= ein;
                    const bool out_sure = has_hi && q.x > eout;     // (never both: lo <= hi, m_lo <= m_hi)
                    if (in_sure) {
                        const unsigned long long kc = ((unsigned long long)R.tkey[c] << 32) | (unsigned)c;
                        pa = kc < pa ? kc : pa;
                    } else if (!out_sure) {
                        const unsigned long long key = R.tkey[c];
                        pb = key < pb ? key : pb;
                    } else {
                        pc = q.x < pc ? q.x : pc;
                    }
                }
                {
                    Red64 r6;
                    r6.a = pa;
                    r6.b = pb;
                    r6.c = pc;
                    r6.i = 0;
                    r6 = block_sel64(r6, &s_sel[1]);
                    pa = r6.a;
                    pb = r6.b;
                    pc = r6.c;
                }
            } else {
                const ulonglong2 *bs = reinterpret_cast<const ulonglong2 *>(R.bsum);
                // a block is read record by record unless every candidate in it is
                // surely out of the band (its smallest lower end above eout)
                auto relevant = [&](int j) {
                    const unsigned long long bl = j < R.nb ? bs[j].x : kKeyNone;
                    return bl != kKeyNone && !(has_hi && bl > eout);
                };
                int nrel = 0;
                for (int j0 = 0; j0 < R.nb; j0 += 32) {
                    const int j = j0 + lane;
                    const bool rel = relevant(j);
                    const unsigned long long bl = j < R.nb ? bs[j].x : kKeyNone;
                    if (bl != kKeyNone && !rel) pc = bl < pc ? bl : pc;        // the whole block surely out
                    nrel += __popc(__ballot_sync(0xffffffffu, rel));
                }
                const bool few = nrel <= kFewBlocks;
                int kq = 0;
                for (int j0 = 0; j0 < R.nb; j0 += 32) {
                    unsigned mask = __ballot_sync(0xffffffffu, relevant(j0 + lane));
                    while (mask) {
                        const int b = __ffs(mask) - 1;
                        mask &= mask - 1;
                        if (few || kq % (NT / 32) == wid) {
                            const int c = 32 * (j0 + b) + lane;
                            if (c < 2 * n) {
                                const ulonglong2 q = R.r1[c];
                                if (q.x != kKeyNone) {
                                    const bool in_sure = q.y <= ein;
                                    const bool out_sure = has_hi && q.x > eout;
                                    const unsigned key = R.tkey[c];
                                    if (in_sure) {
                                        const unsigned long long kc = ((unsigned long long)key << 32) | (unsigned)c;
                                        pa = kc < pa ? kc : pa;
                                    } else if (!out_sure) {
                                        pb = key < pb ? key : pb;
                                    }
                                    if (out_sure) pc = q.x < pc ? q.x : pc;
                                }
                            }
                        }
                        ++kq;
                    }
                }
                if (few) {
                    pa = warp_min64(pa);
                    pb = warp_min64(pb);
                    pc = warp_min64(pc);
                } else {
                    Red64 r6;
                    r6.a = pa;
                    r6.b = pb;
                    r6.c = pc;
                    r6.i = 0;
                    r6 = block_sel64(r6, &s_sel[1]);
                    pa = r6.a;
                    pb = r6.b;
                    pc = r6.c;
                }
            }
            Red rb;
            rb.a = pa == ~0ull ? kNone : (u128)pa;
            rb.b = pb == ~0ull ? kNone : (u128)pb;
            rb.c = pc == ~0ull ? kNone : (u128)pc;
            rb.i = 0;
            const u128 ks = rb.a == kNone ? kNone : (rb.a >> 32);
            if (!(rb.b < ks)) {                          // no uncertain candidate can take the band's smallest key
                ws = (int)(unsigned)(rb.a & 0xffffffffu);
                if (tid == 0 && rb.c != kNone) gap = (double)(key_val((unsigned long long)rb.c) - key_val(eout)) * 0x1p-56;
            } else {
                // FP64 rescoring of R: the possible minimizers and the uncertain
                // candidates with a key below the smallest surely-in key
                const unsigned long long mh = has_hi ? (unsigned long long)ra.b : kKeyNone;
                for (int c = tid; c < 2 * n; c += NT) {
                    const ulonglong2 q = R.r1[c];
                    if (q.x == kKeyNone) continue;
                    const bool in_sure = q.y <= ein;
                    const bool out_sure = has_hi && q.x > eout;
                    const bool unc = !in_sure && !out_sure && (u128)R.tkey[c] < ks;
                    if (unc || q.x <= mh) {
                        const int o = atomicAdd(&s_cnt[3], 1);
                        I.rlist[o] = c;
                        int2 seg[kIncMaxSeg];
                        const int k = full_segments(X.slot[c], rank, seg);
                        write_entry(Lc.ent(o), c, 1, k, seg, X.slot[c]);
                    }
                }
                __syncthreads();
                const int nR = s_cnt[3];
                terms += run_entries<NT, PREC>(T, S, X, I, n, L, G, margin, mlo, mhi, 0, nR, kF64, list_old, list_old,
                                               -1, O, E, sscan, R, Lc);
                // exact selection over R, with the surely-in candidate of key ks
                Red rc;
                rc.a = rc.b = rc.c = kNone;
                rc.i = 0;
                for (int i = tid; i < nR; i += NT) {
                    const int c = I.rlist[i];
                    if (I.vviol[c] == 0) rc.a = umin(rc.a, okey(ld128(I.vacc + 2 * (size_t)c)));
                }
                rc = block_red<NT>(rc, sred);
                Red rd;
                rd.a = rd.b = rd.c = kNone;
                rd.i = 0;
                if (rc.a != kNone) {
                    const u128 edge = (rc.a ^ kSignBit) + tau_fx, ek = okey(edge);
                    for (int i = tid; i < nR; i += NT) {
                        const int c = I.rlist[i];
                        if (I.vviol[c] != 0) continue;
                        const u128 k = okey(ld128(I.vacc + 2 * (size_t)c));
                        if (k <= ek) rd.a = umin(rd.a, ((u128)R.tkey[c] << 32) | (u128)(unsigned)c);
                        else rd.b = umin(rd.b, k);
                    }
                    rd = block_red<NT>(rd, sred);
                    if (tid == 0 && rd.b != kNone) gap = fx_to_d((rd.b ^ kSignBit) - edge);
                }
                const u128 best = umin(rd.a, rb.a);
                ws = best == kNone ? -1 : (int)(unsigned)(best & 0xffffffffu);
                ++rechecks;
                recheck_cands += nR;
            }
        }
        if (ws < 0) {                                    // FP64 rescoring found nothing feasible
            if (tid == 0) { C->done = 1; C->stop_reason = 1; }
            break;
        }
        stamp(0);
        // ============================================================ the merge's changed set
        // The winner's record: every thread builds its own at once (every
        // thread knows ws; one broadcast load of its candidate), so no warp
        // waits for another's copy (r*'s subtree and the decision's bus ids
        // are looked up in the merge step).
        constexpr int NW = NT / 32;
        const int CW = cw;                  // warps that evaluate the merge (1 .. NW - 1)
        const bool commit_warp = (tid >> 5) >= NW - CW;
        const Win hw = make_win(X.slot[ws], ws, rank);
        if (tid == 0) {
            X.dec_gap[t] = gap;
            s_dsum[0] = 0ull;
            s_dsum[1] = 0ull;
        }
        stamp(12);                                      // profile: the winner's record
        O.s = hw.s;
        O.r = hw.r;
        O.nfree = (hw.q1hi - hw.q1lo) + (hw.q2hi - hw.q2lo);
        // ---- which candidates change: rebuilt pairs (next to s* or r*) and
        // changed terms; entries are appended in any order (the sums are exact).
        // The last warps evaluate the merge's own FP64 values meanwhile and
        // map its positions for the overlay.
        {
            if (commit_warp) {
                Commit cm;
                cm.h = &hw;
                cm.wc = X.slot[ws];
                cm.list = list_old;
                cm.ph = Lc.ph;
                cm.O = O;
                cm.map = ovl_map;
                terms += commit_groups(T, S, I, n, L, G, margin, cm, NW - CW, CW);
            } else {
                // the changed buses lie in [hl, hh): a candidate whose span misses it is unchanged
                int hl = min(hw.s, hw.r), hh = max(hw.s, hw.r) + 1;
                if (hw.w1lo < hw.w1hi) { hl = min(hl, hw.w1lo); hh = max(hh, hw.w1hi); }
                if (hw.w2lo < hw.w2hi) { hl = min(hl, hw.w2lo); hh = max(hh, hw.w2hi); }
                for (int w = tid; w < n; w += (NW - CW) * 32) {
                    const ushort4 sp = R.span[w];
                    if (sp.w == 0 || w == hw.r) continue;
                    const int qp = sp.z == 0xffff ? -1 : (int)sp.z;
                    if (w == hw.s || qp == hw.r || qp == hw.s) {
                        I.fpair[atomicAdd(&s_cnt[0], 1)] = w;
                        continue;
                    }
                    if ((int)sp.y <= hl || (int)sp.x >= hh) continue;
                    for (int d = 0; d < 2; ++d) {
                        const Cand &c = X.slot[2 * w + d];
                        if (c.s < 0 || !touched(c, hw)) continue;
                        int2 seg[kIncMaxSeg];
                        const int k = changed_segments(c, hw, rank, seg);
                        write_entry(Lc.ent(atomicAdd(&s_cnt[1], 1)), 2 * w + d, 0, k, seg, c);
                    }
                }
            }
        }
        __syncthreads();
        const int nf_tot = s_cnt[0], np_tot = s_cnt[1];   // (s_cnt[2] is 0: rebuilt entries follow these)
        if (PREC == 1 && tid == 0) {                 // every thread has read both selection results
            reset_sel(&s_sel[0]);
            reset_sel(&s_sel[1]);
        }
        stamp(1);
        // ============================================================ the merge (score change, topology) and,
        // beside it, the rebuilt candidates
        // (the new voltages, extremes and MICE stay in the scratch, with the
        // FP32 copies the merge's evaluation derived, read through the overlay,
        // until the terms before the merge have been evaluated)
        {
            const int n1 = hw.q1hi - hw.q1lo, n2 = hw.q2hi - hw.q2lo;
            const int gl = tid % G, gi = tid / G, NG = NT / G, l = gl >> 2, p = gl & 3;
            u128 dsum = 0;
            // one lane per (position, scenario)
            for (int r0 = 0; r0 < hw.npos; r0 += NG) {
                if (r0 + (tid >> 5) * (32 / G) >= hw.npos) break;
                const int j = r0 + gi;
                bool valid = j < hw.npos;
                int k = hw.s;
                if (valid) {
                    k = j < n1 ? list_old[hw.q1lo + j] : (j < n1 + n2 ? list_old[hw.q2lo + j - n1] : hw.s);
                    valid = k != hw.r;
                }
                const double *cb = I.cbuf + (size_t)j * kIncCbStride * L;
                // the merge's exact score change: its FP64 terms in fixed point
                unsigned long long mb = 0;                  // MICE >= 0: bit patterns order like values
                if (valid && l < L && p == 0) {
                    const double m = cb[9 * L + l];
                    double dd = m - S.mice[(size_t)l * n + k];
                    if (k == hw.s) dd -= S.mice[(size_t)l * n + hw.r];
                    dsum += to_fx(dd);
                    mb = (unsigned long long)__double_as_longlong(m);
                }
                for (int o = 4; o < G; o <<= 1) {
                    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mb, o);
                    mb = y > mb ? y : mb;
                }
                if (valid && gl == 0) {
                    R.maxm[k] = __longlong_as_double((long long)mb);
                    R.touch_sn(k);
                }
            }
            if (dsum != 0) sadd128(&s_dsum[0], &s_dsum[1], dsum);
            // r's members join s (they lie in the subtree of r's top); the new
            // super-node list.  Not on the last warp, which goes straight to the
            // rebuilt pairs below (their chain of dependent loads is this
            // step's longest).
            constexpr int NB = NT - 32;
            if (tid < NB) {
                const int rtop = S.top[hw.r], rtop_end = rtop + T.sz[rtop];
                for (int b = rtop + tid; b < rtop_end; b += NB)
                    if (S.label[b] == hw.r) S.label[b] = hw.s;
                for (int j = tid; j < ns - 1; j += NB) list_new[j] = list_old[j + (j >= hw.jr ? 1 : 0)];
            }
            // s takes r's injection (no term before the merge reads s's injection:
            // every candidate with r = s* is rebuilt)
            const unsigned phr = Lc.ph[hw.r];
            if (tid < 3 * L) {
                const int l = tid / 3, q = tid % 3;
                if (phr >> q & 1u) {
                    const size_t is = sidx(l, q, hw.s, n), ir = sidx(l, q, hw.r, n);
                    const double2 ni = cadd(S.icur[is], S.icur[ir]);
                    S.icur[is] = ni;
                    S.icur32[is] = make_float2((float)ni.x, (float)ni.y);
                }
            }
            if (tid == 0) {
                if (hw.dir == 1) {
                    S.top[hw.s] = S.top[hw.r];
                    S.ptop[hw.s] = S.ptop[hw.r];
                }
                I.qpar[hw.r] = -1;
                R.maxm[hw.r] = 0.0;
                R.touch_sn(hw.r);
                X.dec_s[t] = T.orig[hw.s];
                X.dec_r[t] = T.orig[hw.r];
            }
            if (tid < 2) {
                X.slot[2 * hw.r + tid].s = -1;
                I.viol[2 * hw.r + tid] = kIncDead;
                kill_rec<PREC>(R, 2 * hw.r + tid);
            }
            if (tid == 0) R.span[hw.r] = make_ushort4(0, 0, 0xffff, 0);
        }
        // rebuilt pairs from the last thread down, reading the clusters through the
        // merge's view (the ranks change only after the terms below)
        {
            View V;
            V.s = hw.s;
            V.r = hw.r;
            V.dir = hw.dir;
            rebuild_pairs<NT, PREC>(T, S, X, I, n, I.fpair, nf_tot, &s_cnt[2], np_tot, R, Lc, V);
        }
        __syncthreads();
        ns -= 1;
        const int ne_new = np_tot + s_cnt[2];
        stamp(2);
        if (tid == 0) {
            const u128 sfx = ld128(s_sfx) + ld128(s_dsum);
            st128(s_sfx, sfx);
            X.dec_score[t] = fx_to_d(sfx);
        }
        // ============================================================ the terms that change
        terms += run_entries<NT, PREC>(T, S, X, I, n, L, G, margin, mlo, mhi, 0, ne_new, kMerge, list_old, list_new, hw.r,
                                       O, E, sscan, R, Lc, prof ? C->phase_ns + 6 : nullptr, false);
        // the new values into the state (no term reads the state before the
        // merge any more; this overlaps the last tile's updates of the sums);
        // ranks past r* drop by one
        write_back<NT>(S, I, hw, list_old, Lc.ph, ovl_map, n, L, G);
        for (int b = hw.r + 1 + tid; b <= n; b += NT) rank[b] -= 1;
        __syncthreads();
        stamp(3);
        t += 1;
        maxerr_done = false;
        if (verify) {
            // every candidate again from scratch (after the merge, through the
            // overlay); the carried values must match bit for bit
            if (tid == 0) s_cnt[3] = 0;
            __syncthreads();
            for (int c = tid; c < 2 * n; c += NT) {
                const Cand &cc = X.slot[c];
                if (cc.s < 0) continue;
                int2 seg[kIncMaxSeg];
                const int k = full_segments(cc, rank, seg);
                write_entry(Lc.ent(atomicAdd(&s_cnt[3], 1)), c, 1, k, seg, cc);
            }
            __syncthreads();
            run_entries<NT, PREC>(T, S, X, I, n, L, G, margin, mlo, mhi, 0, s_cnt[3], kFresh, list_new, list_new, -1,
                                  O, E, sscan, R, Lc);
            int bad = 0;
            for (int c = tid; c < 2 * n; c += NT) {
                if (X.slot[c].s < 0) continue;
                if (I.viol[c] != I.vviol[c] || ld128(I.acc + 2 * (size_t)c) != ld128(I.vacc + 2 * (size_t)c)) ++bad;
            }
            Red rv;
            rv.a = rv.b = rv.c = kNone;
            rv.i = bad;
            rv = block_red<NT>(rv, sred);
            if (tid == 0 && rv.i) C->inc_mismatch += rv.i;
        }
    }
    if (!maxerr_done && t > 0) {
        Red rm;
        rm.a = rm.b = rm.c = kNone;
        rm.i = 0;
        for (int w = tid; w < n; w += NT) rm.a = umin(rm.a, ~(u128)(unsigned long long)__double_as_longlong(R.maxm[w]));
        rm = block_red<NT>(rm, sred);
        if (tid == 0) X.dec_maxerr[t - 1] = rm.a == kNone ? 0.0 : __longlong_as_double((long long)(unsigned long long)~rm.a);
    }
    if (prof) {                                     // (phase-node, scenario) items evaluated over the run
        unsigned long long tt = (unsigned long long)terms;
        for (int o = 16; o > 0; o >>= 1) tt += __shfl_xor_sync(0xffffffffu, tt, o);
        if ((tid & 31) == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&C->sweep_ns), tt);
    }
    for (int b = tid; b <= n; b += NT) S.sn_rank[b] = rank[b];
    if (tid == 0) {
        C->t = t;
        C->n_super = ns;
        C->candidates += cands_run;
        C->iters += t + (C->stop_reason == 1 ? 1 : 0);
        C->s_cur = fx_to_d(ld128(s_sfx));
        C->rechecks = rechecks;
        C->recheck_cands = recheck_cands;
    }
}

namespace {

// Per-merge data in dynamic shared memory; rec_mode 0: the selection records
// in I.recbuf; 1: in shared memory; 2: in shared memory, with the largest MICE
// per super-node.  se: work entries in shared memory; cw: warps that evaluate
// the merge beside the changed-set scan.
template <int NT, int PREC>
__global__ void __launch_bounds__(NT, 1) k_search_inc(Topo T, State S, Search X, Inc I, Ctrl *C, int verify,
                                                      int rec_mode, int se, int cw, int pre_init) {
    extern __shared__ __align__(16) unsigned char inc_dyn[];
    if (X.setup_err && *X.setup_err != 0) return;           // the setup failed: no result (C->done stays 0)
    inc_run<NT, PREC>(T, S, X, I, C, verify != 0, inc_dyn, rec_mode, se, cw, pre_init != 0);
}

// The first evaluation of every candidate (every slot pair from the initial
// clusters, all singletons, every term), which needs no merge before it: its
// work is spread over many CTAs instead of the one CTA of the search.  The
// CTAs write the candidates, carried sums and tie keys to device memory, in
// the layout the search reads (k_search_inc with pre_init copies the records
// into shared memory and derives the selection keys from the sums).  The
// terms are evaluated by the same code as in the search, so the carried sums
// are the ones the search's own first evaluation gives.
constexpr int kInitPairs = kIncInitPairs;
constexpr int kInitCtasMax = kIncInitCtasMax;
// The first evaluation of one feeder with its work spread evenly over the
// grid.  A pair's candidates can hold up to n positions each (the pairs next
// to the root), so splitting by pairs leaves one CTA with most of the work.
// Instead every CTA derives the position count of every initial candidate
// (the geometry of a pair of singletons is a few loads), lays the candidates'
// positions end to end in slot order, and takes an equal share of them; a
// candidate cut by a share's ends is summed in parts, added to the carried
// sums with 128-bit atomics (integer sums: exact in any order; the sums start
// at zero).  Each pair's own outputs (the slots, its span, the tie keys and
// the dead slots' records) are written by one CTA, and the search derives
// the live candidates' selection keys from the finished sums.
// Dynamic shared memory: the identity super-node list (2n bytes) and the
// position count of every slot (8n bytes).
// CTA b of the B CTAs that evaluate one feeder (dyn: dynamic shared memory of
// 2n + 8n bytes, 16-byte aligned parts).
template <int NT, int PREC>
__device__ void inc_init_share(const Topo &T, const State &S, const Search &X, const Inc &I, Ctrl *C, int b, int B,
                               unsigned char *dyn, EvalSmem<NT> &E, int *sscan, int &s_first, int &s_ne) {
    const int n = T.n, L = T.L, tid = threadIdx.x;
    const int G = 4 * (L <= 1 ? 1 : (L <= 2 ? 2 : 4));
    const double margin = C->margin;
    const float mlo = __double2float_rd(margin), mhi = __double2float_ru(margin);
    unsigned short *list = reinterpret_cast<unsigned short *>(dyn);
    int *pcnt = reinterpret_cast<int *>(dyn + align16((size_t)2 * n));
    for (int w = tid; w < n; w += NT) list[w] = (unsigned short)w;
    Loc Lc;
    Lc.wsm = nullptr;
    Lc.wgl = I.work;
    Lc.se = 0;
    Lc.lst[0] = Lc.lst[1] = list;
    Lc.ph = T.ph;
    Lc.rank = S.sn_rank;
    Rec R;
    R.r0 = reinterpret_cast<u128 *>(I.recbuf);
    R.r1 = reinterpret_cast<ulonglong2 *>(I.recbuf);
    R.tkey = reinterpret_cast<unsigned *>(I.recbuf + (size_t)32 * n);
    R.maxm = I.maxm;
    R.span = reinterpret_cast<ushort4 *>(I.recbuf + (size_t)40 * n);
    R.bsum = nullptr;
    R.bcnt = nullptr;
    R.bmx = nullptr;
    R.dirty = nullptr;
    R.nb = 0;
    Ovl O;
    O.map = nullptr;                            // (the first evaluation reads the stored state only)
    O.cbuf = I.cbuf;
    O.s = O.r = -1;
    O.nfree = 0;
    const View V = no_view();
    // this CTA's pairs: the slots, the span, the tie keys, the dead slots
    for (int w = b + B * tid; w < n; w += B * NT) {
        Cand c[2];
        const int x = slot_geometry(T, S, V, n, w, c[0], c[1]);
        I.qpar[w] = x;
        int lo = n, hi = 0;
        for (int d = 0; d < 2; ++d) {
            if (c[d].s < 0) continue;
            lo = min(lo, min(min(c[d].s, c[d].r), c[d].ns > 0 ? c[d].js : n));
            lo = min(lo, c[d].nr > 0 ? c[d].jr : n);
            hi = max(hi, max(max(c[d].s, c[d].r) + 1, max(c[d].js + c[d].ns, c[d].jr + c[d].nr)));
        }
        const bool any = c[0].s >= 0 || c[1].s >= 0;
        R.span[w] = make_ushort4((unsigned short)(any ? lo : 0), (unsigned short)(any ? hi : 0),
                                 (unsigned short)(x >= 0 ? x : 0xffff), (unsigned short)(any ? 1 : 0));
        for (int d = 0; d < 2; ++d) {
            const int sl = 2 * w + d;
            X.slot[sl] = c[d];
            if (c[d].s >= 0) {
                R.tkey[sl] = (unsigned)c[d].key;
            } else {
                I.viol[sl] = kIncDead;
                kill_rec<PREC>(R, sl);
            }
        }
    }
    // every slot's position count; thread tid takes the pairs [p0, p1)
    const int per = (n + NT - 1) / NT, p0 = min(n, tid * per), p1 = min(n, p0 + per);
    int mine = 0;
    for (int w = p0; w < p1; ++w) {
        Cand c[2];
        slot_geometry(T, S, V, n, w, c[0], c[1]);
        for (int d = 0; d < 2; ++d) {
            int k = 0;
            if (c[d].s >= 0) {
                int2 seg[kIncMaxSeg];
                const int ns = full_segments(c[d], Lc.rank, seg);
                for (int i = 0; i < ns; ++i) k += seg[i].y - seg[i].x;
            }
            pcnt[2 * w + d] = k;
            mine += k;
        }
    }
    if (tid == 0) { s_first = 2 * n; s_ne = 0; }
    int tot = 0;
    const int base = block_excl_scan<NT>(mine, &tot, sscan);
    // this CTA's share of the positions: [q0, q1)
    const int share = max(1, (tot + B - 1) / B);
    const int q0 = min(tot, b * share), q1 = min(tot, q0 + share);
    {
        int off = base;
        for (int sl = 2 * p0; sl < 2 * p1; ++sl) {
            const int k = pcnt[sl];
            if (k > 0 && off < q1 && off + k > q0) atomicMin(&s_first, sl);
            off += k;
        }
    }
    __syncthreads();
    // the entries: one per candidate that meets the share, its segments cut to
    // the share, at [first slot + b, ...) (the CTAs' ranges do not overlap)
    {
        const int e0 = s_first + b;
        int off = base;
        for (int sl = 2 * p0; sl < 2 * p1; ++sl) {
            const int k = pcnt[sl];
            if (k > 0 && off < q1 && off + k > q0) {
                Cand c[2];
                slot_geometry(T, S, V, n, sl >> 1, c[0], c[1]);
                const Cand &cc = c[sl & 1];
                int2 seg[kIncMaxSeg], cut[kIncMaxSeg];
                const int ns = full_segments(cc, Lc.rank, seg);
                const int lo = max(q0 - off, 0), hi = min(q1 - off, k);    // the share, in the candidate's positions
                int nc = 0, at = 0;
                for (int i = 0; i < ns; ++i) {
                    const int len = seg[i].y - seg[i].x;
                    const int a = max(lo, at), z = min(hi, at + len);
                    if (a < z) cut[nc++] = make_int2(seg[i].x + (a - at), seg[i].x + (z - at));
                    at += len;
                }
                write_entry(Lc.ent(e0 + atomicAdd(&s_ne, 1)), sl, 1, nc, cut, cc);
            }
            off += k;
        }
    }
    __syncthreads();
    if (s_ne == 0) return;
    const long long terms = run_entries<NT, PREC>(T, S, X, I, n, L, G, margin, mlo, mhi, s_first + b, s_first + b + s_ne,
                                                  kInitPart, list, list, -1, O, E, sscan, R, Lc);
    if (C->profile) {                           // (phase-node, scenario) items
        unsigned long long tt = (unsigned long long)terms;
        for (int o = 16; o > 0; o >>= 1) tt += __shfl_xor_sync(0xffffffffu, tt, o);
        if ((tid & 31) == 0 && tt) atomicAdd(reinterpret_cast<unsigned long long *>(&C->sweep_ns), tt);
    }
}

template <int NT, int PREC>
__global__ void __launch_bounds__(NT) k_inc_init(Topo T, State S, Search X, Inc I, Ctrl *C) {
    extern __shared__ __align__(16) unsigned char init_dyn[];
    __shared__ __align__(16) EvalSmem<NT> E;
    __shared__ int sscan[33];
    __shared__ int s_first, s_ne;
    if (X.setup_err && *X.setup_err != 0) return;
    inc_init_share<NT, PREC>(T, S, X, I, C, blockIdx.x, gridDim.x, init_dyn, E, sscan, s_first, s_ne);
}

// The same for many feeders: cta_off[i] = the first CTA of the i-th feeder of
// the order (the feeder's CTAs end where the next feeder's begin, the last
// feeder's at the end of the grid); each feeder's CTAs split its positions
// as above.  Feeders whose setup failed are skipped.  The carried sums of
// every feeder start at zero (k_inc_zero_batch).
template <int NT, int PREC>
__global__ void __launch_bounds__(NT) k_inc_init_batch(const BatchFeeder *fd, const int *order, const int *cta_off,
                                                       int nf) {
    extern __shared__ __align__(16) unsigned char init_dyn[];
    __shared__ __align__(16) EvalSmem<NT> E;
    __shared__ int sscan[33];
    __shared__ int s_first, s_ne;
    __shared__ Topo sT;
    __shared__ State sS;
    __shared__ Search sX;
    __shared__ Inc sI;
    __shared__ int s_f, s_b, s_B;
    const int b = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nf - 1;                 // the last feeder whose first CTA is <= b
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cta_off[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        const int f = order[lo];
        s_f = f;
        s_b = b - cta_off[lo];
        s_B = (lo + 1 < nf ? cta_off[lo + 1] : (int)gridDim.x) - cta_off[lo];
        sT = fd[f].T;
        sS = fd[f].S;
        sX = fd[f].X;
        sI = fd[f].I;
    }
    __syncthreads();
    const int f = s_f;
    if (*fd[f].setup_err != 0 || s_b >= s_B) return;
    inc_init_share<NT, PREC>(sT, sS, sX, sI, fd[f].C, s_b, s_B, init_dyn, E, sscan, s_first, s_ne);
}

// The carried sums, violation counts and their bounds of every feeder of the
// order set to zero before its first evaluation adds to them (one CTA per
// feeder).
__global__ void k_inc_zero_batch(const BatchFeeder *fd, const int *order, int nf) {
    const int q = blockIdx.x;
    if (q >= nf) return;
    const Inc &I = fd[order[q]].I;
    const int n = fd[order[q]].T.n;
    unsigned char *p0 = reinterpret_cast<unsigned char *>(I.acc);
    const size_t bytes = reinterpret_cast<const unsigned char *>(I.vmay + 2 * (size_t)n) - p0;
    for (size_t i = threadIdx.x; i < bytes / 4; i += blockDim.x) reinterpret_cast<unsigned *>(p0)[i] = 0u;
}

// One CTA per feeder, feeders in the order given (largest first).
template <int NT, int PREC>
__global__ void __launch_bounds__(NT) k_search_inc_batch(const BatchFeeder *fd, const int *order, int nf,
                                                         int rec_mode, int se, int cw, int pre_init) {
    extern __shared__ __align__(16) unsigned char inc_dyn[];
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
    if (ok) inc_run<NT, PREC>(sT, sS, sX, sI, C, false, inc_dyn, rec_mode, se, cw, pre_init != 0);
    __syncthreads();
    for (int i = threadIdx.x; i < sT.n; i += NT) fd[f].super_out[i] = ok ? sT.orig[sS.label[sT.pre[i]]] : -1;
    if (threadIdx.x == 0) {
        const int t = ok ? C->t : 0;
        *fd[f].max_err = t > 0 ? sX.dec_maxerr[t - 1] : 0.0;
    }
}

constexpr size_t kIncSmemMax = 200 * 1024;  // largest dynamic shared memory of one search
constexpr int kInitThreads = 384;           // CTAs of the first evaluation

template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

IncShape inc_shape_resolve(IncShape sh) {
    if (sh.threads != 256 && sh.threads != 384 && sh.threads != 512) sh.threads = kIncDefaultThreads;
    const int nw = sh.threads / 32;
    if (sh.cw < 1 || sh.cw > nw - 1) sh.cw = sh.threads == 512 ? 4 : 2;
    if (sh.se < 1 || sh.se > kSEMax) sh.se = kSEMax;
    if (sh.rec < -1 || sh.rec > 2) sh.rec = -1;
    return sh;
}

// Dynamic shared memory for an n-bus feeder: the per-merge data always, the
// selection records (and, when `maxm`, the largest MICE per super-node) when
// the total stays within kIncSmemMax, or where sh.rec places them.  Returns
// false when a forced placement does not fit (or asks for the per-super-node
// maximum where `maxm` is false).
bool inc_smem(int n, bool maxm, const IncShape &sh, int *rec_mode, size_t *bytes) {
    const size_t base = base_bytes(n, sh.se);
    const bool fit2 = maxm && base + rec_maxm_bytes(n) <= kIncSmemMax;
    const bool fit1 = base + rec_bytes(n) <= kIncSmemMax;
    int m = sh.rec;
    if (m < 0) m = fit2 ? 2 : (fit1 ? 1 : 0);
    if ((m == 2 && !fit2) || (m == 1 && !fit1) || base > kIncSmemMax) return false;
    *rec_mode = m;
    *bytes = m == 2 ? base + rec_maxm_bytes(n) : (m == 1 ? base + rec_bytes(n) : base);
    return true;
}

namespace {

template <int NT, int PREC>
cudaError_t launch_one(Topo T, State S, Search X, Inc I, Ctrl *C, int verify, int use, size_t smem, const IncShape &sh,
                       cudaStream_t st) {
    // the first evaluation spread over the SMs (its sums start at zero), then
    // the search on one CTA
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || sms < 1)
            sms = 1;
    }
    const int ginit = std::min(std::min(sms, kInitCtasMax), std::max(1, (T.n + kInitPairs - 1) / kInitPairs));
    const size_t ismem = align16((size_t)2 * T.n) + align16((size_t)8 * T.n);
    cudaError_t e = cudaMemsetAsync(I.acc, 0, reinterpret_cast<const char *>(I.vmay + 2 * (size_t)T.n) -
                                                  reinterpret_cast<const char *>(I.acc), st);
    if (e == cudaSuccess && ismem > 48 * 1024) e = set_smem(k_inc_init<kInitThreads, PREC>, ismem);
    if (e == cudaSuccess) k_inc_init<kInitThreads, PREC><<<ginit, kInitThreads, ismem, st>>>(T, S, X, I, C);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = set_smem(k_search_inc<NT, PREC>, smem);
    if (e == cudaSuccess) k_search_inc<NT, PREC><<<1, NT, smem, st>>>(T, S, X, I, C, verify, use, sh.se, sh.cw, 1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int NT>
cudaError_t set_batch_smem(int precision, size_t smem) {
    return precision == 1 ? set_smem(k_search_inc_batch<NT, 1>, smem) : set_smem(k_search_inc_batch<NT, 0>, smem);
}

template <int NT>
void launch_batch(int precision, const BatchFeeder *fd, const int *order, int nf, int use, size_t smem,
                  const IncShape &sh, cudaStream_t st) {
    if (precision == 1) k_search_inc_batch<NT, 1><<<nf, NT, smem, st>>>(fd, order, nf, use, sh.se, sh.cw, 1);
    else k_search_inc_batch<NT, 0><<<nf, NT, smem, st>>>(fd, order, nf, use, sh.se, sh.cw, 1);
}

}  // namespace

cudaError_t launch_search_inc(int precision, Topo T, State S, Search X, Inc I, Ctrl *C, int verify, IncShape sh,
                              int *rec_used, cudaStream_t st) {
    sh = inc_shape_resolve(sh);
    int use = 0;
    size_t smem = 0;
    if (!inc_smem(T.n, true, sh, &use, &smem)) return cudaErrorInvalidValue;
    if (rec_used) *rec_used = use;
    if (sh.threads == 256)
        return precision == 1 ? launch_one<256, 1>(T, S, X, I, C, verify, use, smem, sh, st)
                              : launch_one<256, 0>(T, S, X, I, C, verify, use, smem, sh, st);
    if (sh.threads == 384)
        return precision == 1 ? launch_one<384, 1>(T, S, X, I, C, verify, use, smem, sh, st)
                              : launch_one<384, 0>(T, S, X, I, C, verify, use, smem, sh, st);
    return precision == 1 ? launch_one<512, 1>(T, S, X, I, C, verify, use, smem, sh, st)
                          : launch_one<512, 0>(T, S, X, I, C, verify, use, smem, sh, st);
}

cudaError_t prepare_search_inc_batch(int precision, int max_n, IncShape sh) {
    sh = inc_shape_resolve(sh);
    int use = 0;
    size_t smem = 0;
    if (!inc_smem(max_n, false, sh, &use, &smem)) return cudaErrorInvalidValue;
    if (sh.threads == 384) return set_batch_smem<384>(precision, smem);
    return sh.threads == 256 ? set_batch_smem<256>(precision, smem) : set_batch_smem<512>(precision, smem);
}

cudaError_t launch_search_inc_batch(int precision, int max_n, const BatchFeeder *fd, const int *order, int nf,
                                    IncShape sh, cudaStream_t st) {
    if (nf <= 0) return cudaSuccess;
    sh = inc_shape_resolve(sh);
    int use = 0;
    size_t smem = 0;
    if (!inc_smem(max_n, false, sh, &use, &smem)) return cudaErrorInvalidValue;
    if (sh.threads == 256) launch_batch<256>(precision, fd, order, nf, use, smem, sh, st);
    else if (sh.threads == 384) launch_batch<384>(precision, fd, order, nf, use, smem, sh, st);
    else launch_batch<512>(precision, fd, order, nf, use, smem, sh, st);
    return cudaGetLastError();
}

cudaError_t prepare_inc_init_batch(int precision, int max_n) {
    const size_t ismem = align16((size_t)2 * max_n) + align16((size_t)8 * max_n);
    if (ismem <= 48 * 1024) return cudaSuccess;
    return precision == 1 ? set_smem(k_inc_init_batch<kInitThreads, 1>, ismem)
                          : set_smem(k_inc_init_batch<kInitThreads, 0>, ismem);
}

cudaError_t launch_inc_init_batch(int precision, int max_n, const BatchFeeder *fd, const int *order,
                                  const int *cta_off, int nf, int ctas, cudaStream_t st) {
    if (nf <= 0 || ctas <= 0) return cudaSuccess;
    const size_t ismem = align16((size_t)2 * max_n) + align16((size_t)8 * max_n);
    k_inc_zero_batch<<<nf, 256, 0, st>>>(fd, order, nf);
    if (precision == 1) k_inc_init_batch<kInitThreads, 1><<<ctas, kInitThreads, ismem, st>>>(fd, order, cta_off, nf);
    else k_inc_init_batch<kInitThreads, 0><<<ctas, kInitThreads, ismem, st>>>(fd, order, cta_off, nf);
    return cudaGetLastError();
}

}  // namespace okr
