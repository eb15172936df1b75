// okr_persist.cu -- the exhaustive search (Algorithm 1, Sec. IV) as one
// persistent cooperative kernel, one CTA per SM, three grid barriers per
// iteration (four when an FP64 recheck is needed):
//
//   phase 1  select + commit of the last sweep (argmin with the tie band, then
//            the merge), fused with the candidate setup of the next sweep
//   phase 2  candidate compaction, work positions, chunk map, super-node list,
//            bookkeeping of the merge
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
// one dense position space, candidates back to back.  A sweep gives each
// position four lanes, one per phase (the fourth idles), and each lane takes the
// scenarios in turn, so a warp holds eight positions: on a 1,000-bus feeder an
// iteration's positions then fit in about one warp each, and the sweep's time is
// one warp's chain of dependent loads rather than two.  (The merge's items use
// one lane per (scenario, phase): 4 * Lp lanes, Lp = scenarios rounded up to a
// power of two.)  Per-candidate sums are reduced in a fixed order (phase
// shuffles, scenarios in order, a segmented warp scan, then the pieces of a
// candidate in chunk order), so results do not depend on timing.
//
// Precision.  precision 0 scores every candidate in FP64.  precision 1 screens
// every candidate in FP32 with a rigorous bound B(c) on the distance between the
// screened score and the FP64 one (and a bound on the screened largest MICE), then
//   U = min over surely feasible candidates of D32(c) + B(c),
//   R = { c not surely infeasible : D32(c) - B(c) <= U + tau }.
// The FP64 minimum and every candidate of its tie band lie in R.  When R holds
// one surely feasible candidate, it is the FP64 winner; otherwise R is scored
// again in FP64 and the selection runs on those scores.  The merge itself is
// always applied in FP64, so the state carried between iterations is FP64 in
// both modes and the FP32 copies are refreshed from it.
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
__device__ __forceinline__ float ldf(const float *p) { return __ldcg(p); }
__device__ __forceinline__ float2 ldf2(const float2 *p) { return __ldcg(p); }
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
// The arrival counter only grows: barrier number k (counted per CTA) completes
// when it reaches k * gridDim.x.  Thread 0 of each CTA publishes the CTA's
// writes (fence, then the arrival) and polls with acquire loads.  Every wait is
// bounded: after max_spins polls the CTA records err = 6 and the kernel unwinds
// (each CTA leaves at its next barrier, whose wait also ends on the error flag).
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ bool grid_barrier(GridBar *gb, Ctrl *C, unsigned nblocks, unsigned &epoch) {
    __shared__ int s_ok;
    __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        const unsigned target = epoch * nblocks;
        __threadfence();
        atomicAdd(&gb->count, 1u);
        int ok = 1;
        long long spins = 0;
        const long long lim = C->max_spins;
        // one L2 round trip per poll; another CTA's give-up is looked for every 64 polls
        while (ld_acquire(&gb->count) < target) {
            if (++spins > lim || ((spins & 63) == 0 && *(volatile int *)&C->err)) { ok = 0; break; }
        }
        if (!ok) atomicCAS(&C->err, 0, 6);
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok;
}

// Barrier of the CTAs that share one feeder: the whole grid (G > 1), or one
// CTA (G == 1), where a fence and __syncthreads suffice.
__device__ __forceinline__ bool team_barrier(GridBar *gb, Ctrl *C, unsigned G, unsigned &epoch) {
    if (G == 1) {
        __threadfence();
        __syncthreads();
        epoch += 1;
        return true;
    }
    return grid_barrier(gb, C, G, epoch);
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
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

// Tie key: (caller r, caller s) lexicographic; caller ids are < 2^15.
__device__ __forceinline__ unsigned long long tie_key(const Topo &T, int s, int r) {
    return ((unsigned long long)(unsigned)T.orig[r] << 15) | (unsigned)T.orig[s];
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
// Scenario l, phase p of the cluster of super-node k for candidate cd.  k < 0
// stands for s's cluster when s is the common ancestor (no voltage change).
struct Item64 {
    double e;       // largest member error max(hi - |V|, |V| - lo), merged extremes for s
    double m;       // |V|
    double2 v;      // new voltage
    bool on;        // phase present
};

__device__ __forceinline__ Item64 eval_item64(const Topo &T, const State &S, int n, const Cand &cd, int k, bool sside,
                                              int l, int p, const double2 *Ir, unsigned phr) {
    Item64 o;
    o.e = 0.0;
    o.m = 0.0;
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
    o.m = mag;
    o.v = v;
    o.on = true;
    return o;
}

// Single-precision screen of the same item with a bound b on |e32 - e64|.
// With u = 2^-24 and S = sum_q |G_pq| |I_q| (1-norms of the complex numbers):
//   G from the split path impedances: relative error <= 3u; I rounded: u;
//   products and sums: <= 4u S, so |dV32 - dV| <= 8u S;
//   delta = |V + dV| - |V| = (2 Re(conj V dV) + |dV|^2) / (|V + dV| + |V|):
//     numerator error <= u (23 |V|_1 + 3 |V|_1 + 11 |V|_1 + 11 S) S,
//     denominator relative error <= 4u, division u;
//   e = max(hr - delta, delta - lr) with hr, lr rounded from FP64 differences.
// The constants below round these up (40 for the numerator, 8 |delta|) and the
// whole bound carries a factor 1.5 and an additive 4e-15 for the FP64 path's own
// rounding.  Merged extremes of s and r add the rounding of the shift
// |V_r| - |V_s| and of the shifted extremes.
struct Item32 {
    float e, b;
};

constexpr float kU = 5.9604645e-08f;    // 2^-24

__device__ __forceinline__ Item32 eval_item32(const Topo &T, const State &S, int n, const Cand &cd, int k, bool sside,
                                              int l, int p, const float2 *Ir, unsigned phr, float &flops) {
    Item32 o;
    o.e = 0.0f;
    o.b = 0.0f;
    const int kk = k < 0 ? cd.s : k;
    if (!(T.ph[kk] >> p & 1u)) return o;
    const size_t ik = sidx(l, p, kk, n);
    float hr = ldf(S.hr32 + ik), lr = ldf(S.lr32 + ik);
    float bx = 0.0f;
    if (kk == cd.s && (T.ph[cd.r] >> p & 1u)) {
        const size_t ir = sidx(l, p, cd.r, n);
        const float dr = (float)(ldd(S.mcur + ir) - ldd(S.mcur + ik));
        const float hrr = ldf(S.hr32 + ir) + dr, lrr = ldf(S.lr32 + ir) + dr;
        hr = fmaxf(hr, hrr);
        lr = fminf(lr, lrr);
        bx = 2.0f * kU * (fabsf(hrr) + fabsf(lrr) + 2.0f * fabsf(dr));
    }
    float delta = 0.0f, bd = 0.0f;
    if (k >= 0) {
        const float2 v = ldf2(S.v32 + ik);
        const int y = T.lca[(size_t)(sside ? cd.s : cd.r) * n + k];
        const float2 *zhy = T.zh + (size_t)y * 9 + p * 3, *zly = T.zlo + (size_t)y * 9 + p * 3;
        const float2 *zha = T.zh + (size_t)cd.a * 9 + p * 3, *zla = T.zlo + (size_t)cd.a * 9 + p * 3;
        float2 dv = make_float2(0.0f, 0.0f);
        float sdv = 0.0f;
        for (int q = 0; q < 3; ++q) {
            if (!(phr >> q & 1u)) continue;
            float gx = (zhy[q].x - zha[q].x) + (zly[q].x - zla[q].x);
            float gy = (zhy[q].y - zha[q].y) + (zly[q].y - zla[q].y);
            if (!sside) { gx = -gx; gy = -gy; }
            dv.x = fmaf(gx, Ir[q].x, fmaf(-gy, Ir[q].y, dv.x));
            dv.y = fmaf(gx, Ir[q].y, fmaf(gy, Ir[q].x, dv.y));
            sdv = fmaf(fabsf(gx) + fabsf(gy), fabsf(Ir[q].x) + fabsf(Ir[q].y), sdv);
        }
        const float num = 2.0f * (v.x * dv.x + v.y * dv.y) + (dv.x * dv.x + dv.y * dv.y);
        const float wx = v.x + dv.x, wy = v.y + dv.y;
        const float mv = sqrtf(v.x * v.x + v.y * v.y);
        const float den = sqrtf(wx * wx + wy * wy) + mv;
        delta = num / den;
        const float v1 = fabsf(v.x) + fabsf(v.y);
        bd = kU * (40.0f * (v1 + sdv) * sdv / den + 8.0f * fabsf(delta));
        flops += 10.0f * __popc(phr) + 14.0f;
    }
    o.e = fmaxf(hr - delta, delta - lr);
    o.b = 1.5f * (kU * (fabsf(hr) + fabsf(lr) + fabsf(o.e)) + bd) + bx + 4e-15f;
    return o;
}

// ---------------------------------------------------------------- chunk scoring
// One warp scores PPW consecutive positions.  Per lane: `ci` the candidate slot
// its position belongs to (used for the partial-sum slot g + ci, the arrival
// counter and the outputs), `cd` the candidate, `q` the position inside the
// candidate, `first` the candidate's first chunk, `np` its chunk count.  Lanes of
// a position reduce over phases (xor 1, 2), then over scenarios (xor 4, 8); the
// lanes of a candidate reduce with a segmented scan in lane order; the last lane
// of a segment stores the piece and the writer of the last piece sums the
// pieces in order.
// Lane `lane` holds the first position cb of candidate c0 + lane (candidates in
// increasing order, c0 owning the chunk's first position q0).  Returns, for a
// lane at position q0 + u, the offset of its candidate from c0: one ballot per
// position of the chunk.
__device__ __forceinline__ int chunk_offset(int cb, int q0, int ppw, int u) {
    int off = 0;
    for (int v = 0; v < ppw; ++v) {
        const int c = __popc(__ballot_sync(0xffffffffu, cb <= q0 + v)) - 1;
        if (v == u) off = c;
    }
    return off;
}

__device__ __forceinline__ void seg_scan_setup(bool active, int ci, int lane, unsigned &heads, int &seg_start,
                                               bool &last) {
    const int cseg = active ? ci : -1 - lane;
    const int prev = __shfl_up_sync(0xffffffffu, cseg, 1);
    const bool head = (lane == 0) || (prev != cseg);
    heads = __ballot_sync(0xffffffffu, head);
    seg_start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    last = (lane == 31) || ((heads >> (lane + 1)) & 1u);
}

// ---------------------------------------------------------------- learned pruning
// The scorer's weights in shared memory (bfloat16 bit patterns; biases FP32).
constexpr int kMlpH = 128;
struct MlpSmem {
    uint16_t w2[kMlpH * kMlpH], w3[kMlpH * kMlpH], w1[kScorerFeatures * kMlpH], w4[kMlpH];
    float b1[kMlpH], b2[kMlpH], b3[kMlpH], b4;
    float feat[kThreads / 32][16];          // per-warp feature scratch
};

__device__ __forceinline__ float bf16f(uint16_t b) { return __uint_as_float((unsigned)b << 16); }

// Order-preserving key of a float (smaller key = smaller value).
__device__ __forceinline__ unsigned fkey(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ void mlp_load_smem(const Search &X, MlpSmem *W) {
    const int F = kScorerFeatures;
    const float *th = X.mlp_theta;
    const int o_b1 = F * kMlpH, o_b2 = o_b1 + kMlpH + kMlpH * kMlpH, o_b3 = o_b2 + kMlpH + kMlpH * kMlpH;
    const int o_b4 = o_b3 + kMlpH + kMlpH;
    for (int e = threadIdx.x; e < kMlpH * kMlpH; e += blockDim.x) {
        W->w2[e] = X.mlp_w2[e];
        W->w3[e] = X.mlp_w3[e];
    }
    for (int e = threadIdx.x; e < F * kMlpH; e += blockDim.x) W->w1[e] = X.mlp_w1[e];
    for (int e = threadIdx.x; e < kMlpH; e += blockDim.x) {
        W->w4[e] = X.mlp_w4[e];
        W->b1[e] = th[o_b1 + e];
        W->b2[e] = th[o_b2 + e];
        W->b3[e] = th[o_b3 + e];
    }
    if (threadIdx.x == 0) W->b4 = th[o_b4];
}

// One candidate's prediction by one warp (the same products, in the same order,
// as the training kernels' forward pass).  f: the warp's feature scratch.
__device__ float mlp_predict_warp(const MlpSmem *W, const float *f) {
    const int lane = threadIdx.x & 31;
    float h[4], g[4];
    // (unrolled, so that the shuffles and weight loads of later k issue ahead
    // of the multiply-adds they feed: one prediction is a latency chain)
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int j = lane + 32 * m;
        float z = W->b1[j];
#pragma unroll
        for (int k = 0; k < kScorerFeatures; ++k) z = fmaf(f[k], bf16f(W->w1[k * kMlpH + j]), z);
        h[m] = fmaxf(z, 0.0f);
    }
#pragma unroll 1
    for (int layer = 0; layer < 2; ++layer) {
        const uint16_t *w = layer == 0 ? W->w2 : W->w3;
        const float *bias = layer == 0 ? W->b2 : W->b3;
#pragma unroll
        for (int m = 0; m < 4; ++m) g[m] = bias[lane + 32 * m];
#pragma unroll
        for (int ms = 0; ms < 4; ++ms)
#pragma unroll 8
            for (int sl = 0; sl < 32; ++sl) {
                const float hk = __shfl_sync(0xffffffffu, h[ms], sl);
                const int k = ms * 32 + sl;
#pragma unroll
                for (int m = 0; m < 4; ++m) g[m] = fmaf(hk, bf16f(w[k * kMlpH + lane + 32 * m]), g[m]);
            }
#pragma unroll
        for (int m = 0; m < 4; ++m) h[m] = fmaxf(g[m], 0.0f);
    }
    float acc = h[0] * bf16f(W->w4[lane]) + h[1] * bf16f(W->w4[lane + 32]) + h[2] * bf16f(W->w4[lane + 64]) +
                h[3] * bf16f(W->w4[lane + 96]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc + W->b4;
}

// Key of the k-th smallest prediction over the candidate slots (radix select,
// four 8-bit digits; every CTA computes it).  Returns ~0u when k >= nc.
__device__ unsigned topk_threshold(const Search &X, int nslots, int k, int nc) {
    if (k >= nc) return ~0u;
    __shared__ unsigned hist[256];
    __shared__ unsigned s_prefix, s_need;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) { s_prefix = 0u; s_need = (unsigned)k; }
    unsigned mask = 0u;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0u;
        __syncthreads();
        const unsigned prefix = s_prefix;
        for (int i = tid; i < nslots; i += blockDim.x) {
            const unsigned key = fkey(__ldcg(X.pred + i));
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid < 32) {                             // the digit holding the need-th key
            unsigned c[8], tot = 0u;
            for (int q = 0; q < 8; ++q) { c[q] = hist[lane * 8 + q]; tot += c[q]; }
            unsigned incl = tot;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned excl = incl - tot, need = s_need;
            const bool mine = excl < need && need <= incl;
            if (mine) {
                unsigned cum = excl;
                int b = 0;
                for (int q = 0; q < 8; ++q) {
                    if (cum + c[q] >= need) { b = q; break; }
                    cum += c[q];
                }
                s_prefix = prefix | ((unsigned)(lane * 8 + b) << shift);
                s_need = need - cum;
            }
        }
        mask |= 255u << shift;
        __syncthreads();
    }
    return s_prefix;
}

// What a candidate's features depend on besides its clusters' state: s, r,
// the common ancestor, the direction and the count of affected clusters,
// packed (~0: not packable, n above 2^16; the prediction is then made again).
__device__ __forceinline__ unsigned long long pred_key(const Cand &c, int n) {
    const unsigned cnt = (unsigned)(c.ns + c.nr);
    if (n >= 65536 || cnt >= (1u << 15)) return ~0ull;
    return (unsigned long long)c.s | ((unsigned long long)c.r << 16) | ((unsigned long long)c.a << 32) |
           ((unsigned long long)(c.dir & 1) << 48) | ((unsigned long long)cnt << 49);
}

__device__ __forceinline__ bool slot_selected(const Search &X, const Cand &c, unsigned theta) {
    return theta == ~0u || fkey(__ldcg(X.pred + c.pad)) <= theta;
}

// ---------------------------------------------------------------- certified pruning
// A cluster evaluated at one voltage magnitude m has, per scenario, MICE =
// max over members and phases of | |Vhat| - m | >= max over phases of
// (hi - lo) / 2, half the spread of its members' |Vhat|.  A candidate (s, r)
// changes SMICE by (new MICE of s u r) - MICE_s - MICE_r plus, over its other
// positions k, (new MICE_k) - MICE_k: the clusters outside its positions keep
// their voltages.  With g_k = sum_l (max_p (hi - lo) / 2 - MICE_{k,l}) <= 0
// the change is therefore at least
//   sum_l (max_p (max(hi_s, hi_r) - min(lo_s, lo_r)) / 2 - MICE_s - MICE_r)
//   + the sum of g_k over the positions other than s and r.
// The positions are the super-nodes whose ranks lie in the candidate's two
// ranges (and s).  Their sum comes from prefix sums over ranks of
// floor(g_k 2^56), exact in 64-bit integers (g_k rounded down), less the
// values of s and r where their ranks lie in the ranges; the candidate's own
// part is rounded down.
__device__ __forceinline__ double half_spread_rd(double hi, double lo) { return __dmul_rd(__dsub_rd(hi, lo), 0.5); }
// floor(g_k 2^56) (|g_k| <= L: no overflow).
__device__ long long cluster_g_fx(const Topo &T, const State &S, int n, int L, int k) {
    const unsigned ph = T.ph[k];
    double g = 0.0;
    for (int l = 0; l < L; ++l) {
        double hs = 0.0;
        for (int p = 0; p < 3; ++p)
            if (ph >> p & 1u) hs = fmax(hs, half_spread_rd(ldd(S.hi + sidx(l, p, k, n)), ldd(S.lo + sidx(l, p, k, n))));
        g = __dadd_rd(g, __dsub_rd(hs, ldd(S.mice + (size_t)l * n + k)));
    }
    return __double2ll_rd(g * 72057594037927936.0);
}
// The candidate's own part of its bound (rounded down); +inf when the merged
// cluster's half spread exceeds the margin in some scenario (surely infeasible).
__device__ double cand_lb_part(const Topo &T, const State &S, int n, int L, const Cand &c, double margin) {
    const unsigned phs = T.ph[c.s], phr = T.ph[c.r];
    double part = 0.0;
    for (int l = 0; l < L; ++l) {
        double hs = 0.0;
        for (int p = 0; p < 3; ++p) {
            if (!(phs >> p & 1u)) continue;
            double hi = ldd(S.hi + sidx(l, p, c.s, n)), lo = ldd(S.lo + sidx(l, p, c.s, n));
            if (phr >> p & 1u) {
                hi = fmax(hi, ldd(S.hi + sidx(l, p, c.r, n)));
                lo = fmin(lo, ldd(S.lo + sidx(l, p, c.r, n)));
            }
            hs = fmax(hs, half_spread_rd(hi, lo));
        }
        if (hs > margin) return INFINITY;
        const double ms = ldd(S.mice + (size_t)l * n + c.s), mr = ldd(S.mice + (size_t)l * n + c.r);
        part = __dadd_rd(part, __dsub_rd(__dsub_rd(hs, ms), mr));
    }
    return part;
}
// The candidate's own part, kept per candidate like the scorer's predictions
// (it reads only s's and r's state): computed again when the candidate changed
// or s or r took part in the merge that made state number t.
__device__ double cand_lb_part_kept(const Topo &T, const State &S, const Search &X, int n, int L, const Cand &c,
                                    double margin, int t) {
    const int cs = 2 * (c.dir == 0 ? c.r : c.s) + c.dir;
    const unsigned long long key = pred_key(c, n);
    if (key != ~0ull && __ldcg(X.lbkey + cs) == key && ldi(X.moved + c.s) != t && ldi(X.moved + c.r) != t)
        return ldd(X.lbc + cs);
    const double part = cand_lb_part(T, S, n, L, c, margin);
    X.lbc[cs] = part;
    X.lbkey[cs] = key;
    return part;
}
// The sum of floor(g_k 2^56) over the ranks below j: the blocks of 32 ranks
// before j's (gbp) and the ranks of j's block below j (gpre, inclusive per block).
__device__ __forceinline__ long long g_prefix(const Search &X, int j) {
    long long v = __ldcg(X.gbp + (j >> 5));
    if (j & 31) v += __ldcg(X.gpre + j - 1);
    return v;
}
// Whether the bound excludes candidate ci from the tie band: its lower bound
// on the score change exceeds thr (or it is surely infeasible).
__device__ __forceinline__ bool lb_excludes(const Search &X, const State &S, int ci, const Cand &cd, double thr) {
    const double part = ldd(X.lbp + ci);
    if (isinf(part)) return true;
    long long g = 0;
    if (cd.ns > 0) g += g_prefix(X, cd.js + cd.ns) - g_prefix(X, cd.js);
    if (cd.nr > 0) g += g_prefix(X, cd.jr + cd.nr) - g_prefix(X, cd.jr);
    auto in_ranges = [&](int j) {
        return (j >= cd.js && j < cd.js + cd.ns) || (j >= cd.jr && j < cd.jr + cd.nr);
    };
    const int rs = ldi(S.sn_rank + cd.s), rr = ldi(S.sn_rank + cd.r);
    if (in_ranges(rs)) g -= g_prefix(X, rs + 1) - g_prefix(X, rs);
    if (in_ranges(rr)) g -= g_prefix(X, rr + 1) - g_prefix(X, rr);
    return __dadd_rd(part, __ll2double_rd(g) * 1.3877787807814457e-17) > thr;      // 2^-56
}

// Objective 1: the largest MICE among the clusters a candidate leaves unchanged,
// i.e. over the super-node ranks outside [js, js+ns), [jr, jr+nr) and, when s is
// the common ancestor, s's own rank.  Whole blocks of 32 ranks come from bmax,
// the (at most five) partly excluded blocks rank by rank.  Warp-cooperative; the
// result is returned to every lane.
__device__ __forceinline__ double unaffected_max(const Search &X, int nsn, int js, int ns, int jr, int nr, int jfix) {
    const int lane = threadIdx.x & 31;
    double u = 0.0;
    const int nb = (nsn + 31) >> 5;
    for (int b = lane; b < nb; b += 32) {
        const int lo = b << 5, hi = min(nsn, lo + 32);
        const bool touch = (js < hi && js + ns > lo && ns > 0) || (jr < hi && jr + nr > lo && nr > 0) ||
                           (jfix >= lo && jfix < hi);
        if (!touch) {
            u = fmax(u, ldd(X.bmax + b));
        } else {
            for (int j = lo; j < hi; ++j) {
                const bool ex = (j >= js && j < js + ns) || (j >= jr && j < jr + nr) || j == jfix;
                if (!ex) u = fmax(u, ldd(X.mrank + j));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) u = fmax(u, __shfl_xor_sync(0xffffffffu, u, o));
    return u;
}

__device__ void score64_chunk(const Topo &T, const State &S, const Search &X, int n, int L, int SP, int g,
                              bool active, int ci, const Cand &cd, int q, int first, int np, const int *list,
                              double margin, double *out_score, int *out_feas, bool prof, double &flops,
                              bool obj1 = false, int nsn = 0, unsigned theta = ~0u, int pmode = 0,
                              double pthr = 0.0, int *n_excl = nullptr) {
    // one lane per phase (SP == 4), the scenarios in turn inside the lane
    const int lane = threadIdx.x & 31, p = lane & 3;
    // pmode 0: the candidates the learned pruning keeps (all with theta = ~0u);
    // pmode 1: the certified pruning's second pass, the candidates the first
    // pass left out and the bound does not exclude (the others keep their scores)
    bool chosen = !active || slot_selected(X, cd, theta);
    if (pmode == 1 && active) {
        const bool excl = !chosen && lb_excludes(X, S, ci, cd, pthr);
        if (excl && q == 0 && p == 0) ++*n_excl;        // counted once per candidate
        chosen = !chosen && !excl;
    }
    int k = cd.r;
    bool sside = false;
    if (active && chosen) k = position_bus(list, cd, q, sside);
    const bool valid = active && chosen && k != cd.r;
    const int kk = k < 0 ? cd.s : k;
    double dl = 0.0, ml = 0.0;
    for (int l = 0; l < L; ++l) {
        Item64 o;
        o.e = 0.0;
        o.on = false;
        if (valid && p < 3) {
            double2 Ir[3];
            for (int qq = 0; qq < 3; ++qq) Ir[qq] = ldz(S.icur + sidx(l, qq, cd.r, n));
            o = eval_item64(T, S, n, cd, k, sside, l, p, Ir, T.ph[cd.r]);
            if (prof && o.on) flops += (k < 0) ? 8.0 : 10.0 * __popc(T.ph[cd.r]) + 10.0;
        }
        double m = o.e;
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 1));
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 2));
        if (valid && p == 0) {
            double d = m - ldd(S.mice + (size_t)l * n + kk);
            if (kk == cd.s) d -= ldd(S.mice + (size_t)l * n + cd.r);
            dl += d;
            ml = fmax(ml, m);
        }
    }
    if (p != 0) { dl = 0.0; ml = 0.0; }
    unsigned heads;
    int seg_start;
    bool last;
    seg_scan_setup(active, ci, lane, heads, seg_start, last);
    for (int o2 = 1; o2 < 32; o2 <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, dl, o2);
        const double z = __shfl_up_sync(0xffffffffu, ml, o2);
        if (lane - o2 >= seg_start) { dl += y; ml = fmax(ml, z); }
    }
    bool fin = false, direct = false;
    if (active && last) {
        if (!chosen) {                      // pruned: never the winner (the same value from every chunk)
            if (pmode == 0) {
                out_score[ci] = INFINITY;
                out_feas[ci] = 0;
            }
        } else if (np == 1) {               // the whole candidate lies in this chunk
            if (obj1) {
                direct = true;
            } else {
                out_score[ci] = dl;
                out_feas[ci] = (ml <= margin);
            }
        } else {
            X.partial[g + ci] = make_double2(dl, ml);
            __threadfence();
            fin = atomicAdd(X.arrive + ci, 1) == np - 1;
        }
    }
    // the warp that stored a candidate's last piece sums all its pieces: lane j
    // takes pieces j, j + 32, ...; then a fixed butterfly
    unsigned finm = __ballot_sync(0xffffffffu, fin);
    if (finm) __threadfence();
    while (finm) {
        const int src = __ffs(finm) - 1;
        finm &= finm - 1;
        const int fci = __shfl_sync(0xffffffffu, ci, src), ff = __shfl_sync(0xffffffffu, first, src);
        const int fnp = __shfl_sync(0xffffffffu, np, src);
        double sum = 0.0, mx = 0.0;
        for (int j = lane; j < fnp; j += 32) {
            const double2 pj = ldz(X.partial + ff + fci + j);
            sum += pj.x;
            mx = fmax(mx, pj.y);
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o2);
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o2));
        }
        if (obj1) {
            const int js = __shfl_sync(0xffffffffu, cd.js, src), nsr = __shfl_sync(0xffffffffu, cd.ns, src);
            const int jr = __shfl_sync(0xffffffffu, cd.jr, src), nr = __shfl_sync(0xffffffffu, cd.nr, src);
            const int fx = __shfl_sync(0xffffffffu, cd.fixed, src), s = __shfl_sync(0xffffffffu, cd.s, src);
            const int jf = fx ? ldi(S.sn_rank + s) : -1;
            sum = fmax(mx, unaffected_max(X, nsn, js, nsr, jr, nr, jf));
        }
        if (lane == 0) {
            out_score[fci] = sum;
            out_feas[fci] = (mx <= margin);
            X.arrive[fci] = 0;
        }
    }
    // objective 1, single-chunk candidates: largest error over the whole network
    unsigned dm = __ballot_sync(0xffffffffu, direct);
    while (dm) {
        const int src = __ffs(dm) - 1;
        dm &= dm - 1;
        const int fci = __shfl_sync(0xffffffffu, ci, src);
        const double fml = __shfl_sync(0xffffffffu, ml, src);
        const int js = __shfl_sync(0xffffffffu, cd.js, src), nsr = __shfl_sync(0xffffffffu, cd.ns, src);
        const int jr = __shfl_sync(0xffffffffu, cd.jr, src), nr = __shfl_sync(0xffffffffu, cd.nr, src);
        const int fx = __shfl_sync(0xffffffffu, cd.fixed, src), s = __shfl_sync(0xffffffffu, cd.s, src);
        const int jf = fx ? ldi(S.sn_rank + s) : -1;
        const double u = unaffected_max(X, nsn, js, nsr, jr, nr, jf);
        if (lane == 0) {
            out_score[fci] = fmax(fml, u);
            out_feas[fci] = (fml <= margin);
        }
    }
}

// FP32 screen of a chunk (precision 1).  Pieces hold (D32, bound, max MICE,
// bound of the max); the final bound adds 32u sum |piece| for the rounding of
// the FP32 sums.
// Objective 1 in the screen: the absolute score max(largest new MICE, largest
// unaffected MICE) as an interval [hi - y, hi + y] that contains
// [max(ml - bml, U), max(ml + bml, U)] (U exact, rounded outward to FP32).
__device__ __forceinline__ float4 obj1_screen(float ml, float bml, double U) {
    const float ulo = __double2float_rd(U), uhi = __double2float_ru(U);
    const float lo = fmaxf(__fsub_rd(ml, bml), ulo), hi = fmaxf(__fadd_ru(ml, bml), uhi);
    return make_float4(hi, __fsub_ru(hi, lo), ml, bml);
}

__device__ void score32_chunk(const Topo &T, const State &S, const Search &X, int n, int L, int SP, int g,
                              bool active, int ci, const Cand &cd, int q, int first, int np, const int *list,
                              bool prof, double &flops, bool obj1 = false, int nsn = 0, unsigned theta = ~0u) {
    // one lane per phase (SP == 4), the scenarios in turn inside the lane
    const int lane = threadIdx.x & 31, p = lane & 3;
    const bool chosen = !active || slot_selected(X, cd, theta);    // learned pruning
    int k = cd.r;
    bool sside = false;
    if (active && chosen) k = position_bus(list, cd, q, sside);
    const bool valid = active && chosen && k != cd.r;
    const int kk = k < 0 ? cd.s : k;
    const unsigned phr = active ? T.ph[cd.r] : 0u;
    float fl = 0.0f;
    float dl = 0.0f, bl = 0.0f, ad = 0.0f, ml = 0.0f, bml = 0.0f;
    for (int l = 0; l < L; ++l) {
        Item32 o;
        o.e = 0.0f;
        o.b = 0.0f;
        if (valid && p < 3) {
            float2 Ir[3];
            for (int qq = 0; qq < 3; ++qq) Ir[qq] = ldf2(S.icur32 + sidx(l, qq, cd.r, n));
            o = eval_item32(T, S, n, cd, k, sside, l, p, Ir, phr, fl);
        }
        float m = o.e, bm = o.b;
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
        bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, 1));
        bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, 2));
        if (valid && p == 0) {
            const float mo = ldf(S.mice32 + (size_t)l * n + kk);
            const float mr = (kk == cd.s) ? ldf(S.mice32 + (size_t)l * n + cd.r) : 0.0f;
            const float d = (m - mo) - mr;
            dl += d;
            bl += bm + 2.0f * kU * (fabsf(mo) + fabsf(mr) + fabsf(m));
            ad += fabsf(d);
            ml = fmaxf(ml, m);
            bml = fmaxf(bml, bm);
        }
    }
    if (prof) flops += fl;
    if (p != 0) { dl = bl = ad = ml = bml = 0.0f; }
    unsigned heads;
    int seg_start;
    bool last;
    seg_scan_setup(active, ci, lane, heads, seg_start, last);
    for (int o2 = 1; o2 < 32; o2 <<= 1) {
        const float y1 = __shfl_up_sync(0xffffffffu, dl, o2);
        const float y2 = __shfl_up_sync(0xffffffffu, bl, o2);
        const float y3 = __shfl_up_sync(0xffffffffu, ad, o2);
        const float y4 = __shfl_up_sync(0xffffffffu, ml, o2);
        const float y5 = __shfl_up_sync(0xffffffffu, bml, o2);
        if (lane - o2 >= seg_start) { dl += y1; bl += y2; ad += y3; ml = fmaxf(ml, y4); bml = fmaxf(bml, y5); }
    }
    float4 *pf = reinterpret_cast<float4 *>(X.partial);
    bool fin = false, direct = false;
    if (active && last) {
        const float pb = bl + 32.0f * kU * ad;
        if (!chosen) {                      // pruned: surely infeasible for the selection
            X.scr[ci] = make_float4(0.0f, 0.0f, INFINITY, 0.0f);
        } else if (np == 1) {               // the whole candidate lies in this chunk
            if (obj1) direct = true;
            else X.scr[ci] = make_float4(dl, 1.001f * (pb + 38.0f * kU * fabsf(dl)), ml, bml);
        } else {
            pf[g + ci] = make_float4(dl, pb, ml, bml);
            __threadfence();
            fin = atomicAdd(X.arrive + ci, 1) == np - 1;
        }
    }
    unsigned finm = __ballot_sync(0xffffffffu, fin);
    if (finm) __threadfence();
    while (finm) {
        const int src = __ffs(finm) - 1;
        finm &= finm - 1;
        const int fci = __shfl_sync(0xffffffffu, ci, src), ff = __shfl_sync(0xffffffffu, first, src);
        const int fnp = __shfl_sync(0xffffffffu, np, src);
        float sum = 0.0f, bsum = 0.0f, asum = 0.0f, mx = 0.0f, bmx = 0.0f;
        for (int j = lane; j < fnp; j += 32) {
            const float4 pj = __ldcg(pf + ff + fci + j);
            sum += pj.x;
            bsum += pj.y;
            asum += fabsf(pj.x);
            mx = fmaxf(mx, pj.z);
            bmx = fmaxf(bmx, pj.w);
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o2);
            bsum += __shfl_xor_sync(0xffffffffu, bsum, o2);
            asum += __shfl_xor_sync(0xffffffffu, asum, o2);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o2));
            bmx = fmaxf(bmx, __shfl_xor_sync(0xffffffffu, bmx, o2));
        }
        double U = 0.0;
        if (obj1) {
            const int js = __shfl_sync(0xffffffffu, cd.js, src), nsr = __shfl_sync(0xffffffffu, cd.ns, src);
            const int jr = __shfl_sync(0xffffffffu, cd.jr, src), nr = __shfl_sync(0xffffffffu, cd.nr, src);
            const int fx = __shfl_sync(0xffffffffu, cd.fixed, src), s = __shfl_sync(0xffffffffu, cd.s, src);
            U = unaffected_max(X, nsn, js, nsr, jr, nr, fx ? ldi(S.sn_rank + s) : -1);
        }
        if (lane == 0) {
            // rounding of the piece sums: at most ceil(np / 32) + 5 additions deep
            const float depth = (float)((fnp + 31) / 32 + 5);
            X.scr[fci] = obj1 ? obj1_screen(mx, bmx, U)
                              : make_float4(sum, 1.001f * (bsum + (depth + 32.0f) * kU * asum), mx, bmx);
            X.arrive[fci] = 0;
        }
    }
    // objective 1, single-chunk candidates
    unsigned dm = __ballot_sync(0xffffffffu, direct);
    while (dm) {
        const int src = __ffs(dm) - 1;
        dm &= dm - 1;
        const int fci = __shfl_sync(0xffffffffu, ci, src);
        const float fml = __shfl_sync(0xffffffffu, ml, src), fbml = __shfl_sync(0xffffffffu, bml, src);
        const int js = __shfl_sync(0xffffffffu, cd.js, src), nsr = __shfl_sync(0xffffffffu, cd.ns, src);
        const int jr = __shfl_sync(0xffffffffu, cd.jr, src), nr = __shfl_sync(0xffffffffu, cd.nr, src);
        const int fx = __shfl_sync(0xffffffffu, cd.fixed, src), s = __shfl_sync(0xffffffffu, cd.s, src);
        const double U = unaffected_max(X, nsn, js, nsr, jr, nr, fx ? ldi(S.sn_rank + s) : -1);
        if (lane == 0) X.scr[fci] = obj1_screen(fml, fbml, U);
    }
}

// ---------------------------------------------------------------- selection
// Doubles compared through order-preserving 64-bit keys, so that the minimum,
// band and gap searches run on the integer pipe (FP64 comparisons issue on the
// slow FP64 pipe of this GPU).
__device__ __forceinline__ unsigned long long dkey(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dval(unsigned long long k) {
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}
struct MinF { __device__ float operator()(float a, float b) const { return fminf(a, b); } };
struct MaxU { __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a > b ? a : b; } };
struct SumLL { __device__ long long operator()(long long a, long long b) const { return a + b; } };

// Exact selection over m entries with FP64 scores (entry i is candidate
// map ? map[i] : i): minimum over feasible entries, tie band [min, min + tau],
// smallest (r, s) inside it.  Identical in every CTA.
struct Sel {
    int w;          // winning candidate (-1: nothing feasible)
    double gap;     // distance of the next score above the tie band
};

__device__ Sel select_exact(const Search &X, int m, const int *map, const double *score, const int *feas, double tau,
                            double *smd, unsigned long long *smu, int *smi, unsigned long long ksure, int nc);

constexpr int kRmax = 1024;     // candidates an FP64 recheck can hold in shared memory

// Screen selection (precision 1), in FP32 with directed rounding so that every
// test holds for the real intervals [D32 - B, D32 + B] and [M32 - Bm, M32 + Bm]
// that contain each candidate's FP64 score and largest MICE.  With
//   m_lo = min over maybe-feasible lower ends, m_hi = min over surely feasible
//   upper ends (the FP64 minimum m lies in [m_lo, m_hi]),
// a candidate is surely in the FP64 tie band when it is surely feasible and its
// upper end is <= m_lo + tau, surely out when it may be infeasible only by
// margin or its lower end is > m_hi + tau, and uncertain otherwise.  The winner
// is the smallest key of the band.  If no uncertain candidate has a key below the
// smallest surely-in key, that candidate wins.  Otherwise R = (candidates whose
// lower end is <= m_hi: they may hold the minimum) + (uncertain candidates with
// a smaller key) is rescored in FP64; the winner is then the smallest key among
// the surely-in candidates and the members of R inside the exact band.
__device__ __forceinline__ bool surely_feasible(float4 q, float margin_lo) { return __fadd_ru(q.z, q.w) <= margin_lo; }

struct Screen {
    int nR;                     // size of R (0 when no recheck is needed)
    int win;                    // winner when no recheck is needed (-1 otherwise / none)
    unsigned long long ksure;   // smallest surely-in key (~0 if none)
    bool any;                   // some candidate may be feasible
    double gap;                 // screen distance from the band edge to the next candidate
};

// Block-wide minima of two floats with one pair of barriers.
__device__ __forceinline__ void block_min2f(float &a, float &b) {
    __shared__ float2 sm[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fminf(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    __syncthreads();
    if (lane == 0) sm[wid] = make_float2(a, b);
    __syncthreads();
    a = sm[0].x;
    b = sm[0].y;
    for (int w = 1; w < nw; ++w) {
        a = fminf(a, sm[w].x);
        b = fminf(b, sm[w].y);
    }
}

// Block-wide minima of two 64-bit keys and a float with one pair of barriers.
__device__ __forceinline__ void block_min_uuf(unsigned long long &a, unsigned long long &b, float &c) {
    struct R3 {
        unsigned long long a, b;
        float c;
    };
    __shared__ R3 sm[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        a = min(a, (unsigned long long)__shfl_xor_sync(0xffffffffu, a, o));
        b = min(b, (unsigned long long)__shfl_xor_sync(0xffffffffu, b, o));
        c = fminf(c, __shfl_xor_sync(0xffffffffu, c, o));
    }
    __syncthreads();
    if (lane == 0) sm[wid] = R3{a, b, c};
    __syncthreads();
    a = sm[0].a;
    b = sm[0].b;
    c = sm[0].c;
    for (int w = 1; w < nw; ++w) {
        a = min(a, sm[w].a);
        b = min(b, sm[w].b);
        c = fminf(c, sm[w].c);
    }
}

__device__ Sel select_exact(const Search &X, int m, const int *map, const double *score, const int *feas, double tau,
                            double *smd, unsigned long long *smu, int *smi, unsigned long long ksure, int nc) {
    const int tid = threadIdx.x;
    unsigned long long bk = ~0ull;
    for (int i = tid; i < m; i += kThreads)
        if (ldi(feas + i)) bk = min(bk, dkey(ldd(score + i)));
    bk = block_reduce(bk, MinU(), smu);
    Sel out;
    out.w = -1;
    out.gap = INFINITY;
    if (bk == ~0ull || dval(bk) == INFINITY) return out;
    const double edge = dval(bk) + tau;
    const unsigned long long ek = dkey(edge);
    // one pass: the band's smallest key packed with its index, and the
    // smallest score above the band
    unsigned long long kp = ~0ull, gk = ~0ull;
    float unused = INFINITY;
    for (int i = tid; i < m; i += kThreads) {
        if (!ldi(feas + i)) continue;
        const unsigned long long k = dkey(ldd(score + i));
        if (k <= ek) {
            const unsigned long long t = __ldcg(X.ckey + (map ? map[i] : i));
            kp = min(kp, (t << 32) | (unsigned)i);
        } else if (k < gk) {
            gk = k;
        }
    }
    block_min_uuf(kp, gk, unused);
    const unsigned long long key = (kp == ~0ull) ? ~0ull : (kp >> 32);
    if (ksure < key) {              // a candidate known to be in the band has the smallest key
        int w = 0x7fffffff;
        for (int c = tid; c < nc; c += kThreads)
            if (__ldcg(X.ckey + c) == ksure) w = min(w, c);
        w = block_reduce(w, MinI(), smi);
        out.w = (w < nc) ? w : -2;
    } else if (kp == ~0ull) {
        out.w = -2;
    } else {
        const int w = (int)(kp & 0xffffffffu);
        out.w = map ? map[w] : w;
    }
    out.gap = (gk == ~0ull) ? INFINITY : dval(gk) - edge;
    return out;
}

__device__ Screen screen_select(const Search &X, int nc, double margin, double tau, int *s_R, int2 *sm2, float *smf,
                                unsigned long long *smu, int *smi) {
    const int tid = threadIdx.x;
    const float margin_lo = __double2float_rd(margin), margin_hi = __double2float_ru(margin);
    const float tau_lo = __double2float_rd(tau), tau_hi = __double2float_ru(tau);
    float mhi = INFINITY, mlo = INFINITY;
    for (int c = tid; c < nc; c += kThreads) {
        const float4 q = __ldcg(X.scr + c);
        if (__fsub_rd(q.z, q.w) <= margin_hi) mlo = fminf(mlo, __fsub_rd(q.x, q.y));
        if (surely_feasible(q, margin_lo)) mhi = fminf(mhi, __fadd_ru(q.x, q.y));
    }
    block_min2f(mlo, mhi);
    Screen out;
    out.nR = 0;
    out.win = -1;
    out.ksure = ~0ull;
    out.any = mlo < INFINITY;
    out.gap = INFINITY;
    if (!out.any) return out;
    const float edge_in = __fadd_rd(mlo, tau_lo), edge_out = __fadd_ru(mhi, tau_hi);
    // one pass: the smallest surely-in key (packed with its candidate index), the
    // smallest key of an uncertain candidate, and the gap above the band
    unsigned long long kp = ~0ull, ku = ~0ull;
    float g = INFINITY;
    for (int c = tid; c < nc; c += kThreads) {
        const float4 q = __ldcg(X.scr + c);
        const bool maybe = __fsub_rd(q.z, q.w) <= margin_hi;
        if (!maybe) continue;
        const float lo = __fsub_rd(q.x, q.y), hi = __fadd_ru(q.x, q.y);
        const bool in_sure = surely_feasible(q, margin_lo) && hi <= edge_in;
        const bool out_sure = lo > edge_out;
        const unsigned long long key = __ldcg(X.ckey + c);
        if (in_sure) kp = min(kp, (key << 32) | (unsigned)c);
        else if (!out_sure) ku = min(ku, key);
        if (out_sure) g = fminf(g, lo - edge_out);
    }
    block_min_uuf(kp, ku, g);
    const unsigned long long ks = (kp == ~0ull) ? ~0ull : (kp >> 32);
    out.ksure = ks;
    out.gap = (double)g;
    if (!(ku < ks)) {                   // no uncertain candidate can take the band's smallest key
        out.win = (kp == ~0ull) ? -2 : (int)(kp & 0xffffffffu);
        return out;
    }
    // R: possible minimizers and uncertain candidates with a key below ks
    int nR = 0;
    for (int c0 = 0; c0 < nc; c0 += kThreads) {
        const int c = c0 + tid;
        int flag = 0;
        if (c < nc) {
            const float4 q = __ldcg(X.scr + c);
            if (__fsub_rd(q.z, q.w) <= margin_hi) {
                const float lo = __fsub_rd(q.x, q.y), hi = __fadd_ru(q.x, q.y);
                const bool in_sure = surely_feasible(q, margin_lo) && hi <= edge_in;
                const bool out_sure = lo > edge_out;
                const bool unc = !in_sure && !out_sure && __ldcg(X.ckey + c) < ks;
                if (unc || lo <= mhi) flag = 1;
            }
        }
        int2 tot;
        const int2 ex = block_scan2(make_int2(flag, 0), sm2, &tot);
        if (flag && nR + ex.x < kRmax) s_R[nR + ex.x] = c;
        nR += tot.x;
    }
    out.nR = nR;
    __syncthreads();
    return out;
}

// ---------------------------------------------------------------- scorer features
// Local features of candidate (s, r) on the current state, for the learned
// scorer: how far r's injection moves (path impedance between r and the
// common ancestor, and between s and it), how much is moved (injections of r
// and s), phase counts, the current MICE and voltage spread of both clusters
// relative to the margin, the direction, the number of affected clusters and
// the merged cluster's error at s's present voltage magnitude.  The whole
// warp computes them (every lane must call this): the loads are spread over
// the lanes, reduced by shuffles, and lane i < kScorerFeatures writes f[i].
__device__ void cand_features_warp(const Topo &T, const State &S, int n, int L, const Cand &c, double margin,
                                   float *f) {
    const int lane = threadIdx.x & 31;
    auto wsum = [](double v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    auto wmax = [](double v) {                 // (every value is >= 0)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    };
    const unsigned phs = T.ph[c.s], phr = T.ph[c.r];
    // path impedances to the common ancestor: r on lanes 0-8, s on lanes 9-17
    double zr = 0.0, zs = 0.0;
    if (lane < 18) {
        const int u = lane < 9 ? c.r : c.s, q = lane < 9 ? lane : lane - 9;
        const double2 d = csub(ldz(T.zc + (size_t)u * 9 + q), ldz(T.zc + (size_t)c.a * 9 + q));
        (lane < 9 ? zr : zs) = fabs(d.x) + fabs(d.y);
    }
    // per (scenario, phase) on lanes 0 .. 3L-1: injections, spreads, the merged error
    double ir = 0.0, is = 0.0, spr = 0.0, sps = 0.0, em = 0.0;
    if (lane < 3 * L) {
        const int l = lane / 3, p = lane % 3;
        const double2 a = ldz(S.icur + sidx(l, p, c.r, n)), b = ldz(S.icur + sidx(l, p, c.s, n));
        ir = fabs(a.x) + fabs(a.y);
        is = fabs(b.x) + fabs(b.y);
        const size_t kr = sidx(l, p, c.r, n), ks = sidx(l, p, c.s, n);
        if (phr >> p & 1u) spr = ldd(S.hi + kr) - ldd(S.lo + kr);
        if (phs >> p & 1u) {
            const double hs = ldd(S.hi + ks), lo = ldd(S.lo + ks), ms = ldd(S.mcur + ks);
            sps = hs - lo;
            em = fmax(hs - ms, ms - lo);
            if (phr >> p & 1u) em = fmax(em, fmax(ldd(S.hi + kr) - ms, ms - ldd(S.lo + kr)));
        }
    }
    // MICE per scenario: r on lanes 0 .. L-1, s on lanes 8 .. 8+L-1
    double mr = 0.0, msx = 0.0;
    if (lane < L) mr = ldd(S.mice + (size_t)lane * n + c.r);
    if (lane >= 8 && lane < 8 + L) msx = ldd(S.mice + (size_t)(lane - 8) * n + c.s);
    zr = wsum(zr);
    zs = wsum(zs);
    ir = wsum(ir);
    is = wsum(is);
    spr = wmax(spr);
    sps = wmax(sps);
    em = wmax(em);
    mr = wmax(mr);
    msx = wmax(msx);
    if (lane >= kScorerFeatures) return;
    float v = 0.0f;
    switch (lane) {
        case 0: v = (float)log10(1e-9 + zr); break;
        case 1: v = (float)log10(1e-9 + zs); break;
        case 2: v = (float)log10(1e-9 + ir); break;
        case 3: v = (float)log10(1e-9 + is); break;
        case 4: v = (float)__popc(phr) / 3.0f; break;
        case 5: v = (float)__popc(phs) / 3.0f; break;
        case 6: v = (float)(mr / margin); break;
        case 7: v = (float)(msx / margin); break;
        case 8: v = (float)c.dir; break;
        case 9: v = (float)log10(1.0 + c.ns + c.nr); break;
        case 10: v = (float)(spr / margin); break;
        case 11: v = (float)(sps / margin); break;
        case 12: v = (float)(em / margin); break;
        default: v = (float)((em - mr - msx) / margin); break;
    }
    f[lane] = v;
}

// ---------------------------------------------------------------- the kernel
// One feeder's search on a team of G CTAs (rank = this CTA's index in the team).
template <int PREC>
__device__ __forceinline__ void search_run(const Topo &T, const State &S, const Search &X, Ctrl *C, GridBar *gb,
                                           int rank, unsigned G, unsigned &epoch) {
    __shared__ double smd[32];
    __shared__ float smf[32];
    __shared__ unsigned long long smu[32];
    __shared__ int smi[32];
    __shared__ int2 sm2[33];
    __shared__ int2 s_pref, s_tot, s_mine;
    __shared__ int s_R[kRmax];
    __shared__ int s_Rbase[kRmax + 1];
    const int n = T.n, L = T.L;
    const int Lp = L <= 1 ? 1 : (L <= 2 ? 2 : 4);
    const int SPC = 4 * Lp;                    // lanes per position of the merge's items
    constexpr int SP = 4, PPW = 8;             // sweeps: one lane per phase, 8 positions per warp
    constexpr int nt = kThreads;           // every search kernel runs 512-thread CTAs
    const int tid = threadIdx.x, lane = tid & 31;
    const int gt = rank * nt + tid, gs = (int)G * nt;
    const int warp = gt >> 5, nwarps = gs >> 5;
    const double margin = C->margin, tau = C->tau;
    const int max_merges = C->max_merges;
    const bool prof = C->profile != 0;
    const bool obj1 = C->objective == 1;
    const bool lead = (rank == 0 && tid == 0);
    int t = C->t, ns = C->n_super;
    double s_cur = C->s_cur;               // SMICE of the committed state
    bool have = false;                     // a sweep's scores wait for selection
    int nc = 0, P = 0, nchunks = 0;        // current candidate list
    int2 my_ex = make_int2(0, 0);          // this thread's offsets inside its CTA
    double flops = 0.0;
    int nw_commit = 0;                     // warps that held items of the last commit
    unsigned theta = ~0u;                  // learned pruning: key of the k-th best prediction (~0: none)
    if (t >= max_merges || C->done) return;
    extern __shared__ unsigned char dyn_smem[];
    MlpSmem *MW = X.topk > 0 ? reinterpret_cast<MlpSmem *>(dyn_smem) : nullptr;
    if (MW) {
        mlp_load_smem(X, MW);
        __syncthreads();
    }

    for (;;) {
        // ============================================================ phase 1
        s_cur = ldd(&C->s_cur);                // updated by one thread in the last phase 2
        unsigned long long tp = (prof && lead) ? gtimer() : 0;
        auto stamp = [&](int i) {
            if (prof && lead) { const unsigned long long now = gtimer(); C->phase_ns[i] += now - tp; tp = now; }
        };
        const int told = t;
        const int *list_old = S.sn_list[told & 1];
        bool committed = false, finishing = false;
        int r0 = -1, s0 = -1, dir0 = 0, jr0 = 0;
        if (have) {
            Sel sel;
            bool full64 = (PREC == 0);
            if (PREC == 1) {
                const Screen sc = screen_select(X, nc, margin, tau, s_R, sm2, smf, smu, smi);
                const int nR = sc.nR;
                stamp(0);
                if (rank == 0 && t < X.rec_iters) {
                    for (int c = tid >> 5; c < nc; c += nt >> 5) {        // one warp per candidate
                        const Cand cc = ldcand(X.cand + c);
                        if (lane == 0) {
                            const float4 q = __ldcg(X.scr + c);
                            const bool out = __fsub_rd(q.z, q.w) > __double2float_ru(margin);
                            X.rec_s[(size_t)t * 2 * n + c] = T.orig[cc.s];
                            X.rec_r[(size_t)t * 2 * n + c] = T.orig[cc.r];
                            X.rec_score[(size_t)t * 2 * n + c] = out ? INFINITY : (obj1 ? 0.0 : s_cur) + (double)q.x;
                            X.rec_bound[(size_t)t * 2 * n + c] = out ? 0.0 : (double)q.y;
                        }
                        cand_features_warp(T, S, n, L, cc, margin, X.rec_feat + ((size_t)t * 2 * n + c) * kScorerFeatures);
                    }
                }
                if (!sc.any) {
                    sel.w = -1;
                } else if (nR == 0) {
                    sel.w = sc.win;
                    sel.gap = sc.gap;
                } else if (nR <= kRmax) {
                    // FP64 recheck of R: positions of R back to back
                    for (int i0 = 0; i0 < nR; i0 += nt) {
                        const int i = i0 + tid;
                        const int cnt = i < nR ? cand_positions(ldcand(X.cand + s_R[i])) : 0;
                        int2 tot;
                        const int2 ex = block_scan2(make_int2(cnt, 0), sm2, &tot);
                        const int off = (i0 == 0) ? 0 : s_Rbase[i0];
                        __syncthreads();
                        if (i < nR) s_Rbase[i] = off + ex.x;
                        if (tid == 0) s_Rbase[min(i0 + nt, nR)] = off + tot.x;
                        __syncthreads();
                    }
                    const int PR = s_Rbase[nR];
                    const int rchunks = (PR + PPW - 1) / PPW;
                    const int *list = S.sn_list[t & 1];
                    for (int g = warp; g < rchunks; g += nwarps) {
                        const int q = g * PPW + lane / SP;
                        const bool active = q < PR;
                        int lo = 0, hi = nR - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (s_Rbase[mid] <= q) lo = mid;
                            else hi = mid - 1;
                        }
                        const Cand cd = ldcand(X.cand + s_R[lo]);
                        const int b0 = s_Rbase[lo], cnt = s_Rbase[lo + 1] - b0;
                        const int first = b0 / PPW, np = (b0 + cnt - 1) / PPW - first + 1;
                        score64_chunk(T, S, X, n, L, SP, g, active, lo, cd, q - b0, first, np, list, margin,
                                      X.score, X.feas, false, flops, obj1, ns);
                    }
                    if (lead) { C->rechecks += 1; C->recheck_cands += nR; }
                    if (!team_barrier(gb, C, G, epoch)) return;
                    sel = select_exact(X, nR, s_R, X.score, X.feas, tau, smd, smu, smi, sc.ksure, nc);
                    stamp(1);
                } else {
                    full64 = true;                      // R too large: rescore everything in FP64
                    if (lead) { C->rechecks += 1; C->recheck_cands += nc; }
                }
                if (full64) {
                    const int *list = S.sn_list[t & 1];
                    for (int g = warp; g < nchunks; g += nwarps) {
                        const int c0 = ldi(X.chunk_first + g);
                        const int q = g * PPW + lane / SP;
                        const int cb = (c0 + lane <= nc) ? ldi(X.base + c0 + lane) : 0x7fffffff;    // base[nc] = P
                        const int off = chunk_offset(cb, g * PPW, PPW, lane / SP);
                        const int cbase = __shfl_sync(0xffffffffu, cb, off);
                        const int c = c0 + off;
                        const bool active = q < P;
                        Cand cd;
                        cd.r = -1;
                        int first = 0, np = 1;
                        if (active) {
                            cd = ldcand(X.cand + c);
                            first = cbase / PPW;
                            np = (cbase + cand_positions(cd) - 1) / PPW - first + 1;
                        }
                        score64_chunk(T, S, X, n, L, SP, g, active, c, cd, q - cbase, first, np, list, margin,
                                      X.score, X.feas, false, flops, obj1, ns, theta);
                    }
                    if (!team_barrier(gb, C, G, epoch)) return;
                }
            }
            if (full64) {
                if (PREC == 0 && rank == 0 && t < X.rec_iters) {
                    for (int c = tid >> 5; c < nc; c += nt >> 5) {        // one warp per candidate
                        const Cand cc = ldcand(X.cand + c);
                        if (lane == 0) {
                            X.rec_s[(size_t)t * 2 * n + c] = T.orig[cc.s];
                            X.rec_r[(size_t)t * 2 * n + c] = T.orig[cc.r];
                            X.rec_score[(size_t)t * 2 * n + c] =
                                ldi(X.feas + c) ? (obj1 ? 0.0 : s_cur) + ldd(X.score + c) : INFINITY;
                            X.rec_bound[(size_t)t * 2 * n + c] = 0.0;
                        }
                        cand_features_warp(T, S, n, L, cc, margin, X.rec_feat + ((size_t)t * 2 * n + c) * kScorerFeatures);
                    }
                }
                sel = select_exact(X, nc, nullptr, X.score, X.feas, tau, smd, smu, smi, ~0ull, nc);
                stamp(PREC == 0 ? 0 : 1);
            }
            if (theta != ~0u && X.prune_exact) {
                // certified pruning, second pass: every candidate the learned
                // ordering left out is scored too, unless its lower bound on the
                // score change exceeds the first pass's best feasible score plus
                // the tie band (1e-12 covers the rounding of the FP64 scores)
                const double thr = sel.w >= 0 ? __dadd_ru(__dadd_ru(ldd(X.score + sel.w), tau), 1e-12) : INFINITY;
                int excl = 0;
                const int *list = S.sn_list[t & 1];
                for (int g = warp; g < nchunks; g += nwarps) {
                    const int c0 = ldi(X.chunk_first + g);
                    const int q = g * PPW + lane / SP;
                    const int cb = (c0 + lane <= nc) ? ldi(X.base + c0 + lane) : 0x7fffffff;    // base[nc] = P
                    const int off = chunk_offset(cb, g * PPW, PPW, lane / SP);
                    const int cbase = __shfl_sync(0xffffffffu, cb, off);
                    const int c = c0 + off;
                    const bool active = q < P;
                    Cand cd;
                    cd.r = -1;
                    int first = 0, np = 1;
                    if (active) {
                        cd = ldcand(X.cand + c);
                        first = cbase / PPW;
                        np = (cbase + cand_positions(cd) - 1) / PPW - first + 1;
                    }
                    score64_chunk(T, S, X, n, L, SP, g, active, c, cd, q - cbase, first, np, list, margin, X.score,
                                  X.feas, false, flops, obj1, ns, theta, 1, thr, &excl);
                }
                for (int o2 = 16; o2 > 0; o2 >>= 1) excl += __shfl_xor_sync(0xffffffffu, excl, o2);
                if (lane == 0 && excl) atomicAdd(reinterpret_cast<unsigned long long *>(&C->pruned), (unsigned long long)excl);
                if (!team_barrier(gb, C, G, epoch)) return;
                sel = select_exact(X, nc, nullptr, X.score, X.feas, tau, smd, smu, smi, ~0ull, nc);
            }
            if (theta != ~0u && sel.w < 0 && !X.prune_exact) {
                // learned pruning left no feasible candidate: evaluate them all in FP64
                const int *list = S.sn_list[t & 1];
                for (int g = warp; g < nchunks; g += nwarps) {
                    const int c0 = ldi(X.chunk_first + g);
                    const int q = g * PPW + lane / SP;
                    const int cb = (c0 + lane <= nc) ? ldi(X.base + c0 + lane) : 0x7fffffff;    // base[nc] = P
                    const int off = chunk_offset(cb, g * PPW, PPW, lane / SP);
                    const int cbase = __shfl_sync(0xffffffffu, cb, off);
                    const int c = c0 + off;
                    const bool active = q < P;
                    Cand cd;
                    cd.r = -1;
                    int first = 0, np = 1;
                    if (active) {
                        cd = ldcand(X.cand + c);
                        first = cbase / PPW;
                        np = (cbase + cand_positions(cd) - 1) / PPW - first + 1;
                    }
                    score64_chunk(T, S, X, n, L, SP, g, active, c, cd, q - cbase, first, np, list, margin, X.score,
                                  X.feas, false, flops, obj1, ns, ~0u);
                }
                if (!team_barrier(gb, C, G, epoch)) return;
                sel = select_exact(X, nc, nullptr, X.score, X.feas, tau, smd, smu, smi, ~0ull, nc);
                if (lead) C->scorer_fallbacks += 1;
            }
            if (lead && t < X.rec_iters) X.rec_count[t] = nc;
            if (sel.w == -2) {                          // unreachable: the minimum lies in the band
                if (lead) { C->err = 5; C->done = 1; }
                break;
            }
            if (sel.w < 0) {                            // nothing feasible
                if (lead) { C->done = 1; C->stop_reason = 1; C->t = t; C->s_cur = s_cur; C->n_super = ns; }
                break;
            }

            // ---- commit in FP64: r's cluster joins s
            const Cand cd = ldcand(X.cand + sel.w);
            const unsigned phr = T.ph[cd.r];
            // the merge runs on the last warps of the grid, the candidate setup
            // below on the first threads, so that the two overlap
            const int rgt = gs - 1 - gt, cwarp = nwarps - 1 - warp;
            for (int i = rgt; i < n; i += gs)
                if (ldi(S.label + i) == cd.r) S.label[i] = cd.s;
            const int nitems = cand_positions(cd) * SPC;
            double acc = 0.0;
            for (int i0 = cwarp * 32; i0 < nitems; i0 += nwarps * 32) {
                const int item = i0 + lane;
                const int q = item / SPC, sub = item % SPC, l = sub >> 2, p = sub & 3;
                bool sside = false;
                const int k = item < nitems ? position_bus(list_old, cd, q, sside) : cd.r;
                const bool live = item < nitems && l < L && p < 3 && k != cd.r;
                const int kk = k < 0 ? cd.s : k;
                Item64 o;
                o.e = 0.0;
                o.on = false;
                if (live) {
                    double2 Ir[3];
                    for (int qq = 0; qq < 3; ++qq) Ir[qq] = ldz(S.icur + sidx(l, qq, cd.r, n));
                    o = eval_item64(T, S, n, cd, k, sside, l, p, Ir, phr);
                }
                double m = o.e;
                m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 1));
                m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 2));
                if (live && o.on) {
                    const size_t ik = sidx(l, p, kk, n);
                    double h = ldd(S.hi + ik), lo = ldd(S.lo + ik);
                    if (kk == cd.s) {
                        h = fmax(h, ldd(S.hi + sidx(l, p, cd.r, n)));
                        lo = fmin(lo, ldd(S.lo + sidx(l, p, cd.r, n)));
                        S.hi[ik] = h;
                        S.lo[ik] = lo;
                    }
                    S.vcur[ik] = o.v;
                    S.mcur[ik] = o.m;
                    S.v32[ik] = make_float2((float)o.v.x, (float)o.v.y);
                    S.hr32[ik] = (float)(h - o.m);
                    S.lr32[ik] = (float)(lo - o.m);
                }
                if (live && p == 0 && l == 0 && X.moved) X.moved[kk] = t + 1;   // its inputs change with this merge
                if (live && p == 0) {
                    const double mold = ldd(S.mice + (size_t)l * n + kk);
                    double d = m - mold;
                    if (kk == cd.s) d -= ldd(S.mice + (size_t)l * n + cd.r);
                    acc += d;
                    S.mice[(size_t)l * n + kk] = m;
                    S.mice32[(size_t)l * n + kk] = (float)m;
                }
            }
            for (int o2 = 16; o2 > 0; o2 >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o2);
            nw_commit = min(nwarps, (nitems + 31) / 32);
            if (lane == 0 && cwarp < nw_commit) X.wsum[cwarp] = acc;
            if (rgt == 0) {
                for (int l = 0; l < L; ++l)
                    for (int q = 0; q < 3; ++q)
                        if (phr >> q & 1u) {
                            const size_t is = sidx(l, q, cd.s, n);
                            const double2 ni = cadd(ldz(S.icur + is), ldz(S.icur + sidx(l, q, cd.r, n)));
                            S.icur[is] = ni;
                            S.icur32[is] = make_float2((float)ni.x, (float)ni.y);
                        }
                if (cd.dir == 1) {
                    S.top[cd.s] = ldi(S.top + cd.r);
                    S.ptop[cd.s] = ldi(S.ptop + cd.r);
                }
                if (X.moved) {
                    X.moved[cd.s] = t + 1;
                    X.moved[cd.r] = t + 1;
                }
                X.dec_s[t] = T.orig[cd.s];
                X.dec_r[t] = T.orig[cd.r];
                X.dec_gap[t] = sel.gap;
                X.dec_ncand[t] = nc;
            }
            stamp(2);
            committed = true;
            r0 = cd.r; s0 = cd.s; dir0 = cd.dir;
            jr0 = ldi(S.sn_rank + r0);
            t += 1;
            ns -= 1;
            finishing = (t >= max_merges);
        }

        // ---- candidate setup for the next sweep (reads adjusted for the merge
        // committed above: label r -> s, rank drops past r, s's top)
        if (!finishing) {
            int2 mine = make_int2(0, 0);
            // each thread owns `per` consecutive super-node slots (one on a full grid)
            const int per = (ns + gs - 1) / gs, jb = gt * per, je = min(ns, jb + per);
            for (int j = jb; j < je; ++j) {
            Cand c0, c1;
            c0.s = -1;
            c1.s = -1;
            if (j >= 1) {
                const int w = ldi(list_old + j + (committed && j >= jr0 ? 1 : 0));
                const bool moved = committed && w == s0 && dir0 == 1;     // s took r's top this merge
                const int tw = moved ? ldi(S.top + r0) : ldi(S.top + w);
                const int pw_bus = moved ? ldi(S.ptop + r0) : ldi(S.ptop + w);
                int x = ldi(S.label + pw_bus);
                if (committed && x == r0) x = s0;
                // when x's own bus is the parent of w's top, x is the common ancestor
                // and w's branch starts at its top: no table lookup or search
                const bool direct = (x == pw_bus);
                const int a = direct ? x : (int)T.lca[(size_t)x * n + w];
                const int cw = direct ? tw : child_toward(T, a, w);
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
            X.slot[2 * j] = c0;
            X.slot[2 * j + 1] = c1;
            }
            int2 tot;
            my_ex = block_scan2(mine, sm2, &tot);
            if (tid == 0) { X.block_tot[rank] = tot; s_mine = tot; }
        }
        stamp(3);
        if (!team_barrier(gb, C, G, epoch)) return;
        stamp(4);

        // ============================================================ phase 2
        if (committed) {
            // The merge's bookkeeping runs on the grid's last warps, so that it
            // overlaps the compaction and chunk map on the first CTAs.
            // Exact score change of the merge, in warp order (the last warp);
            // its lane 0 is the only writer of C->s_cur in this phase.
            if (rank == (int)G - 1 && tid >= nt - 32) {
                double d = 0.0;
                for (int w2 = lane; w2 < nw_commit; w2 += 32) d += ldd(X.wsum + w2);
                for (int o2 = 16; o2 > 0; o2 >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o2);
                if (lane == 0) {
                    s_cur += d;
                    if (!obj1) X.dec_score[told] = s_cur;
                    for (int l = 0; l < L; ++l) {
                        S.mice[(size_t)l * n + r0] = 0.0;
                        S.mice32[(size_t)l * n + r0] = 0.0f;
                    }
                    C->t = t;
                    C->s_cur = s_cur;
                    C->n_super = ns;
                }
            }
            stamp(8);
            // super-node list after the merge (other buffer), ranks, largest MICE
            int *list_new = S.sn_list[t & 1];
            unsigned long long m = 0;          // MICE >= 0: bit patterns order like the values
            const int rwarp = nwarps - 1 - warp;
            // CTAs whose (reversed) warps hold no list entry skip the loop and its reduction
            const bool has_list = (nwarps - (rank + 1) * (nt / 32)) * 32 < ns;
            for (int j0 = rwarp * 32; has_list && j0 < ns; j0 += gs) {    // warp-uniform trip count
                const int j = j0 + lane;
                double mr = 0.0;
                long long gk = 0;              // certified pruning: floor(g_k 2^56) of rank j
                if (j < ns) {
                    const int k = ldi(list_old + j + (j >= jr0 ? 1 : 0));
                    list_new[j] = k;
                    for (int l = 0; l < L; ++l) mr = fmax(mr, ldd(S.mice + (size_t)l * n + k));
                    m = max(m, (unsigned long long)__double_as_longlong(mr));
                    if (obj1) X.mrank[j] = mr;
                    if (X.prune_exact) gk = cluster_g_fx(T, S, n, L, k);
                }
                if (X.prune_exact) {                          // prefix within the block of 32 ranks
                    for (int o2 = 1; o2 < 32; o2 <<= 1) {
                        const long long y = __shfl_up_sync(0xffffffffu, gk, o2);
                        if (lane >= o2) gk += y;
                    }
                    if (j < ns) X.gpre[j] = gk;
                    if (lane == 31) X.gblk[j0 >> 5] = gk;
                }
                if (obj1) {                                   // 32 consecutive ranks per warp
                    for (int o2 = 16; o2 > 0; o2 >>= 1) mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o2));
                    if (lane == 0) X.bmax[j0 >> 5] = mr;
                }
            }
            for (int b = r0 + 1 + (gs - 1 - gt); b <= n; b += gs) S.sn_rank[b] = ldi(S.sn_rank + b) - 1;
            if (has_list) {
                m = block_reduce(m, MaxU(), smu);
                if (tid == 0 && m > 0) atomicMax((unsigned long long *)&X.dec_maxerr[told], m);
            }
            stamp(9);
        }
        if (finishing) {
            if (lead) { C->done = 1; C->stop_reason = 0; }
            break;
        }
        if (tid < 32) {
            int2 acc = make_int2(0, 0), all = make_int2(0, 0);
            for (int b = lane; b < (int)G; b += 32) {
                const int2 v = __ldcg(X.block_tot + b);
                if (b < (int)rank) { acc.x += v.x; acc.y += v.y; }
                all.x += v.x;
                all.y += v.y;
            }
            for (int o2 = 16; o2 > 0; o2 >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o2);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o2);
                all.x += __shfl_xor_sync(0xffffffffu, all.x, o2);
                all.y += __shfl_xor_sync(0xffffffffu, all.y, o2);
            }
            if (lane == 0) { s_pref = acc; s_tot = all; }
        }
        __syncthreads();
        stamp(10);
        const int2 pref = s_pref, tot = s_tot;
        nc = tot.x;
        P = tot.y;
        nchunks = (P + PPW - 1) / PPW;
        // (C->s_cur already holds this iteration's value: the merge's sum wrote it)
        if (nc == 0) {                                  // no candidate at all: nothing is feasible
            if (lead) { C->done = 1; C->stop_reason = 1; C->t = t; C->n_super = ns; }
            break;
        }
        if (nchunks > X.max_chunks) {                   // grow the work buffers and relaunch
            if (lead) { C->err = 7; C->total_pos = P; C->t = t; C->n_super = ns; }
            break;
        }
        {
            // this CTA's candidates into the compact list; their first positions
            // also into shared memory for the chunk map below
            int *s_lbase = s_Rbase;
            const bool in_smem = s_mine.x <= kRmax;     // this CTA's candidate bases fit shared memory
            if (gs >= ns) {                             // one slot per thread (a full grid)
                if (gt >= 1 && gt < ns) {
                    int ci = pref.x + my_ex.x, pos = pref.y + my_ex.y, li = my_ex.x;
                    for (int d = 0; d < 2; ++d) {
                        Cand c = X.slot[2 * gt + d];
                        if (c.s < 0) continue;
                        c.pad = 2 * gt + d;                 // the candidate's slot (its prediction)
                        if (X.prune_exact) X.lbp[ci] = cand_lb_part_kept(T, S, X, n, L, c, margin, t);
                        X.cand[ci] = c;
                        X.ckey[ci] = c.key;
                        X.base[ci] = pos;
                        if (in_smem) s_lbase[li] = pos;
                        ++ci;
                        ++li;
                        pos += cand_positions(c);
                    }
                }
            } else {
                const int per = (ns + gs - 1) / gs, jb = max(1, gt * per), je = min(ns, gt * per + per);
                int ci = pref.x + my_ex.x, pos = pref.y + my_ex.y, li = my_ex.x;
                for (int j = jb; j < je; ++j)
                    for (int d = 0; d < 2; ++d) {
                        Cand c = X.slot[2 * j + d];
                        if (c.s < 0) continue;
                        c.pad = 2 * j + d;
                        if (X.prune_exact) X.lbp[ci] = cand_lb_part_kept(T, S, X, n, L, c, margin, t);
                        X.cand[ci] = c;
                        X.ckey[ci] = c.key;
                        X.base[ci] = pos;
                        if (in_smem) s_lbase[li] = pos;
                        ++ci;
                        ++li;
                        pos += cand_positions(c);
                    }
            }
            if (!in_smem) __threadfence();
            __syncthreads();
            stamp(11);
            // chunk map: every chunk that starts inside this CTA's positions gets the
            // candidate holding its first position (binary search in shared memory)
            const int2 mt = s_mine;
            const int p0 = pref.y, p1 = pref.y + mt.y;
            for (int g = (p0 + PPW - 1) / PPW + tid; g * PPW < p1; g += nt) {
                const int q = g * PPW;
                int lo = 0, hi = mt.x - 1;
                if (in_smem) {
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_lbase[mid] <= q) lo = mid;
                        else hi = mid - 1;
                    }
                } else {
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (ldi(X.base + pref.x + mid) <= q) lo = mid;
                        else hi = mid - 1;
                    }
                }
                X.chunk_first[g] = pref.x + lo;
            }
        }
        if (MW) {
            // the scorer's prediction for every candidate slot (slots are readable
            // since barrier 1), warps of the CTAs that compact taking the last slots.
            // Predictions are kept per candidate (by its slot pair's super-node,
            // which, unlike the slot index, does not shift with the ranks) and
            // made again only when the candidate changed (s, r, the common
            // ancestor, the direction or the count of affected clusters) or s or
            // r took part in the last merge: every feature reads only those.
            const int nsl = 2 * ns, wl = tid >> 5;
            const int mw = (warp + nwarps - min(32, nwarps)) % nwarps;
            for (int sl = mw; sl < nsl; sl += nwarps) {
                const Cand c = ldcand(X.slot + sl);
                float y = INFINITY;
                if (c.s >= 0) {
                    const int cs = 2 * (c.dir == 0 ? c.r : c.s) + c.dir;     // the slot pair's super-node
                    const unsigned long long key = pred_key(c, n);
                    if (key != ~0ull && __ldcg(X.pkey + cs) == key && ldi(X.moved + c.s) != t && ldi(X.moved + c.r) != t) {
                        y = __ldcg(X.pcache + cs);                       // (the same for the whole warp)
                    } else {
                        cand_features_warp(T, S, n, L, c, margin, MW->feat[wl]);
                        __syncwarp();
                        y = mlp_predict_warp(MW, MW->feat[wl]);
                        __syncwarp();
                        if (lane == 0) {
                            X.pcache[cs] = y;
                            X.pkey[cs] = key;
                        }
                    }
                }
                if (lane == 0) X.pred[sl] = y;
            }
        }
        if (lead) {
            X.base[nc] = P;
            C->n_cand = nc;
            C->total_pos = P;
            C->candidates += nc;
            C->iters += 1;
        }
        stamp(5);
        if (!team_barrier(gb, C, G, epoch)) return;
        stamp(6);

        // ============================================================ phase 3
        if (X.prune_exact && warp == nwarps - 1) {
            // certified pruning: the blocks' sums of floor(g_k 2^56) into exclusive
            // prefix sums (read by the next phase 1, after this phase's barrier)
            const int nb = (ns + 31) >> 5;
            long long carry = 0;
            for (int b0 = 0; b0 <= nb; b0 += 32) {
                const int b = b0 + lane;
                const long long v = b < nb ? __ldcg(X.gblk + b) : 0;
                long long x = v;
                for (int o2 = 1; o2 < 32; o2 <<= 1) {
                    const long long y = __shfl_up_sync(0xffffffffu, x, o2);
                    if (lane >= o2) x += y;
                }
                if (b <= nb) X.gbp[b] = carry + x - v;
                carry += __shfl_sync(0xffffffffu, x, 31);
            }
        }
        theta = MW ? topk_threshold(X, 2 * ns, X.topk, nc) : ~0u;
        {
            const int *list_new = S.sn_list[t & 1];
            unsigned long long t_start = 0, w_start = 0;
            if (prof && lead) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
            if (prof) w_start = gtimer();
            int my_chunks = 0;
            for (int g = warp; g < nchunks; g += nwarps) {
                ++my_chunks;
                const int c0 = ldi(X.chunk_first + g);
                const int q = g * PPW + lane / SP;
                const int cb = (c0 + lane <= nc) ? ldi(X.base + c0 + lane) : 0x7fffffff;    // base[nc] = P
                const int off = chunk_offset(cb, g * PPW, PPW, lane / SP);
                const int cbase = __shfl_sync(0xffffffffu, cb, off);
                const int c = c0 + off;
                const bool active = q < P;
                Cand cd;
                cd.r = -1;
                int first = 0, np = 1;
                if (active) {
                    cd = ldcand(X.cand + c);
                    first = cbase / PPW;
                    np = (cbase + cand_positions(cd) - 1) / PPW - first + 1;
                }
                if (PREC == 0)
                    score64_chunk(T, S, X, n, L, SP, g, active, c, cd, q - cbase, first, np, list_new, margin,
                                  X.score, X.feas, prof, flops, obj1, ns, theta);
                else
                    score32_chunk(T, S, X, n, L, SP, g, active, c, cd, q - cbase, first, np, list_new, prof, flops,
                                  obj1, ns, theta);
            }
            if (prof && lane == 0 && my_chunks > 0) {      // per-warp sweep time: sum, count, largest
                const unsigned long long d = gtimer() - w_start;
                atomicAdd(&C->phase_ns[12], d);
                atomicAdd(&C->phase_ns[13], 1ull);
                atomicMax(&C->phase_ns[14], d);
                atomicAdd(&C->phase_ns[15], (unsigned long long)my_chunks);
            }
            if (!team_barrier(gb, C, G, epoch)) return;
            if (prof && lead) {
                unsigned long long t_end;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
                C->sweep_ns += t_end - t_start;
            }
            stamp(7);
        }
        have = true;
    }
    if (prof) {
        for (int o2 = 16; o2 > 0; o2 >>= 1) flops += __shfl_xor_sync(0xffffffffu, flops, o2);
        if (lane == 0 && flops > 0.0) atomicAdd(&C->sweep_flops, flops);
    }
}

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) k_search(Topo T, State S, Search X, Ctrl *C, GridBar *gb) {
    unsigned epoch = 0;
    search_run<PREC>(T, S, X, C, gb, blockIdx.x, gridDim.x, epoch);
}

// Many feeders in one launch.  The grid is split into teams of k CTAs; each
// team takes the next feeder from the queue (feeders listed largest first),
// runs that feeder's whole search with team-wide barriers (a plain CTA barrier
// when k = 1), then writes the feeder's assignment in caller numbering.  All
// CTAs are co-resident (cooperative launch), and every wait is bounded.
template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) k_search_batch(const BatchFeeder *fd, const int *order, int nf,
                                                              int *queue, BatchTeam *teams, int k) {
    __shared__ Topo sT;
    __shared__ State sS;
    __shared__ Search sX;
    __shared__ int s_q;
    const int team = blockIdx.x / k, rank = blockIdx.x % k;
    BatchTeam *tm = teams + team;
    unsigned epoch = 0;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) tm->slot = atomicAdd(queue, 1);
        if (!team_barrier(&tm->bar, &tm->ctrl, k, epoch)) return;
        if (threadIdx.x == 0) s_q = *(volatile int *)&tm->slot;
        __syncthreads();
        const int q = s_q;
        if (q >= nf) return;
        const int f = order[q];
        if (threadIdx.x == 0) {
            sT = fd[f].T;
            sS = fd[f].S;
            sX = fd[f].X;
        }
        __syncthreads();
        Ctrl *C = fd[f].C;
        const bool ok = ldi(fd[f].setup_err) == 0;
        if (ok) search_run<PREC>(sT, sS, sX, C, &tm->bar, rank, k, epoch);
        if (!team_barrier(&tm->bar, &tm->ctrl, k, epoch)) return;
        for (int i = rank * kThreads + threadIdx.x; i < sT.n; i += k * kThreads)
            fd[f].super_out[i] = ok ? sT.orig[ldi(sS.label + sT.pre[i])] : -1;
        if (rank == 0 && threadIdx.x == 0) {
            const int t = ok ? ldi(&C->t) : 0;
            *fd[f].max_err = t > 0 ? ldd(sX.dec_maxerr + t - 1) : 0.0;
        }
        if (!team_barrier(&tm->bar, &tm->ctrl, k, epoch)) return;     // the slot is read by all before reuse
    }
}

// Host entry points for the search kernel (kept in this translation unit with
// the template instantiations).
cudaError_t launch_search(int precision, int grid, Topo T, State S, Search X, Ctrl *C, GridBar *gb, cudaStream_t st) {
    void *args[] = {&T, &S, &X, &C, &gb};
    const void *fn = precision == 1 ? (const void *)k_search<1> : (const void *)k_search<0>;
    const size_t smem = X.topk > 0 ? sizeof(MlpSmem) : 0;    // the scorer's weights for learned pruning
    if (smem) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), args, smem, st);
}

int search_blocks_per_sm() {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_search<0>, kThreads, 0) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_search<1>, kThreads, 0) != cudaSuccess) return 0;
    return a < b ? a : b;
}

cudaError_t launch_search_batch(int precision, int team, int grid, const BatchFeeder *fd, const int *order, int nf,
                                int *queue, BatchTeam *teams, cudaStream_t st) {
    void *args[] = {&fd, &order, &nf, &queue, &teams, &team};
    const void *fn = precision == 1 ? (const void *)k_search_batch<1> : (const void *)k_search_batch<0>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), args, 0, st);
}

int search_batch_blocks_per_sm(int precision) {
    int a = 0;
    const void *fn = precision == 1 ? (const void *)k_search_batch<1> : (const void *)k_search_batch<0>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fn, kThreads, 0) != cudaSuccess) return 0;
    return a;
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
