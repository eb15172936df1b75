// okr_search.cu -- one iteration of the exhaustive search (Algorithm 1, Sec. IV)
// as five kernels: candidate setup, chunk scan, candidate sweep, selection,
// commit.
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
// Both sets are contiguous preorder ranges.  Clusters outside them keep their
// voltages and their MICE, so a candidate's SMICE differs from the current one
// by D(c) = sum over affected clusters of (new MICE - current MICE), the merged
// cluster of s and r counted once (post-merge clusters).  Unaffected clusters
// already satisfy the margin, so feasibility is decided on the affected ones.
//
// MICE of a cluster for a candidate voltage m = |V^c_k|: with hi/lo the largest
// and smallest |Vhat| of the members on phase p, max_i | |Vhat_i| - m | =
// max(hi - m, m - lo); the MICE is the largest of these over phases.
#include "okr_internal.cuh"
#include "okr_kernels.cuh"

#include <cfloat>

namespace okr {

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

// New MICE (per scenario) of the cluster of super-node k when its voltage moves
// by G * I_r (G == nullptr: no move).  merged: k == s, the cluster of r joins.
__device__ __forceinline__ void cluster_mice(const Topo &T, const State &S, int n, int L, int k, bool merged,
                                             int r, const double2 *G, const double2 *Ir, unsigned phr,
                                             double *mnew) {
    const unsigned phk = T.ph[k];
    for (int l = 0; l < L; ++l) {
        double m_l = 0.0;
        for (int p = 0; p < 3; ++p) {
            if (!(phk >> p & 1u)) continue;
            double2 v = S.vcur[sidx(l, p, k, n)];
            if (G) {
                double2 dv = make_double2(0.0, 0.0);
                for (int q = 0; q < 3; ++q)
                    if (phr >> q & 1u) dv = cadd(dv, cmul(G[p * 3 + q], Ir[l * 3 + q]));
                v = cadd(v, dv);
            }
            const double mag = cmag(v);
            double h = S.hi[sidx(l, p, k, n)], lo = S.lo[sidx(l, p, k, n)];
            if (merged) {
                h = fmax(h, S.hi[sidx(l, p, r, n)]);
                lo = fmin(lo, S.lo[sidx(l, p, r, n)]);
            }
            m_l = fmax(m_l, fmax(h - mag, mag - lo));
        }
        mnew[l] = m_l;
    }
}

// Path-impedance difference for affected bus k of candidate cd.
__device__ __forceinline__ void delta_z(const Topo &T, int n, const Cand &cd, bool sside, int k, double2 *G) {
    const int y = T.lca[(size_t)(sside ? cd.s : cd.r) * n + k];
    const double2 *zy = T.zc + (size_t)y * 9;
    const double2 *za = T.zc + (size_t)cd.a * 9;
    for (int q = 0; q < 9; ++q) G[q] = sside ? csub(zy[q], za[q]) : csub(za[q], zy[q]);
}

__device__ __forceinline__ void load_ir(const State &S, int n, int L, int r, double2 *Ir) {
    for (int l = 0; l < L; ++l)
        for (int q = 0; q < 3; ++q) Ir[l * 3 + q] = S.icur[sidx(l, q, r, n)];
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------- setup
// One thread per bus w.  For a super-node w other than the slack's cluster, its
// quotient edge goes to x = label[parent[top[w]]]; slot 2w is (s = x, r = w),
// slot 2w+1 is (s = w, r = x).  Phase availability: phi(r) within phi(s); the
// slack is never r.  Also folds the largest MICE of the committed state into the
// previous iteration's record.
__global__ void k_setup(Topo T, State S, Search X, Ctrl *C) {
    const int n = T.n, L = T.L;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    const int t = C->t;
    if (gt == 0) C->commit = 0;
    if (t >= 1) {
        double m = 0.0;
        for (int k = gt; k < n; k += gs)
            if (S.label[k] == k)
                for (int l = 0; l < L; ++l) m = fmax(m, S.mice[(size_t)l * n + k]);
        m = warp_max(m);
        if ((threadIdx.x & 31) == 0 && m > 0.0)
            atomicMax((unsigned long long *)&X.dec_maxerr[t - 1], (unsigned long long)__double_as_longlong(m));
    }
    if (C->done) return;
    for (int w = gt; w < n; w += gs) {
        int nc0 = 0, nc1 = 0;
        if (w > 0 && S.label[w] == w) {
            const int tw = S.top[w];
            const int x = S.label[T.parent[tw]];
            const int a = T.lca[(size_t)x * n + w];
            const int cw = child_toward(T, a, w);
            const int lw = T.sz[cw];
            int cx = -1, lx = 0;
            if (x != a) { cx = child_toward(T, a, x); lx = T.sz[cx]; }
            const unsigned pw = T.ph[w], px = T.ph[x];
            if ((pw & px) == pw) {
                Cand c; c.s = x; c.r = w; c.a = a; c.dir = 0;
                c.lo_s = cx; c.len_s = lx; c.lo_r = cw; c.len_r = lw; c.key = tie_key(T, x, w);
                X.cand[2 * w] = c;
                nc0 = (lx + lw + kChunk - 1) / kChunk;
            }
            if (x != 0 && (px & pw) == px) {
                Cand c; c.s = w; c.r = x; c.a = a; c.dir = 1;
                c.lo_s = cw; c.len_s = lw; c.lo_r = cx; c.len_r = lx; c.key = tie_key(T, w, x);
                X.cand[2 * w + 1] = c;
                nc1 = (lx + lw + kChunk - 1) / kChunk;
            }
        }
        X.nchunk[2 * w] = nc0;
        X.nchunk[2 * w + 1] = nc1;
    }
}

// ---------------------------------------------------------------- scan (one CTA)
// Exclusive prefix of the per-candidate chunk counts and the chunk -> candidate
// map.  Each thread owns a contiguous run of slots.
__global__ void __launch_bounds__(1024) k_scan(Topo T, Search X, Ctrl *C) {
    if (C->done) return;
    __shared__ int s_sum[32], s_cnt[32];
    const int m = 2 * T.n;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (m + nt - 1) / nt;
    const int b = min(tid * per, m), e = min(b + per, m);
    int sum = 0, cnt = 0;
    for (int i = b; i < e; ++i) { int c = X.nchunk[i]; sum += c; cnt += (c > 0); }
    // block exclusive scan of sum, block total of cnt
    const int lane = tid & 31, wid = tid >> 5;
    int inc = sum;
    for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, inc, o); if (lane >= o) inc += y; }
    int wc = cnt;
    for (int o = 16; o > 0; o >>= 1) wc += __shfl_xor_sync(0xffffffffu, wc, o);
    if (lane == 31) s_sum[wid] = inc;
    if (lane == 0) s_cnt[wid] = wc;
    __syncthreads();
    if (wid == 0) {
        const int nw = (nt + 31) >> 5;
        int v = lane < nw ? s_sum[lane] : 0;
        int vi = v;
        for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, vi, o); if (lane >= o) vi += y; }
        if (lane < nw) s_sum[lane] = vi - v;               // exclusive warp offsets
        int c = lane < nw ? s_cnt[lane] : 0;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) s_cnt[0] = c;
    }
    __syncthreads();
    int acc = s_sum[wid] + inc - sum;
    for (int i = b; i < e; ++i) {
        const int c = X.nchunk[i];
        X.base[i] = acc;
        if (acc + c <= X.max_chunks)
            for (int j = 0; j < c; ++j) X.chunk_cand[acc + j] = i;
        acc += c;
    }
    if (tid == nt - 1) {
        X.base[m] = acc;
        C->n_valid = s_cnt[0];
        C->candidates += s_cnt[0];
        if (acc > X.max_chunks) {           // cannot happen with the sizing rule; stop cleanly
            C->err = 4;
            C->done = 1;
            C->total_chunks = 0;
        } else {
            C->total_chunks = acc;
        }
    }
}

// ---------------------------------------------------------------- sweep
// One warp per chunk of kChunk consecutive positions of one candidate's
// affected ranges (s side first, then r side); one position per lane.  The
// warp writes the chunk's sum of score changes and its largest new MICE.
__global__ void __launch_bounds__(256) k_sweep(Topo T, State S, Search X, Ctrl *C) {
    if (C->done) return;
    const int n = T.n, L = T.L;
    const int total = C->total_chunks;
    const bool prof = C->profile;
    if (prof && blockIdx.x == 0 && threadIdx.x == 0) C->sweeps_run += 1;
    double flops = 0.0;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int g = warp; g < total; g += nwarps) {
        const int c = X.chunk_cand[g];
        const Cand cd = X.cand[c];
        const int j = g - X.base[c];
        const int pos = j * kChunk + lane;
        const unsigned phr = T.ph[cd.r];
        double2 Ir[kMaxScen * 3];
        load_ir(S, n, L, cd.r, Ir);
        double dsum = 0.0, mx = 0.0;
        double mnew[kMaxScen];
        if (pos < cd.len_s + cd.len_r) {
            const bool sside = pos < cd.len_s;
            const int k = sside ? cd.lo_s + pos : cd.lo_r + (pos - cd.len_s);
            if (S.label[k] == k && k != cd.r) {
                double2 G[9];
                delta_z(T, n, cd, sside, k, G);
                const bool merged = (k == cd.s);
                cluster_mice(T, S, n, L, k, merged, cd.r, G, Ir, phr, mnew);
                for (int l = 0; l < L; ++l) {
                    dsum += mnew[l] - S.mice[(size_t)l * n + k];
                    if (merged) dsum -= S.mice[(size_t)l * n + cd.r];
                    mx = fmax(mx, mnew[l]);
                }
                // G: 9 complex subtractions; per scenario and phase: |phi_r| complex
                // multiply-adds, the voltage update, |V|, two differences, two maxima
                if (prof) flops += 18.0 + (double)L * __popc(T.ph[k]) * (8.0 * __popc(phr) + 10.0);
            }
        }
        if (j == 0 && lane == 0 && cd.s == cd.a) {
            // s is the common ancestor: its voltage does not move, its cluster grows
            cluster_mice(T, S, n, L, cd.s, true, cd.r, nullptr, Ir, phr, mnew);
            for (int l = 0; l < L; ++l) {
                dsum += mnew[l] - S.mice[(size_t)l * n + cd.s] - S.mice[(size_t)l * n + cd.r];
                mx = fmax(mx, mnew[l]);
            }
            if (prof) flops += (double)L * __popc(T.ph[cd.s]) * 8.0;
        }
        dsum = warp_sum(dsum);
        mx = warp_max(mx);
        if (lane == 0) X.partial[g] = make_double2(dsum, mx);
    }
    if (prof) {
        flops = warp_sum(flops);
        if (lane == 0 && flops > 0.0) atomicAdd(&C->sweep_flops, flops);
    }
}

// ---------------------------------------------------------------- selection (one CTA)
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
struct MinU { __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a < b ? a : b; } };

// Scores D(c), feasibility (every affected cluster within the margin), the
// minimum m over feasible candidates, the tie band [m, m + tau] and the
// smallest (r, s) in it.  Stops the search when nothing is feasible.
__global__ void __launch_bounds__(1024) k_select(Topo T, Search X, Ctrl *C) {
    if (C->done) return;
    __shared__ double s_d[32];
    __shared__ unsigned long long s_u[32];
    const int m = 2 * T.n;
    const int t = C->t;
    const double margin = C->margin, tau = C->tau, s_cur = C->s_cur;
    double best = INFINITY;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        const int nc = X.nchunk[c];
        if (nc == 0) continue;
        const int b = X.base[c];
        double d = 0.0, mx = 0.0;
        for (int g = b; g < b + nc; ++g) { double2 p = X.partial[g]; d += p.x; mx = fmax(mx, p.y); }
        const int f = (mx <= margin);
        X.score[c] = d;
        X.feas[c] = f;
        if (f) best = fmin(best, d);
    }
    best = block_reduce(best, MinD(), s_d);
    const bool rec = t < X.rec_iters;
    if (best == INFINITY) {
        if (rec) {
            for (int c = threadIdx.x; c < m; c += blockDim.x) {
                if (X.nchunk[c] == 0) continue;
                const int i = atomicAdd(&X.rec_count[t], 1);
                X.rec_s[(size_t)t * m + i] = T.orig[X.cand[c].s];
                X.rec_r[(size_t)t * m + i] = T.orig[X.cand[c].r];
                X.rec_score[(size_t)t * m + i] = INFINITY;
            }
        }
        if (threadIdx.x == 0) { C->done = 1; C->stop_reason = 1; C->commit = 0; }
        return;
    }
    const double edge = best + tau;
    unsigned long long key = ~0ull;
    double gap = INFINITY;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        if (X.nchunk[c] == 0 || !X.feas[c]) continue;
        const double d = X.score[c];
        if (d <= edge) { unsigned long long k = X.cand[c].key; if (k < key) key = k; }
        else gap = fmin(gap, d - edge);
    }
    key = block_reduce(key, MinU(), s_u);
    gap = block_reduce(gap, MinD(), s_d);
    for (int c = threadIdx.x; c < m; c += blockDim.x)
        if (X.nchunk[c] != 0 && X.feas[c] && X.score[c] <= edge && X.cand[c].key == key) C->win = c;
    if (rec) {
        for (int c = threadIdx.x; c < m; c += blockDim.x) {
            if (X.nchunk[c] == 0) continue;
            const int i = atomicAdd(&X.rec_count[t], 1);
            X.rec_s[(size_t)t * m + i] = T.orig[X.cand[c].s];
            X.rec_r[(size_t)t * m + i] = T.orig[X.cand[c].r];
            X.rec_score[(size_t)t * m + i] = X.feas[c] ? s_cur + X.score[c] : INFINITY;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int w = C->win;
        X.dec_s[t] = T.orig[X.cand[w].s];
        X.dec_r[t] = T.orig[X.cand[w].r];
        X.dec_score[t] = s_cur + X.score[w];
        X.dec_gap[t] = gap;
        X.dec_ncand[t] = C->n_valid;
        C->win_d = X.score[w];
        C->gap = gap;
        C->commit = 1;
    }
}

// ---------------------------------------------------------------- commit
// Applies the selected candidate: r's cluster joins s (labels), the affected
// super-nodes take their new voltages and MICE, s takes the merged extremes and
// the sum of both injections (I = A Ihat), and the quotient edge of the merged
// cluster is the one of whichever cluster was above.  Runs only when the
// selection chose a winner (commit flag); nothing in this kernel reads the
// fields that its own thread 0 updates.
__global__ void k_commit(Topo T, State S, Search X, Ctrl *C) {
    if (!C->commit) return;
    const int n = T.n, L = T.L;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    const Cand cd = X.cand[C->win];
    const unsigned phr = T.ph[cd.r];
    double2 Ir[kMaxScen * 3];
    load_ir(S, n, L, cd.r, Ir);
    const int count = cd.len_s + cd.len_r;
    const int span = max(n, count);
    double mnew[kMaxScen];
    for (int i = gt; i < span; i += gs) {
        if (i < n && S.label[i] == cd.r) S.label[i] = cd.s;
        if (i >= count) continue;
        const bool sside = i < cd.len_s;
        const int k = sside ? cd.lo_s + i : cd.lo_r + (i - cd.len_s);
        if (k == cd.r || S.label[k] != k) continue;     // members and r carry no voltage
        double2 G[9];
        delta_z(T, n, cd, sside, k, G);
        const bool merged = (k == cd.s);
        cluster_mice(T, S, n, L, k, merged, cd.r, G, Ir, phr, mnew);
        const unsigned phk = T.ph[k];
        for (int l = 0; l < L; ++l) {
            for (int p = 0; p < 3; ++p) {
                if (!(phk >> p & 1u)) continue;
                double2 dv = make_double2(0.0, 0.0);
                for (int q = 0; q < 3; ++q)
                    if (phr >> q & 1u) dv = cadd(dv, cmul(G[p * 3 + q], Ir[l * 3 + q]));
                S.vcur[sidx(l, p, k, n)] = cadd(S.vcur[sidx(l, p, k, n)], dv);
                if (merged) {
                    S.hi[sidx(l, p, k, n)] = fmax(S.hi[sidx(l, p, k, n)], S.hi[sidx(l, p, cd.r, n)]);
                    S.lo[sidx(l, p, k, n)] = fmin(S.lo[sidx(l, p, k, n)], S.lo[sidx(l, p, cd.r, n)]);
                }
            }
            S.mice[(size_t)l * n + k] = mnew[l];
        }
    }
    if (gt == 0) {
        if (cd.s == cd.a) {
            cluster_mice(T, S, n, L, cd.s, true, cd.r, nullptr, Ir, phr, mnew);
            for (int l = 0; l < L; ++l) {
                for (int p = 0; p < 3; ++p) {
                    S.hi[sidx(l, p, cd.s, n)] = fmax(S.hi[sidx(l, p, cd.s, n)], S.hi[sidx(l, p, cd.r, n)]);
                    S.lo[sidx(l, p, cd.s, n)] = fmin(S.lo[sidx(l, p, cd.s, n)], S.lo[sidx(l, p, cd.r, n)]);
                }
                S.mice[(size_t)l * n + cd.s] = mnew[l];
            }
        }
        for (int l = 0; l < L; ++l) {
            for (int q = 0; q < 3; ++q)
                if (phr >> q & 1u) S.icur[sidx(l, q, cd.s, n)] = cadd(S.icur[sidx(l, q, cd.s, n)], Ir[l * 3 + q]);
            S.mice[(size_t)l * n + cd.r] = 0.0;
        }
        if (cd.dir == 1) S.top[cd.s] = S.top[cd.r];
        C->s_cur += C->win_d;
        const int t = C->t + 1;
        C->t = t;
        if (t >= C->max_merges) { C->done = 1; C->stop_reason = 0; }
    }
}

// Largest MICE of the final state into the record of the last merge (the
// per-iteration setup does this for all earlier merges).
__global__ void k_final_maxerr(Topo T, State S, Search X, const Ctrl *C) {
    const int n = T.n, L = T.L, t = C->t;
    if (t < 1) return;
    double m = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        if (S.label[k] == k)
            for (int l = 0; l < L; ++l) m = fmax(m, S.mice[(size_t)l * n + k]);
    m = warp_max(m);
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
