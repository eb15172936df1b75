// okr_kron.cu -- the Kron-reduced admittance Y_Kron of a kept bus set
// (Sec. II-B, eq. Y_kron: Y_KK - Y_KR Y_RR^-1 Y_RK over the kept phase-nodes,
// the slack bus included).
//
// Structure used.  The reduced buses form connected components of the tree.
// Eliminating one component R touches only the lines incident to R, so its
// contribution to Y_Kron is the Schur complement of that small sub-network
// onto its boundary: the kept bus p above R's top and the kept buses ("ports")
// whose parent lies in R.  A kept bus whose parent is kept forms a one-line
// group of its own.  Two groups share at most one bus, so every off-diagonal
// block of Y_Kron is written by exactly one group.
//
// Per group, with p as the reference, the sub-network's bus impedance matrix
// between ports is a path-impedance difference (the same closed form as the
// search uses): Z_port[(i,a),(j,b)] = Zc(lca(c_i, c_j))[a][b] - Zc(p)[a][b].
// Its inverse is the port block of the Schur complement; the blocks between p
// and the ports follow from the zero row and column sums that every
// series-only network has per phase (Y 1_b = 0 and 1_b^T Y = 0).  Diagonal
// blocks, which several groups share, are taken at the end from the same zero
// row sums, so that no two threads accumulate into one entry.
//
// Arithmetic: FP64 throughout.  Groups are small (a few to a few tens of
// phase-nodes on realistic feeders), so each is inverted by one CTA with
// Gauss-Jordan elimination and partial pivoting, in shared memory up to
// kKronShared phase-nodes and in a global scratch region above.
#include "okr_internal.cuh"
#include "okr_kernels.cuh"

namespace okr {

namespace {

__device__ __forceinline__ int popc3(unsigned m) { return __popc(m & 7u); }

// Exclusive block-wide scan of one value per thread (blockDim.x = 1024);
// returns the prefix and writes the block total to *total.
__device__ long long block_exscan(long long v, long long *sh, long long *total) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) sh[lane] = w;
    }
    __syncthreads();
    const long long before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
    *total = sh[nw - 1];
    __syncthreads();
    return before;
}

// In-place heap sort of a[0..m) (ascending).
__device__ void heap_sort(int *a, int m) {
    auto sift = [&](int root, int end) {
        while (2 * root + 1 < end) {
            int c = 2 * root + 1;
            if (c + 1 < end && a[c + 1] > a[c]) ++c;
            if (a[root] >= a[c]) return;
            const int t = a[root]; a[root] = a[c]; a[c] = t;
            root = c;
        }
    };
    for (int s = m / 2 - 1; s >= 0; --s) sift(s, m);
    for (int e = m - 1; e > 0; --e) {
        const int t = a[0]; a[0] = a[e]; a[e] = t;
        sift(0, e);
    }
}

// Output row of phase a of preorder bus v.
__device__ __forceinline__ int out_row(const Topo &T, const int *out_off, int v, int a) {
    return out_off[T.orig[v]] + popc3(T.ph[v] & ((1u << a) - 1u));
}

}  // namespace

// Groups, ports and output numbering (one CTA of 1024 threads).
//   kept_in (caller order, may be null) or label (kept = label[v] == v).
__global__ void __launch_bounds__(1024) k_kron_groups(Topo T, const int *label, const uint8_t *kept_in, KronWork W) {
    const int n = T.n, tid = threadIdx.x, nt = blockDim.x;
    __shared__ long long sh[32];
    __shared__ int s_bad, s_maxd;
    if (tid == 0) { s_bad = 0; s_maxd = 0; }
    for (int v = tid; v < n; v += nt) {
        W.keptp[v] = kept_in ? (kept_in[T.orig[v]] != 0) : (label[v] == v);
        W.cnt[v] = 0;
        W.dsum[v] = 0;
        W.fill[v] = 0;
        W.g[v] = -1;
    }
    __syncthreads();
    if (!W.keptp[0]) {
        if (tid == 0) W.hdr->err = 1;
        return;
    }
    // output offsets in caller order
    long long carry = 0;
    for (int base = 0; base < n; base += nt) {
        const int i = base + tid;
        long long c = 0;
        if (i < n) { const int v = T.pre[i]; c = W.keptp[v] ? popc3(T.ph[v]) : 0; }
        long long tot;
        const long long ex = block_exscan(c, sh, &tot);
        if (i < n) W.out_off[i] = (int)(carry + ex);
        carry += tot;
    }
    const int kphi = (int)carry;
    if (tid == 0) W.out_off[n] = kphi;
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        const int v = T.pre[i];
        if (!W.keptp[v]) continue;
        int r = W.out_off[i];
        for (int a = 0; a < 3; ++a)
            if (T.ph[v] >> a & 1u) W.pn[r++] = 3 * i + a;
    }
    // component top of every reduced bus, level by level
    const int maxd = T.maxd[0];
    for (int d = 1; d <= maxd; ++d) {
        for (int x = T.level_off[d] + tid; x < T.level_off[d + 1]; x += nt) {
            const int v = T.level_bus[x];
            if (W.keptp[v]) continue;
            const int par = T.parent[v];
            W.g[v] = W.keptp[par] ? v : W.g[par];
        }
        __syncthreads();
    }
    // group key of every kept non-root bus: its parent's component, or itself
    for (int c = 1 + tid; c < n; c += nt) {
        if (!W.keptp[c]) continue;
        const int par = T.parent[c];
        const int k = W.keptp[par] ? c : W.g[par];
        W.key[c] = k;
        atomicAdd(&W.cnt[k], 1);
        atomicAdd(&W.dsum[k], popc3(T.ph[c]));
    }
    __syncthreads();
    // port offsets, group index, row offsets, big-scratch offsets (keys in preorder)
    long long c_port = 0, c_grp = 0, c_row = 0;
    for (int base = 0; base < n; base += nt) {
        const int v = base + tid;
        const int m = v < n ? W.cnt[v] : 0;
        long long t1, t2, t3;
        const long long e1 = block_exscan(m, sh, &t1);
        const long long e2 = block_exscan(m > 0 ? 1 : 0, sh, &t2);
        const long long e3 = block_exscan(m > 0 ? W.dsum[v] : 0, sh, &t3);
        if (v < n) {
            W.goff[v] = (int)(c_port + e1);
            if (m > 0) {
                const int gi = (int)(c_grp + e2);
                W.gkey[gi] = v;
                W.gp[gi] = T.parent[v];
                W.gd[gi] = W.dsum[v];
                W.gport[gi] = (int)(c_port + e1);
                W.grow[gi] = (int)(c_row + e3);
                atomicMax(&s_maxd, W.dsum[v]);
            }
        }
        c_port += t1;
        c_grp += t2;
        c_row += t3;
    }
    const int ngroups = (int)c_grp;
    if (tid == 0) { W.gport[ngroups] = (int)c_port; W.grow[ngroups] = (int)c_row; }
    __syncthreads();
    for (int c = 1 + tid; c < n; c += nt) {
        if (!W.keptp[c]) continue;
        const int k = W.key[c];
        const int slot = atomicAdd(&W.fill[k], 1);
        W.ports[W.goff[k] + slot] = c;
    }
    __syncthreads();
    // per group: ports in increasing preorder id, then its phase-node rows
    for (int gi = tid; gi < ngroups; gi += nt) {
        int *pl = W.ports + W.gport[gi];
        const int m = W.gport[gi + 1] - W.gport[gi];
        heap_sort(pl, m);
        int r = W.grow[gi];
        for (int x = 0; x < m; ++x) {
            const int c = pl[x];
            for (int a = 0; a < 3; ++a)
                if (T.ph[c] >> a & 1u) W.rows[r++] = 4 * c + a;
        }
    }
    // global scratch for groups above the shared-memory size
    long long c_big = 0;
    for (int base = 0; base < ngroups; base += nt) {
        const int gi = base + tid;
        long long need = 0;
        if (gi < ngroups) {
            const long long d = W.gd[gi];
            need = d > kKronShared ? d * (d + 2) : 0;
        }
        long long tot;
        const long long ex = block_exscan(need, sh, &tot);
        if (gi < ngroups) W.gbig[gi] = c_big + ex;
        c_big += tot;
    }
    if (tid == 0) {
        W.hdr->n_groups = ngroups;
        W.hdr->k_phi = kphi;
        W.hdr->max_d = s_maxd;
        W.hdr->big_total = c_big;
    }
}

// One group per CTA: Z_port, its inverse, and the off-diagonal blocks of Y_Kron.
__global__ void k_kron_solve(Topo T, KronWork W, double2 *big, double2 *Y, int K) {
    extern __shared__ double2 smem[];
    const int gi = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int n = T.n;
    const int d = W.gd[gi], p = W.gp[gi];
    const int *rows = W.rows + W.grow[gi];
    double2 *A, *col;
    int *perm;
    if (d <= kKronShared) {
        A = smem;
        col = smem + kKronShared * kKronShared;
        perm = reinterpret_cast<int *>(col + kKronShared);
    } else {
        A = big + W.gbig[gi];
        col = A + (size_t)d * d;
        perm = reinterpret_cast<int *>(col + d);
    }
    __shared__ int s_piv, s_sing;
    __shared__ double s_best[32];
    __shared__ int s_bidx[32];
    if (tid == 0) s_sing = 0;
    const double2 *zp = T.zc + (size_t)p * 9;
    for (int e = tid; e < d * d; e += nt) {
        const int r = e / d, s = e % d;
        const int cr = rows[r] >> 2, a = rows[r] & 3, cs = rows[s] >> 2, b = rows[s] & 3;
        const int y = T.lca[(size_t)cr * n + cs];
        A[e] = csub(T.zc[(size_t)y * 9 + a * 3 + b], zp[a * 3 + b]);
    }
    __syncthreads();
    // Gauss-Jordan inversion in place, partial pivoting by rows
    for (int k = 0; k < d; ++k) {
        double best = -1.0;
        int bi = d;
        for (int i = k + tid; i < d; i += nt) {
            const double2 x = A[(size_t)i * d + k];
            const double m = x.x * x.x + x.y * x.y;
            if (m > best) { best = m; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((tid & 31) == 0) { s_best[tid >> 5] = best; s_bidx[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            double bb = -1.0;
            int ii = d;
            for (int w = 0; w < (nt + 31) / 32; ++w)
                if (s_best[w] > bb || (s_best[w] == bb && s_bidx[w] < ii)) { bb = s_best[w]; ii = s_bidx[w]; }
            s_piv = ii;
            if (!(bb > 0.0)) s_sing = 1;
            perm[k] = ii;
        }
        __syncthreads();
        if (s_sing) break;
        const int pr = s_piv;
        if (pr != k)
            for (int j = tid; j < d; j += nt) {
                const double2 t = A[(size_t)k * d + j];
                A[(size_t)k * d + j] = A[(size_t)pr * d + j];
                A[(size_t)pr * d + j] = t;
            }
        __syncthreads();
        const double2 inv = cdiv(make_double2(1.0, 0.0), A[(size_t)k * d + k]);
        __syncthreads();
        for (int j = tid; j < d; j += nt)
            A[(size_t)k * d + j] = (j == k) ? inv : cmul(A[(size_t)k * d + j], inv);
        for (int i = tid; i < d; i += nt)
            if (i != k) col[i] = A[(size_t)i * d + k];
        __syncthreads();
        for (int e = tid; e < d * d; e += nt) {
            const int i = e / d, j = e % d;
            if (i == k) continue;
            const double2 f = col[i];
            if (j == k) A[e] = make_double2(-(f.x * inv.x - f.y * inv.y), -(f.x * inv.y + f.y * inv.x));
            else A[e] = csub(A[e], cmul(f, A[(size_t)k * d + j]));
        }
        __syncthreads();
    }
    if (s_sing) {
        if (tid == 0) atomicExch(&W.hdr->err, 2);
        return;
    }
    for (int k = d - 1; k >= 0; --k) {
        const int pr = perm[k];
        if (pr != k)
            for (int i = tid; i < d; i += nt) {
                const double2 t = A[(size_t)i * d + k];
                A[(size_t)i * d + k] = A[(size_t)i * d + pr];
                A[(size_t)i * d + pr] = t;
            }
        __syncthreads();
    }
    // port-port blocks of distinct buses
    for (int e = tid; e < d * d; e += nt) {
        const int r = e / d, s = e % d;
        const int cr = rows[r] >> 2, cs = rows[s] >> 2;
        if (cr == cs) continue;
        Y[(size_t)out_row(T, W.out_off, cr, rows[r] & 3) * K + out_row(T, W.out_off, cs, rows[s] & 3)] = A[e];
    }
    // p-port blocks: minus the per-phase column sums, and row sums
    for (int e = tid; e < 3 * d; e += nt) {
        const int a = e / d, x = e % d;
        if (!(T.ph[p] >> a & 1u)) continue;
        double2 cs = make_double2(0.0, 0.0), rs = make_double2(0.0, 0.0);
        for (int t = 0; t < d; ++t) {
            if ((rows[t] & 3) == a) cs = cadd(cs, A[(size_t)t * d + x]);
            if ((rows[t] & 3) == a) rs = cadd(rs, A[(size_t)x * d + t]);
        }
        const int op = out_row(T, W.out_off, p, a), ox = out_row(T, W.out_off, rows[x] >> 2, rows[x] & 3);
        Y[(size_t)op * K + ox] = make_double2(-cs.x, -cs.y);
        Y[(size_t)ox * K + op] = make_double2(-rs.x, -rs.y);
    }
}

// Diagonal blocks from the zero row sums: one warp per output row.
__global__ void k_kron_diag(KronWork W, double2 *Y, int K) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int R = gw; R < K; R += nw) {
        const int bus = W.pn[R] / 3;
        double2 a0 = make_double2(0.0, 0.0), a1 = a0, a2 = a0;
        for (int c = lane; c < K; c += 32) {
            const int q = W.pn[c];
            if (q / 3 == bus) continue;
            const double2 y = Y[(size_t)R * K + c];
            const int b = q % 3;
            if (b == 0) a0 = cadd(a0, y);
            else if (b == 1) a1 = cadd(a1, y);
            else a2 = cadd(a2, y);
        }
        for (int o = 16; o > 0; o >>= 1) {
            a0.x += __shfl_xor_sync(0xffffffffu, a0.x, o);
            a0.y += __shfl_xor_sync(0xffffffffu, a0.y, o);
            a1.x += __shfl_xor_sync(0xffffffffu, a1.x, o);
            a1.y += __shfl_xor_sync(0xffffffffu, a1.y, o);
            a2.x += __shfl_xor_sync(0xffffffffu, a2.x, o);
            a2.y += __shfl_xor_sync(0xffffffffu, a2.y, o);
        }
        // the bus's own columns are the (at most three) entries around R
        if (lane < 3) {
            const int b = lane;
            const double2 acc = b == 0 ? a0 : (b == 1 ? a1 : a2);
            for (int c = max(0, R - 2); c < min(K, R + 3); ++c)
                if (W.pn[c] == 3 * bus + b) Y[(size_t)R * K + c] = make_double2(-acc.x, -acc.y);
        }
    }
}

// Radialization (Sec. V): in the tree, the buses of a reduced component and
// its boundary span a sub-tree; a reduced bus is critical when it has degree
// >= 3 in that sub-tree, i.e. when two or more of its children lead to the
// boundary (a kept child, or a reduced child with a kept bus below it in the
// component) -- its parent edge always leads to the boundary bus above the
// component.  One CTA, deepest level first.  crit: [n] flags, caller order.
__global__ void __launch_bounds__(1024) k_radial_critical(Topo T, const int *label, const uint8_t *kept_in, KronWork W,
                                                          uint8_t *crit, int *count) {
    const int n = T.n, tid = threadIdx.x, nt = blockDim.x;
    __shared__ int s_cnt;
    if (tid == 0) s_cnt = 0;
    for (int v = tid; v < n; v += nt) {
        W.keptp[v] = kept_in ? (kept_in[T.orig[v]] != 0) : (label[v] == v);
        W.fill[v] = 0;                              // reused: "a kept bus lies below, inside the component"
    }
    __syncthreads();
    const int maxd = T.maxd[0];
    for (int d = maxd; d >= 0; --d) {
        for (int x = T.level_off[d] + tid; x < T.level_off[d + 1]; x += nt) {
            const int v = T.level_bus[x];
            int c2 = 0;
            if (!W.keptp[v])
                for (int c = T.child_off[v]; c < T.child_off[v + 1]; ++c) {
                    const int ch = T.child[c];
                    if (W.keptp[ch] || W.fill[ch]) ++c2;
                }
            W.fill[v] = c2 > 0;
            const int cr = (!W.keptp[v] && c2 >= 2) ? 1 : 0;
            crit[T.orig[v]] = (uint8_t)cr;
            if (cr) atomicAdd(&s_cnt, 1);
        }
        __syncthreads();
    }
    if (tid == 0) *count = s_cnt;
}

cudaError_t launch_kron_solve(int n_groups, Topo T, KronWork W, double2 *big, double2 *Y, int K, cudaStream_t st) {
    const size_t smem = sizeof(double2) * ((size_t)kKronShared * kKronShared + kKronShared) + sizeof(int) * kKronShared;
    cudaError_t e = cudaFuncSetAttribute(k_kron_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (n_groups > 0) k_kron_solve<<<n_groups, 256, smem, st>>>(T, W, big, Y, K);
    return cudaGetLastError();
}

}  // namespace okr
