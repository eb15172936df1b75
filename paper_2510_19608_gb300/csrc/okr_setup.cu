// okr_setup.cu -- once-per-feeder work on the device: validation, preorder
// renumbering, lowest-common-ancestor table, path impedances, the
// backward/forward-sweep load flow that produces the scenario library
// (Sec. III: operating points of the full network), the injections
// Ihat = Y Vhat (Sec. II-A), and the initial reduction state of Algorithm 1
// (every bus its own super-node, I = Ihat).
#include "okr_internal.cuh"
#include "okr_kernels.cuh"

namespace okr {

// ---------------------------------------------------------------- small dense helpers
// Inverse of the sub-block of a 3x3 complex matrix on phase mask m (Gauss-Jordan
// with partial pivoting); entries outside the sub-block are zero.  Returns false
// if the sub-block is singular.
__device__ bool inv3_sub(const double2 *a, unsigned m, double2 *out) {
    int idx[3], k = 0;
    for (int p = 0; p < 3; ++p)
        if (m >> p & 1u) idx[k++] = p;
    double2 w[3][6];
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < 2 * k; ++j)
            w[i][j] = (j < k) ? a[idx[i] * 3 + idx[j]] : make_double2(j - k == i ? 1.0 : 0.0, 0.0);
    for (int c = 0; c < k; ++c) {
        int piv = c;
        double best = cmag(w[c][c]);
        for (int i = c + 1; i < k; ++i) {
            double v = cmag(w[i][c]);
            if (v > best) { best = v; piv = i; }
        }
        if (best == 0.0) return false;
        if (piv != c)
            for (int j = 0; j < 2 * k; ++j) { double2 t = w[c][j]; w[c][j] = w[piv][j]; w[piv][j] = t; }
        double2 d = w[c][c];
        for (int j = 0; j < 2 * k; ++j) w[c][j] = cdiv(w[c][j], d);
        for (int i = 0; i < k; ++i) {
            if (i == c) continue;
            double2 f = w[i][c];
            for (int j = 0; j < 2 * k; ++j) w[i][j] = csub(w[i][j], cmul(f, w[c][j]));
        }
    }
    for (int q = 0; q < 9; ++q) out[q] = make_double2(0.0, 0.0);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) out[idx[i] * 3 + idx[j]] = w[i][k + j];
    return true;
}

__device__ __forceinline__ void block_barrier() { __syncthreads(); }

// out[i] = in[0] + ... + in[i - 1] for i <= n (one CTA, blockDim.x a multiple
// of 32, at most 1024; tiles of blockDim.x with a carried total).
__device__ void block_exclusive_scan(const int *in, int *out, int n) {
    __shared__ int s_w[32];
    __shared__ int s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + tid;
        const int c = i < n ? in[i] : 0;
        int x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nw ? s_w[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < nw) s_w[lane] = w;
        }
        __syncthreads();
        const int carry = s_carry;
        if (i < n) out[i] = carry + (warp > 0 ? s_w[warp - 1] : 0) + x - c;
        __syncthreads();
        if (tid == 0) s_carry = carry + s_w[nw - 1];
        __syncthreads();
    }
    if (tid == 0) out[n] = s_carry;
    __syncthreads();
}

// ---------------------------------------------------------------- topology (one CTA)
// Input in caller numbering.  Scratch arrays (caller numbering): dep, anc/anc2,
// d2, size, ccount.  Writes the Topo arrays in preorder numbering.
__device__ void dev_topology(int n, const int *__restrict__ parent_in, const uint8_t *__restrict__ ph_in,
                           Topo T, int *dep, int *anc, int *anc2, int *d2, int *size, int *ccount,
                           int *coff_c, int *child_c, int *err) {
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ int s_bad, s_maxd;
    if (tid == 0) { s_bad = 0; s_maxd = 0; }
    block_barrier();
    // 1. validation
    for (int i = tid; i < n; i += nt) {
        int p = parent_in[i];
        unsigned m = ph_in[i];
        bool ok = (m != 0u) && (m <= 7u);
        if (i == 0) ok = ok && (p == -1);
        else ok = ok && (p >= 0) && (p < i) && ((m & ph_in[p]) == m);
        if (!ok) atomicExch(&s_bad, 1);
    }
    block_barrier();
    if (s_bad) { if (tid == 0) atomicCAS(err, 0, 1); return; }
    // 2. depth by pointer jumping (caller numbering)
    for (int i = tid; i < n; i += nt) { anc[i] = (i == 0) ? 0 : parent_in[i]; dep[i] = (i == 0) ? 0 : 1; }
    block_barrier();
    int *a0 = anc, *a1 = anc2, *d0 = dep, *d1 = d2;
    for (int step = 1; step < 2 * n; step <<= 1) {
        for (int i = tid; i < n; i += nt) { d1[i] = d0[i] + d0[a0[i]]; a1[i] = a0[a0[i]]; }
        block_barrier();
        int *t = a0; a0 = a1; a1 = t;
        t = d0; d0 = d1; d1 = t;
    }
    if (d0 != dep) {
        for (int i = tid; i < n; i += nt) dep[i] = d0[i];
        block_barrier();
    }
    for (int i = tid; i < n; i += nt) atomicMax(&s_maxd, dep[i]);
    block_barrier();
    const int maxd = s_maxd;
    // 3. level lists (caller ids, stable order inside a level is irrelevant)
    for (int i = tid; i < maxd + 2; i += nt) T.level_off[i] = 0;
    for (int i = tid; i < n; i += nt) { size[i] = 1; ccount[i] = 0; }
    block_barrier();
    for (int i = tid; i < n; i += nt) atomicAdd(&T.level_off[dep[i] + 1], 1);
    block_barrier();
    if (tid == 0) {
        for (int d = 0; d <= maxd; ++d) T.level_off[d + 1] += T.level_off[d];
    }
    block_barrier();
    // children counts
    for (int i = tid + 1; i < n; i += nt) atomicAdd(&ccount[parent_in[i]], 1);
    block_barrier();
    // 4. subtree sizes, deepest level first (integer atomics: order-independent)
    for (int d = maxd; d >= 1; --d) {
        for (int i = tid; i < n; i += nt)
            if (dep[i] == d) atomicAdd(&size[parent_in[i]], size[i]);
        block_barrier();
    }
    // 5. children CSR in caller numbering, each list sorted by caller id
    block_exclusive_scan(ccount, coff_c, n);
    for (int i = tid; i < n; i += nt) ccount[i] = 0;
    block_barrier();
    for (int i = tid + 1; i < n; i += nt) {
        int p = parent_in[i];
        int slot = atomicAdd(&ccount[p], 1);
        child_c[coff_c[p] + slot] = i;
    }
    block_barrier();
    for (int p = tid; p < n; p += nt) {
        int b = coff_c[p], e = coff_c[p + 1];
        for (int x = b + 1; x < e; ++x) {           // insertion sort (degrees are small)
            int v = child_c[x], y = x - 1;
            while (y >= b && child_c[y] > v) { child_c[y + 1] = child_c[y]; --y; }
            child_c[y + 1] = v;
        }
    }
    block_barrier();
    // 6. preorder positions, top-down
    if (tid == 0) T.pre[0] = 0;
    block_barrier();
    for (int d = 0; d < maxd; ++d) {
        for (int i = tid; i < n; i += nt) {
            if (dep[i] != d) continue;
            int pos = T.pre[i] + 1;
            for (int x = coff_c[i]; x < coff_c[i + 1]; ++x) {
                int c = child_c[x];
                T.pre[c] = pos;
                pos += size[c];
            }
        }
        block_barrier();
    }
    // 7. preorder-indexed copies; child lists become preorder ids
    for (int i = tid; i < n; i += nt) {
        int v = T.pre[i];
        T.orig[v] = i;
        T.parent[v] = (i == 0) ? -1 : T.pre[parent_in[i]];
        T.sz[v] = size[i];
        T.depth[v] = dep[i];
        T.ph[v] = ph_in[i];
    }
    block_barrier();
    for (int x = tid; x < n - 1; x += nt) child_c[x] = T.pre[child_c[x]];
    for (int i = tid; i < n; i += nt) ccount[i] = 0;
    block_barrier();
    for (int i = tid; i < n; i += nt) {
        int d = dep[i];
        int slot = atomicAdd(&ccount[d], 1);
        T.level_bus[T.level_off[d] + slot] = T.pre[i];
    }
    __shared__ int s_sum;
    if (tid == 0) s_sum = 0;
    __syncthreads();
    int part = 0;
    for (int i = tid; i < n; i += nt) part += size[i];
    atomicAdd(&s_sum, part);
    __syncthreads();
    if (tid == 0) { T.maxd[0] = maxd; T.maxd[1] = s_sum; }
}

__global__ void __launch_bounds__(1024) k_topology(int n, const int *__restrict__ parent_in, const uint8_t *__restrict__ ph_in,
                           Topo T, int *dep, int *anc, int *anc2, int *d2, int *size, int *ccount,
                           int *coff_c, int *child_c, int *err) {
    dev_topology(n, parent_in, ph_in, T, dep, anc, anc2, d2, size, ccount, coff_c, child_c, err);
}

// Children CSR indexed by preorder id (one CTA).  The children of preorder
// node v are those of caller bus orig[v], already converted to preorder ids
// and increasing.
__device__ void dev_child_offsets(int n, Topo T, const int *__restrict__ coff_c, const int *__restrict__ child_c) {
    // exclusive scan of the child counts in preorder, 1024 buses per pass
    __shared__ int s_w[32];
    __shared__ int s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int v = base + tid;
        int c = 0;
        if (v < n) { const int i = T.orig[v]; c = coff_c[i + 1] - coff_c[i]; }
        int x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nw ? s_w[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < nw) s_w[lane] = w;
        }
        __syncthreads();
        const int carry = s_carry;
        if (v < n) T.child_off[v] = carry + (warp > 0 ? s_w[warp - 1] : 0) + x - c;
        __syncthreads();
        if (tid == 0) s_carry = carry + s_w[nw - 1];
        __syncthreads();
    }
    if (tid == 0) T.child_off[n] = s_carry;
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        int i = T.orig[v];
        int b = coff_c[i], e = coff_c[i + 1];
        int o = T.child_off[v];
        for (int x = b; x < e; ++x) T.child[o + (x - b)] = child_c[x];
    }
}

__global__ void __launch_bounds__(1024) k_child_offsets(int n, Topo T, const int *__restrict__ coff_c, const int *__restrict__ child_c) {
    dev_child_offsets(n, T, coff_c, child_c);
}

// Sparse table of the minimum-depth bus over preorder windows: st[j*n + v] is the
// index of the shallowest bus in [v, v + 2^j).
__global__ void k_rmq_level(int n, int j, const int *__restrict__ depth, uint16_t *st) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    if (j == 0) { st[v] = (uint16_t)v; return; }
    int h = 1 << (j - 1);
    int a = st[(size_t)(j - 1) * n + v];
    int w = v + h;
    if (w + h <= n) {
        int b = st[(size_t)(j - 1) * n + w];
        if (depth[b] < depth[a]) a = b;
    }
    st[(size_t)j * n + v] = (uint16_t)a;
}

// All levels of the sparse table in one CTA (levels 0 .. nlev-1).
__device__ void dev_rmq_all(int n, int nlev, const int *__restrict__ depth, uint16_t *st) {
    for (int v = threadIdx.x; v < n; v += blockDim.x) st[v] = (uint16_t)v;
    __syncthreads();
    for (int j = 1; j < nlev; ++j) {
        const int h = 1 << (j - 1);
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            int a = st[(size_t)(j - 1) * n + v];
            const int w = v + h;
            if (w + h <= n) {
                const int b = st[(size_t)(j - 1) * n + w];
                if (depth[b] < depth[a]) a = b;
            }
            st[(size_t)j * n + v] = (uint16_t)a;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_rmq_all(int n, int nlev, const int *__restrict__ depth, uint16_t *st) {
    dev_rmq_all(n, nlev, depth, st);
}

// LCA[u][v] for all pairs (preorder ids).  For u < v: if v lies in u's subtree
// the answer is u; otherwise it is the parent of the shallowest bus in (u, v].
__device__ void dev_lca_fill(int n, const int *__restrict__ parent, const int *__restrict__ sz,
                             const int *__restrict__ depth, const uint16_t *__restrict__ st, uint16_t *lca,
                             size_t first, size_t stride) {
    // (u, v) of element e advanced by the stride without a division per
    // element (n * n < 2^31 for the 16-bit table)
    const size_t tot = (size_t)n * n;
    if (first >= tot) return;
    const int du = (int)(stride / n), dv = (int)(stride % n);
    int u = (int)(first / n), v = (int)(first % n);
    for (size_t e = first; e < tot; e += stride) {
        int lo = u < v ? u : v, hi = u < v ? v : u;
        int res;
        if (lo == hi || hi < lo + sz[lo]) {
            res = lo;
        } else {
            int len = hi - lo;                       // window (lo, hi]
            int j = 31 - __clz(len);
            int a = st[(size_t)j * n + lo + 1];
            int b = st[(size_t)j * n + hi - (1 << j) + 1];
            int m = depth[b] < depth[a] ? b : a;
            res = parent[m];
        }
        lca[e] = (uint16_t)res;
        u += du;
        v += dv;
        if (v >= n) { v -= n; ++u; }
    }
}

__global__ void k_lca_fill(int n, const int *__restrict__ parent, const int *__restrict__ sz,
                           const int *__restrict__ depth, const uint16_t *__restrict__ st, uint16_t *lca) {
    dev_lca_fill(n, parent, sz, depth, st, lca, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

// Line data in preorder: zl, yl (inverse on the bus phases); path impedance by
// levels (parents first).  One CTA.
// Line data: copies of the impedances and their inverses on the line's phases,
// one thread per bus over the whole grid.
__device__ void dev_line_inverses(int n, Topo T, const double *__restrict__ z_in, int *err, int first, int stride) {
    for (int v = first; v < n; v += stride) {
        const int i = T.orig[v];
        double2 z[9];
        for (int q = 0; q < 9; ++q) {
            z[q] = (v == 0) ? make_double2(0.0, 0.0) : make_double2(z_in[((size_t)i * 9 + q) * 2], z_in[((size_t)i * 9 + q) * 2 + 1]);
            T.zl[(size_t)v * 9 + q] = z[q];
        }
        double2 y[9];
        if (v == 0) {
            for (int q = 0; q < 9; ++q) y[q] = make_double2(0.0, 0.0);
        } else if (!inv3_sub(z, T.ph[v], y)) {
            atomicCAS(err, 0, 2);
            for (int q = 0; q < 9; ++q) y[q] = make_double2(0.0, 0.0);
        }
        for (int q = 0; q < 9; ++q) T.yl[(size_t)v * 9 + q] = y[q];
    }
}

__global__ void k_line_inverses(int n, Topo T, const double *__restrict__ z_in, int *err) {
    dev_line_inverses(n, T, z_in, err, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Path impedances root -> k level by level (one CTA), then their split into
// two floats for the screening sweep.
__device__ void dev_path_impedance(int n, Topo T) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int q = tid; q < 9; q += nt) T.zc[q] = make_double2(0.0, 0.0);
    __syncthreads();
    const int maxd = T.maxd[0];
    for (int d = 1; d <= maxd; ++d) {
        for (int x = T.level_off[d] + tid; x < T.level_off[d + 1]; x += nt) {
            int v = T.level_bus[x], p = T.parent[v];
            for (int q = 0; q < 9; ++q) T.zc[(size_t)v * 9 + q] = cadd(T.zc[(size_t)p * 9 + q], T.zl[(size_t)v * 9 + q]);
        }
        __syncthreads();
    }
    // single-precision split of the path impedances: zc ~ zh + zl
    for (int e = tid; e < 9 * n; e += nt) {
        const double2 z = T.zc[e];
        const float2 h = make_float2((float)z.x, (float)z.y);
        T.zh[e] = h;
        T.zlo[e] = make_float2((float)(z.x - (double)h.x), (float)(z.y - (double)h.y));
    }
}

__global__ void __launch_bounds__(1024) k_path_impedance(int n, Topo T) {
    dev_path_impedance(n, T);
}

cudaError_t launch_line_inverses(int n, Topo T, const double *z_in, int *err, int num_sms, cudaStream_t st) {
    // one warp per CTA: each line's inverse is a chain of FP64 operations, and
    // an SM's FP64 unit serves few warps at speed, so the lines go to as many
    // SMs as possible
    int blocks = (n + 31) / 32;
    if (blocks > num_sms * 8) blocks = num_sms * 8;
    k_line_inverses<<<blocks, 32, 0, st>>>(n, T, z_in, err);
    return cudaGetLastError();
}

cudaError_t launch_path_impedance(int n, Topo T, cudaStream_t st) {
    k_path_impedance<<<1, 1024, 0, st>>>(n, T);
    return cudaGetLastError();
}

cudaError_t launch_lines(int n, Topo T, const double *z_in, int *err, int num_sms, cudaStream_t st) {
    const cudaError_t e = launch_line_inverses(n, T, z_in, err, num_sms, st);
    return e != cudaSuccess ? e : launch_path_impedance(n, T, st);
}

// ---------------------------------------------------------------- load flow
// Backward/forward sweep for every scenario.  Constant-power wye loads: the
// current drawn at (k,p) is conj(S/V).  Backward: J_k = load(k) + the sum of the
// children's J (children in preorder order).  Forward: V_k = V_parent - z_k J_k.
// A scenario stops when max |dV| < tol (tested as max |dV|^2 < tol^2); one that
// has not stopped after max_iter sweeps is a failure.
//
// FP64 reciprocals, the 3x3 products and the squared changes dominate the arithmetic,
// and GB300's FP64 rate per SM is low, so these run over the whole cooperative
// grid; only the level-by-level sums (additions) run one CTA per (scenario,
// phase), staged in shared memory.  Four grid barriers per sweep:
//   S1 load currents I1 = conj(S / V)          (grid)
//   S2 line currents J = I1 + sum children J  (CTA per (l, p), deepest level first)
//   S3 drops D = z J                            (grid)
//   S4 new voltages Vn = Vn_parent - D          (CTA per (l, p), top down)
//   S5 |Vn - V|^2, V = Vn, per-scenario maximum (grid)
// S5 and the next sweep's S1 touch the same element on the same thread, so
// they run as one pass (the load currents of a scenario that has just
// converged are computed and never read).  I1, D and Vn share one buffer W
// (D overwrites I1, Vn overwrites D in place, I1 overwrites Vn).  The
// arithmetic is the same, operation for operation, as a one-thread-per-bus
// sweep.
constexpr int kPfShared = 2048;     // buses whose (l, p) slice is staged in shared memory

__device__ __forceinline__ unsigned pf_ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier on a monotonic counter; bounded by max_spins polls: returns
// false (and sets err = 6) when the wait gives up or another CTA already gave up.
__device__ bool pf_grid_sync(unsigned *count, int *err, unsigned nblocks, unsigned &epoch, long long max_spins) {
    __shared__ int s_ok;
    __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        const unsigned target = epoch * nblocks;
        __threadfence();
        atomicAdd(count, 1u);
        int ok = 1;
        long long spins = 0;
        // one L2 round trip per poll; another CTA's give-up is looked for every 64 polls
        while (pf_ld_acquire(count) < target) {
            if (++spins > max_spins || ((spins & 63) == 0 && *(volatile int *)err == 6)) { ok = 0; break; }
        }
        if (!ok) atomicCAS(err, 0, 6);
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok;
}

__global__ void __launch_bounds__(256) k_power_flow(int n, int L, Topo T, const double *__restrict__ s_in, double tol,
                                                    int max_iter, double2 *J, double2 *W, double *red, unsigned *bar,
                                                    int *iters, int *err, long long max_spins) {
    extern __shared__ double2 pf_sm[];
    __shared__ int s_live[kMaxScen];
    const int tid = threadIdx.x, nt = blockDim.x;
    const unsigned G = gridDim.x;
    const int gt = blockIdx.x * nt + tid, gs = (int)G * nt;
    const size_t N3 = (size_t)3 * n;
    const size_t tot = (size_t)L * N3;
    // an earlier setup step failed (every CTA reads the same flag: no writer runs)
    if (*reinterpret_cast<volatile const int *>(err) != 0) return;
    const int maxd = T.maxd[0];
    const double tol2 = tol * tol;                  // the test is max |dV|^2 < tol^2
    unsigned epoch = 0;
    for (size_t e = gt; e < tot; e += gs) {
        const int v = (int)(e % n), p = (int)((e / n) % 3);
        T.vhat[e] = (T.ph[v] >> p & 1u) ? T.vslack[p] : make_double2(0.0, 0.0);
    }
    if (tid < kMaxScen) s_live[tid] = tid < L;
    const bool line_cta = blockIdx.x < (unsigned)(3 * L);
    const int ll = blockIdx.x / 3, lp = blockIdx.x % 3;      // (scenario, phase) of a level CTA
    double2 *const loc = n <= kPfShared ? pf_sm : nullptr;
    bool conv_all = false;
    // the load current of element e on voltage vv (S1)
    auto set_load_current = [&](size_t e, int l, int p, int v, double2 vv) {
        double2 j = make_double2(0.0, 0.0);
        if (T.ph[v] >> p & 1u) {
            const size_t o = (((size_t)l * n + T.orig[v]) * 3 + p) * 2;
            const double2 sv = make_double2(__ldg(s_in + o), __ldg(s_in + o + 1));
            j = load_current(sv, vv);
        }
        W[e] = j;
    };
    __syncthreads();                                         // (s_live)
    // S1 of the first sweep (each element on the thread that set its voltage)
    for (size_t e = gt; e < tot; e += gs) {
        const int l = (int)(e / N3), p = (int)((e / n) % 3), v = (int)(e % n);
        set_load_current(e, l, p, v, T.vhat[e]);
    }
    if (!pf_grid_sync(bar, err, G, epoch, max_spins)) return;
    int it;
    for (it = 1; it <= max_iter; ++it) {
        if (gt == 0) for (int l = 0; l < L; ++l) red[((it + 1) % 3) * L + l] = 0.0;
        // S2: line currents, deepest level first
        if (line_cta && s_live[ll]) {
            const size_t off = ((size_t)ll * 3 + lp) * n;
            double2 *Jx = loc ? loc : J + off;
            if (loc) {
                for (int v = tid; v < n; v += nt) loc[v] = W[off + v];
            } else {
                for (int v = tid; v < n; v += nt) Jx[v] = W[off + v];
            }
            __syncthreads();
            for (int d = maxd; d >= 1; --d) {
                for (int x = T.level_off[d] + tid; x < T.level_off[d + 1]; x += nt) {
                    const int v = T.level_bus[x];
                    double2 j = Jx[v];
                    for (int c = T.child_off[v]; c < T.child_off[v + 1]; ++c) j = cadd(j, Jx[T.child[c]]);
                    Jx[v] = j;
                }
                __syncthreads();
            }
            if (loc)
                for (int v = tid; v < n; v += nt) J[off + v] = loc[v];
        }
        if (!pf_grid_sync(bar, err, G, epoch, max_spins)) return;
        // S3: drops z J on the phases of each line (root excluded)
        for (size_t e = gt; e < tot; e += gs) {
            const int l = (int)(e / N3), p = (int)((e / n) % 3), v = (int)(e % n);
            if (!s_live[l]) continue;
            const unsigned ph = T.ph[v];
            double2 drop = make_double2(0.0, 0.0);
            if (v > 0 && (ph >> p & 1u))
                for (int q = 0; q < 3; ++q)
                    if (ph >> q & 1u)
                        drop = cadd(drop, cmul(T.zl[(size_t)v * 9 + p * 3 + q], J[(size_t)l * N3 + (size_t)q * n + v]));
            W[e] = drop;
        }
        if (!pf_grid_sync(bar, err, G, epoch, max_spins)) return;
        // S4: new voltages, top down (Vn overwrites D)
        if (line_cta && s_live[ll]) {
            const size_t off = ((size_t)ll * 3 + lp) * n;
            double2 *Vx = loc ? loc : W + off;
            if (loc)
                for (int v = tid; v < n; v += nt) loc[v] = W[off + v];
            __syncthreads();
            if (tid == 0) Vx[0] = T.vhat[off];
            __syncthreads();
            for (int d = 1; d <= maxd; ++d) {
                for (int x = T.level_off[d] + tid; x < T.level_off[d + 1]; x += nt) {
                    const int v = T.level_bus[x];
                    Vx[v] = csub(Vx[T.parent[v]], Vx[v]);
                }
                __syncthreads();
            }
            if (loc)
                for (int v = tid; v < n; v += nt) W[off + v] = loc[v];
        }
        if (!pf_grid_sync(bar, err, G, epoch, max_spins)) return;
        // S5: change of the voltages, per-scenario maximum; then S1 of the next sweep
        double mx[kMaxScen] = {0.0, 0.0, 0.0, 0.0};
        for (size_t e = gt; e < tot; e += gs) {
            const int l = (int)(e / N3), p = (int)((e / n) % 3), v = (int)(e % n);
            if (!s_live[l]) continue;
            double2 vv = T.vhat[e];
            if (v != 0 && (T.ph[v] >> p & 1u)) {
                const double2 vn = W[e];
                double dd = cmag2(csub(vn, vv));             // squared change (compared with tol^2)
                if (!isfinite(dd)) dd = INFINITY;           // a diverging sweep never converges
                T.vhat[e] = vn;
                vv = vn;
                for (int l2 = 0; l2 < kMaxScen; ++l2)
                    if (l2 == l) mx[l2] = fmax(mx[l2], dd);
            }
            set_load_current(e, l, p, v, vv);
        }
        for (int l = 0; l < L; ++l) {
            double m = mx[0];
            if (l == 1) m = mx[1];
            if (l == 2) m = mx[2];
            if (l == 3) m = mx[3];
            for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            if ((tid & 31) == 0 && m > 0.0)
                atomicMax((unsigned long long *)&red[(it % 3) * L + l], (unsigned long long)__double_as_longlong(m));
        }
        if (!pf_grid_sync(bar, err, G, epoch, max_spins)) return;
        conv_all = true;
        __syncthreads();
        if (tid < L && s_live[tid]) {
            const double m = __longlong_as_double((long long)__ldcg((const unsigned long long *)&red[(it % 3) * L + tid]));
            if (m < tol2) {
                s_live[tid] = 0;
                if (blockIdx.x == 0) iters[tid] = it;
            }
        }
        __syncthreads();
        for (int l = 0; l < L; ++l) conv_all = conv_all && !s_live[l];
        if (conv_all) break;
    }
    if (blockIdx.x == 0 && tid < L && s_live[tid]) {
        iters[tid] = -1;
        atomicCAS(err, 0, 3);
    }
}

// Blocks of the cooperative load flow: enough for the grid-wide stages, at
// least one per (scenario, phase), at most one per SM.
cudaError_t launch_power_flow(int n, int L, Topo T, const double *s_in, double tol, int max_iter, double2 *J,
                              double2 *W, double *red, int *iters, int *err, int num_sms, cudaStream_t st,
                              long long max_spins) {
    int G = (int)(((size_t)3 * L * n + 127) / 128);
    if (G < 3 * L) G = 3 * L;
    if (G > num_sms) G = num_sms;
    const size_t smem = n <= kPfShared ? sizeof(double2) * (size_t)n : 0;
    unsigned *bar = reinterpret_cast<unsigned *>(red + 3 * L);
    cudaError_t e = cudaMemsetAsync(red, 0, sizeof(double) * (3 * L + 1), st);
    if (e != cudaSuccess) return e;
    void *args[] = {&n, &L, &T, &s_in, &tol, &max_iter, &J, &W, &red, &bar, &iters, &err, &max_spins};
    return cudaLaunchCooperativeKernel((const void *)k_power_flow, dim3(G), dim3(256), args, smem, st);
}

// Ihat = Y Vhat line by line: line current J_k = y_k (V_parent - V_k) on the
// phases of k; injection I_k = sum of children's J - J_k.  Also |Vhat|.
__device__ void dev_line_currents(int n, int L, Topo T, double2 *J, size_t first, size_t stride) {
    size_t tot = (size_t)L * n;
    for (size_t e = first; e < tot; e += stride) {
        int l = (int)(e / n), v = (int)(e % n);
        for (int p = 0; p < 3; ++p) {
            double2 j = make_double2(0.0, 0.0);
            if (v > 0 && (T.ph[v] >> p & 1u)) {
                int par = T.parent[v];
                for (int q = 0; q < 3; ++q)
                    if (T.ph[v] >> q & 1u)
                        j = cadd(j, cmul(T.yl[(size_t)v * 9 + p * 3 + q], csub(T.vhat[sidx(l, q, par, n)], T.vhat[sidx(l, q, v, n)])));
            }
            J[sidx(l, p, v, n)] = j;
            double2 vv = T.vhat[sidx(l, p, v, n)];
            T.amag[sidx(l, p, v, n)] = (T.ph[v] >> p & 1u) ? cmag(vv) : 0.0;
        }
    }
}

__global__ void k_line_currents(int n, int L, Topo T, double2 *J) {
    dev_line_currents(n, L, T, J, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

__device__ void dev_injections(int n, int L, Topo T, const double2 *__restrict__ J, size_t first, size_t stride) {
    size_t tot = (size_t)L * n;
    for (size_t e = first; e < tot; e += stride) {
        int l = (int)(e / n), v = (int)(e % n);
        for (int p = 0; p < 3; ++p) {
            double2 s = make_double2(0.0, 0.0);
            for (int c = T.child_off[v]; c < T.child_off[v + 1]; ++c) s = cadd(s, J[sidx(l, p, T.child[c], n)]);
            T.ihat[sidx(l, p, v, n)] = csub(s, J[sidx(l, p, v, n)]);
        }
    }
}

__global__ void k_injections(int n, int L, Topo T, const double2 *__restrict__ J) {
    dev_injections(n, L, T, J, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

// Caller-supplied scenario library (host layout [L][n][3][2], caller numbering).
__global__ void k_import_ops(int n, int L, Topo T, const double *__restrict__ vh, const double *__restrict__ ih) {
    size_t tot = (size_t)L * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        int l = (int)(e / n), v = (int)(e % n);
        int i = T.orig[v];
        for (int p = 0; p < 3; ++p) {
            size_t src = (((size_t)l * n + i) * 3 + p) * 2;
            bool on = T.ph[v] >> p & 1u;
            double2 vv = on ? make_double2(vh[src], vh[src + 1]) : make_double2(0.0, 0.0);
            T.vhat[sidx(l, p, v, n)] = vv;
            T.ihat[sidx(l, p, v, n)] = on ? make_double2(ih[src], ih[src + 1]) : make_double2(0.0, 0.0);
            T.amag[sidx(l, p, v, n)] = on ? cmag(vv) : 0.0;
        }
    }
}

// Initial state of Algorithm 1: every bus is its own super-node, I = Ihat,
// V = Vhat, cluster extremes = |Vhat|, MICE = 0.
__device__ void dev_state_init(int n, int L, Topo T, State S, size_t first, size_t stride) {
    size_t tot = (size_t)L * n;
    for (size_t e = first; e < tot; e += stride) {
        int l = (int)(e / n), v = (int)(e % n);
        if (l == 0) {
            S.label[v] = v;
            S.top[v] = v;
            S.ptop[v] = T.parent[v];
            S.sn_list[0][v] = v;
            S.sn_rank[v] = v;
            if (v == n - 1) S.sn_rank[n] = n;
        }
        S.mice[(size_t)l * n + v] = 0.0;
        S.mice32[(size_t)l * n + v] = 0.0f;
        for (int p = 0; p < 3; ++p) {
            size_t q = sidx(l, p, v, n);
            bool on = T.ph[v] >> p & 1u;
            S.vcur[q] = T.vhat[q];
            S.icur[q] = T.ihat[q];
            S.hi[q] = on ? T.amag[q] : -INFINITY;
            S.lo[q] = on ? T.amag[q] : INFINITY;
            S.mcur[q] = T.amag[q];
            S.v32[q] = make_float2((float)T.vhat[q].x, (float)T.vhat[q].y);
            S.hr32[q] = 0.0f;
            S.lr32[q] = 0.0f;
            S.icur32[q] = make_float2((float)T.ihat[q].x, (float)T.ihat[q].y);
        }
    }
}

__global__ void k_state_init(int n, int L, Topo T, State S) {
    dev_state_init(n, L, T, S, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

}  // namespace okr

namespace okr {

// ---------------------------------------------------------------- many feeders
// Load flow of one scenario by one CTA (the batch runs many such CTAs side by
// side, which spreads the FP64 arithmetic over the SMs): the same sweep,
// operation for operation, as k_power_flow.
__device__ void dev_power_flow_cta(int n, int l, const Topo &T, const double *__restrict__ s_in, double tol,
                                   int max_iter, double2 *J, int *iters, int *err) {
    const int tid = threadIdx.x, nt = blockDim.x;
    double2 *V = T.vhat;
    double2 *Jl = J + (size_t)l * 3 * n;
    __shared__ double s_red[32];
    __shared__ int s_conv;
    for (int v = tid; v < n; v += nt)
        for (int p = 0; p < 3; ++p)
            V[sidx(l, p, v, n)] = (T.ph[v] >> p & 1u) ? T.vslack[p] : make_double2(0.0, 0.0);
    __syncthreads();
    const int maxd = T.maxd[0];
    const double tol2 = tol * tol;                  // the test is max |dV|^2 < tol^2
    int it;
    bool conv = false;
    for (it = 1; it <= max_iter; ++it) {
        for (int d = maxd; d >= 1; --d) {
            for (int x = T.level_off[d] + tid; x < T.level_off[d + 1]; x += nt) {
                const int v = T.level_bus[x], i = T.orig[v];
                for (int p = 0; p < 3; ++p) {
                    double2 j = make_double2(0.0, 0.0);
                    if (T.ph[v] >> p & 1u) {
                        const size_t o = (((size_t)l * n + i) * 3 + p) * 2;
                        j = load_current(make_double2(s_in[o], s_in[o + 1]), V[sidx(l, p, v, n)]);
                    }
                    for (int c = T.child_off[v]; c < T.child_off[v + 1]; ++c) j = cadd(j, Jl[(size_t)p * n + T.child[c]]);
                    Jl[(size_t)p * n + v] = j;
                }
            }
            __syncthreads();
        }
        double dmax = 0.0;
        for (int d = 1; d <= maxd; ++d) {
            for (int x = T.level_off[d] + tid; x < T.level_off[d + 1]; x += nt) {
                const int v = T.level_bus[x], par = T.parent[v];
                for (int p = 0; p < 3; ++p) {
                    if (!(T.ph[v] >> p & 1u)) continue;
                    double2 drop = make_double2(0.0, 0.0);
                    for (int q = 0; q < 3; ++q)
                        if (T.ph[v] >> q & 1u) drop = cadd(drop, cmul(T.zl[(size_t)v * 9 + p * 3 + q], Jl[(size_t)q * n + v]));
                    const double2 vn = csub(V[sidx(l, p, par, n)], drop);
                    double dd = cmag2(csub(vn, V[sidx(l, p, v, n)]));   // squared change
                    if (!isfinite(dd)) dd = INFINITY;
                    dmax = fmax(dmax, dd);
                    V[sidx(l, p, v, n)] = vn;
                }
            }
            __syncthreads();
        }
        for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        if ((tid & 31) == 0) s_red[tid >> 5] = dmax;
        __syncthreads();
        if (tid == 0) {
            double m = 0.0;
            for (int w = 0; w < (nt + 31) / 32; ++w) m = fmax(m, s_red[w]);
            s_conv = (m < tol2);
        }
        __syncthreads();
        if (s_conv) { conv = true; break; }
    }
    if (tid == 0) {
        iters[l] = conv ? it : -1;
        if (!conv) atomicCAS(err, 0, 3);
    }
}

// Per feeder, one CTA: validation and renumbering, children, sparse table,
// line inverses, path impedances.
__global__ void __launch_bounds__(1024) k_batch_prep(const BatchSetup *bs) {
    __shared__ BatchSetup b;
    if (threadIdx.x == 0) b = bs[blockIdx.x];
    __syncthreads();
    dev_topology(b.n, b.parent_in, b.ph_in, b.T, b.dep, b.anc, b.anc2, b.d2, b.size, b.ccount, b.coff_c, b.child_c,
                 b.err);
    __syncthreads();
    if (*(volatile int *)b.err) return;
    dev_child_offsets(b.n, b.T, b.coff_c, b.child_c);
    __syncthreads();
    dev_rmq_all(b.n, b.nlev, b.T.depth, b.rmq);
    dev_line_inverses(b.n, b.T, b.z_in, b.err, threadIdx.x, blockDim.x);
    __syncthreads();
    dev_path_impedance(b.n, b.T);
}

// LCA tables: blockIdx.y = feeder.
__global__ void k_batch_lca(const BatchSetup *bs) {
    const BatchSetup &b = bs[blockIdx.y];
    if (*(volatile int *)b.err == 1) return;
    dev_lca_fill(b.n, b.T.parent, b.T.sz, b.T.depth, b.rmq, b.T.lca, (size_t)blockIdx.x * blockDim.x + threadIdx.x,
                 (size_t)gridDim.x * blockDim.x);
}

// Load flow: blockIdx.y = feeder, blockIdx.x = scenario.
__global__ void __launch_bounds__(256) k_batch_pf(const BatchSetup *bs, double tol, int max_iter) {
    __shared__ BatchSetup b;
    if (threadIdx.x == 0) b = bs[blockIdx.y];
    __syncthreads();
    if ((int)blockIdx.x >= b.L || *(volatile int *)b.err == 1) return;
    dev_power_flow_cta(b.n, blockIdx.x, b.T, b.s_in, tol, max_iter, b.J, b.pf_iters, b.err);
}

// Per feeder, one CTA: Ihat = Y Vhat, |Vhat|, the initial search state and the
// zeroed per-run counters of the search.
__global__ void __launch_bounds__(1024) k_batch_finish(const BatchSetup *bs) {
    __shared__ BatchSetup b;
    if (threadIdx.x == 0) b = bs[blockIdx.x];
    __syncthreads();
    if (*(volatile int *)b.err) return;
    const size_t first = threadIdx.x, stride = blockDim.x;
    dev_line_currents(b.n, b.L, b.T, b.J, first, stride);
    __syncthreads();
    dev_injections(b.n, b.L, b.T, b.J, first, stride);
    __syncthreads();
    dev_state_init(b.n, b.L, b.T, b.S, first, stride);
    for (int i = threadIdx.x; i < b.n; i += blockDim.x) {
        b.dec_maxerr[i] = 0.0;
        b.mrank[i] = 0.0;
        b.arrive[2 * i] = 0;
        b.arrive[2 * i + 1] = 0;
    }
    for (int i = threadIdx.x; i < b.n / 32 + 2; i += blockDim.x) b.bmax[i] = 0.0;
}

cudaError_t launch_batch_setup(int nf, int max_L, long long max_nn, const BatchSetup *bs, double tol, int max_iter,
                               int num_sms, cudaStream_t st, cudaStream_t side, cudaEvent_t ev_fork,
                               cudaEvent_t ev_join) {
    if (nf <= 0) return cudaSuccess;
    k_batch_prep<<<nf, 1024, 0, st>>>(bs);
    // the LCA tables (integer work, read only by the searches) on the side
    // stream beside the load flows (FP64 work)
    cudaError_t e = cudaEventRecord(ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_fork, 0);
    if (e != cudaSuccess) return e;
    long long bx = (max_nn + 255) / 256;
    if (bx > num_sms * 2) bx = num_sms * 2;
    if (bx < 1) bx = 1;
    k_batch_lca<<<dim3((unsigned)bx, nf), 256, 0, side>>>(bs);
    e = cudaEventRecord(ev_join, side);
    if (e != cudaSuccess) return e;
    // 256 threads: every (feeder, scenario) CTA resident at once, so that the
    // SMs interleave many CTAs' level-by-level chains (1,024-thread CTAs ran
    // in waves: 4.0 -> 3.2 ms for 256 feeders)
    k_batch_pf<<<dim3(max_L, nf), 256, 0, st>>>(bs, tol, max_iter);
    k_batch_finish<<<nf, 1024, 0, st>>>(bs);
    e = cudaStreamWaitEvent(st, ev_join, 0);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace okr

namespace okr {

// ---------------------------------------------------------------- a given reduced network
// The reduced network of a caller assignment, for the scenarios of T (Algorithm 1's
// solve with the aggregated injections, eq. i_agg): every super-node takes the
// injections of its members (members listed per super-node in increasing caller
// id, so the sums are deterministic), the tree is solved with those injections
// and the slack fixed, every bus takes its super-node's voltage, and the largest
// per-phase magnitude error against Vhat is reported.  One CTA per scenario.
//   moff/mem: members of each super-node (caller ids), CSR over caller ids.
//   sup: [n] super-node of each bus (caller ids).  W: [L*3n] work (injections, then
//   line currents), V: [L*3n] work (voltages).  vred: [L][n][3][2] (may be null).
__global__ void __launch_bounds__(1024) k_eval_reduced(Topo T, const int *__restrict__ sup, const int *__restrict__ moff,
                                                      const int *__restrict__ mem, double2 *W, double2 *V, double *vred,
                                                      double *err) {
    const int n = T.n, l = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    double2 *Wl = W + (size_t)l * 3 * n, *Vl = V + (size_t)l * 3 * n;
    __shared__ double s_red[32];
    // aggregated injections at the super-nodes (preorder), zero elsewhere
    for (int e = tid; e < 3 * n; e += nt) {
        const int p = e / n, v = e % n, i = T.orig[v];
        double2 acc = make_double2(0.0, 0.0);
        for (int x = moff[i]; x < moff[i + 1]; ++x) {
            const int u = T.pre[mem[x]];
            if (T.ph[u] >> p & 1u) acc = cadd(acc, T.ihat[sidx(l, p, u, n)]);
        }
        Wl[e] = acc;
    }
    __syncthreads();
    // line currents J_v = -I_v + sum of the children's J, deepest level first
    const int maxd = T.maxd[0];
    for (int d = maxd; d >= 1; --d) {
        for (int x = T.level_off[d] + tid; x < T.level_off[d + 1]; x += nt) {
            const int v = T.level_bus[x];
            for (int p = 0; p < 3; ++p) {
                double2 j = make_double2(-Wl[(size_t)p * n + v].x, -Wl[(size_t)p * n + v].y);
                for (int c = T.child_off[v]; c < T.child_off[v + 1]; ++c) j = cadd(j, Wl[(size_t)p * n + T.child[c]]);
                Wl[(size_t)p * n + v] = j;
            }
        }
        __syncthreads();
    }
    // voltages, top down: V_v = V_parent - z_v J_v on the phases of v
    for (int e = tid; e < 3; e += nt) Vl[(size_t)e * n] = (T.ph[0] >> e & 1u) ? T.vslack[e] : make_double2(0.0, 0.0);
    __syncthreads();
    for (int d = 1; d <= maxd; ++d) {
        for (int x = T.level_off[d] + tid; x < T.level_off[d + 1]; x += nt) {
            const int v = T.level_bus[x], par = T.parent[v];
            for (int p = 0; p < 3; ++p) {
                double2 vv = make_double2(0.0, 0.0);
                if (T.ph[v] >> p & 1u) {
                    double2 drop = make_double2(0.0, 0.0);
                    for (int q = 0; q < 3; ++q)
                        if (T.ph[v] >> q & 1u) drop = cadd(drop, cmul(T.zl[(size_t)v * 9 + p * 3 + q], Wl[(size_t)q * n + v]));
                    vv = csub(Vl[(size_t)p * n + par], drop);
                }
                Vl[(size_t)p * n + v] = vv;
            }
        }
        __syncthreads();
    }
    // every bus at its super-node's voltage; largest magnitude error
    double m = 0.0;
    for (int e = tid; e < 3 * n; e += nt) {
        const int p = e / n, i = e % n;
        const int v = T.pre[i], s = T.pre[sup[i]];
        const bool on = T.ph[v] >> p & 1u;
        const double2 vr = on ? Vl[(size_t)p * n + s] : make_double2(0.0, 0.0);
        if (on) m = fmax(m, fabs(T.amag[sidx(l, p, v, n)] - cmag(vr)));
        if (vred) {
            const size_t o = (((size_t)l * n + i) * 3 + p) * 2;
            vred[o] = vr.x;
            vred[o + 1] = vr.y;
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) s_red[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
        double r = 0.0;
        for (int w = 0; w < (nt + 31) / 32; ++w) r = fmax(r, s_red[w]);
        err[l] = r;
    }
}

}  // namespace okr
