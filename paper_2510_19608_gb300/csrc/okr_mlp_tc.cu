// okr_mlp_tc.cu -- the learned scorer's forward pass on the 5th-generation
// tensor cores (tcgen05): inference for many candidates at once.
//
// One CTA per SM, four warpgroups of 128 threads; each warpgroup carries its
// own stream of tiles of 128 samples through the network, so that while one
// warpgroup runs its epilogue the others' products keep the tensor core busy.
// The weights sit once in shared memory (W2, W3, W1: 68 KB); each warpgroup
// has its own input buffers (36 KB) and 128 of the SM's 512 tensor-memory
// columns.  Thread m of a warpgroup owns sample m of its tile.  A hidden layer is one 128 x 128 x K
// product D = A B (A: the tile's inputs, M = 128 samples x K; B: the layer's
// weights, K x N = 128 units), issued by one thread as K / 16 tcgen05.mma
// instructions of kind::f16 with bfloat16 operands and FP32 accumulators in
// tensor memory (128 lanes x 128 columns).  Operands are staged in shared
// memory in the no-swizzle K-major layout: 8 x 8 core matrices of 16-byte rows,
// consecutive along M (stride 128 B, the descriptor's "stride" offset) and
// then along K (stride ROWS/8 x 128 B, its "leading" offset).  When the
// products are done (tcgen05.commit arrives on an mbarrier), each thread reads
// its own row of the accumulators back with tcgen05.ld, adds the bias, applies
// the ReLU and writes the row, rounded to bfloat16, as the next layer's input.
// The output layer (128 -> 1) is a per-thread dot product in FP32.
//
// Numerics: weights are the bfloat16 copies of the FP32 master weights (as in
// k_mlp_forward), and so are the layers' inputs here (the features and the
// hidden activations), because both operands of a kind::f16 product are
// bfloat16; products and sums are FP32.  The training kernels keep FP32
// activations; this path is for ranking many candidates.
//
// Every wait on the mbarrier is bounded; a wait that gives up sets the error
// flag, the CTA waits (again bounded) for its products in flight, frees its
// tensor memory and returns.
#include "okr_internal.cuh"
#include "okr_kernels.cuh"

#include <cuda_bf16.h>

namespace okr {

namespace {

constexpr int kH = kMlpHidden;          // 128 units per hidden layer = tile rows = N
constexpr int kRegion = kH * kH * 2;    // bytes of a 128 x 128 bf16 operand
constexpr int kRegion16 = kH * 16 * 2;  // bytes of a 128 x 16 bf16 operand (the features, W1)
constexpr int kGroups = 4;              // warpgroups per CTA, each with its own stream of tiles
constexpr int kThreads = kGroups * kH;
constexpr long long kMbarSpins = 1 << 22;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, k) of a [128 rows] x [K] bf16 operand in the
// no-swizzle K-major core-matrix layout.
__device__ __forceinline__ unsigned core_off(int row, int k) {
    return (unsigned)((((k >> 3) * (kH / 8)) + (row >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K) and
// stride (M/N) byte offsets in 16-byte units, version 1, no swizzle.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D FP32, A and B bfloat16, both K-major,
// N = 128, M = 128.
constexpr unsigned kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kH >> 3) << 17) | ((unsigned)(128 >> 4) << 24);

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                         unsigned accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(unsigned mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// Bounded wait for phase `parity` of the mbarrier; false when it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity) {
    for (long long i = 0; i < kMbarSpins; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 consecutive FP32 accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float *v) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Two FP32 values to a bfloat16 pair (nearest even), negative values to zero
// (the ReLU folded into the conversion; rounding keeps the sign, so this is
// the rounded ReLU).  The first value goes to the lower half.
__device__ __forceinline__ unsigned relu_bf16x2(float lo, float hi) {
    unsigned d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Eight consecutive K elements (k0 a multiple of 8) of row `row`, rounded to
// bfloat16 (nearest even), as one 16-byte row of a core matrix.
__device__ __forceinline__ void store8_bf16(unsigned char *base, int row, int k0, const float *v) {
    uint4 q;
    unsigned *w = reinterpret_cast<unsigned *>(&q);
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);   // .x (lower address) = v[2j]
        w[j] = *reinterpret_cast<const unsigned *>(&p);
    }
    *reinterpret_cast<uint4 *>(base + core_off(row, k0)) = q;
}

// Barrier of the 128 threads of warpgroup g (named barrier 1 + g).
__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kH) : "memory");
}

// Barrier of warpgroup g that returns whether any of its threads passed `pred`.
__device__ __forceinline__ bool group_or(int g, bool pred) {
    unsigned out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(out)
        : "r"((unsigned)pred), "r"(1 + g), "r"(kH)
        : "memory");
    return out != 0;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace

// y[i] for samples i < N of x [N][F] (F <= 16), weights from theta (biases,
// b4) and the bfloat16 copies w1..w4.  err: set to 1 when a wait gave up.
__global__ void __launch_bounds__(kThreads, 1) k_mlp_forward_tc(const float *__restrict__ x, int N, int F,
                                                                const float *__restrict__ theta,
                                                                const __nv_bfloat16 *__restrict__ w1,
                                                                const __nv_bfloat16 *__restrict__ w2,
                                                                const __nv_bfloat16 *__restrict__ w3,
                                                                const __nv_bfloat16 *__restrict__ w4, float *y,
                                                                int *err) {
    extern __shared__ __align__(1024) unsigned char tc_sm[];
    // shared: W2, W3, W1; then per warpgroup its hidden input and its features
    unsigned char *sW2 = tc_sm, *sW3 = tc_sm + kRegion, *sW1 = tc_sm + 2 * kRegion;
    __shared__ __align__(16) float sb[3][kH];
    __shared__ __align__(16) float sw4[kH];
    __shared__ __align__(8) unsigned long long mbar[kGroups];
    __shared__ unsigned tmem_holder;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid / kH, row = tid % kH;             // warpgroup, and the tile row this thread owns
    unsigned char *sA = tc_sm + 2 * kRegion + kRegion16 + g * (kRegion + kRegion16);
    unsigned char *sX = sA + kRegion;
    // parameter offsets (as offsets() in okr_mlp.cu): b1, b2, b3, b4
    const int B1off = F * kH, B2off = B1off + kH + kH * kH, B3off = B2off + kH + kH * kH, B4off = B3off + 2 * kH;
    // weights into shared memory as B operands: element (n, k) = W[k][n]
    for (int e = tid; e < kH * kH; e += kThreads) {
        const int k = e / kH, n = e % kH;
        *reinterpret_cast<__nv_bfloat16 *>(sW2 + core_off(n, k)) = w2[e];
        *reinterpret_cast<__nv_bfloat16 *>(sW3 + core_off(n, k)) = w3[e];
    }
    for (int e = tid; e < 16 * kH; e += kThreads) {
        const int k = e / kH, n = e % kH;
        *reinterpret_cast<__nv_bfloat16 *>(sW1 + core_off(n, k)) = k < F ? w1[k * kH + n] : __float2bfloat16_rn(0.0f);
    }
    if (tid < kH) {
        sb[0][tid] = theta[B1off + tid];
        sb[1][tid] = theta[B2off + tid];
        sb[2][tid] = theta[B3off + tid];
        sw4[tid] = __bfloat162float(w4[tid]);
    }
    const float b4 = theta[B4off];
    if (tid < kGroups) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[tid])), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(kGroups * kH)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    // this warpgroup's accumulators: columns [128 g, 128 g + 128); a warp reads
    // the 32 lanes of its rank within the warpgroup
    const unsigned tmem_g = tmem_holder + (unsigned)(g * kH);
    const unsigned taddr = tmem_g + ((unsigned)((warp & 3) * 32) << 16);
    const unsigned mb = smem_u32(&mbar[g]);
    const bool issuer = row == 0;
    unsigned phase = 0;
    bool ok = true;                         // uniform within the warpgroup

    // descriptors: K = 16 per instruction, i.e. two core matrices along K
    const unsigned lbo = (kH / 8) * 128, sbo = 128;
    auto layer = [&](unsigned char *a, unsigned char *b, int ksteps) -> bool {
        if (issuer) {
            fence_after();
            for (int s = 0; s < ksteps; ++s) {
                const unsigned off = (unsigned)s * 2 * lbo;
                mma_bf16(tmem_g, smem_desc(smem_u32(a) + off, lbo, sbo), smem_desc(smem_u32(b) + off, lbo, sbo),
                         s > 0 ? 1u : 0u);
            }
            mma_commit(mb);
        }
        const bool got = mbar_wait(mb, phase);
        phase ^= 1u;
        if (group_or(g, !got)) return false;        // the same decision in every thread of the group
        fence_after();
        return true;
    };
    // this thread's accumulator row + bias, ReLU, as the next layer's input
    // (bfloat16, K-major); the last layer returns the output instead
    auto epilogue = [&](int li, bool last) {
        float acc = 0.0f;
        for (int c = 0; c < kH; c += 32) {
            float v[32];
            tmem_ld32(taddr + (unsigned)c, v);
            for (int j = 0; j < 8; ++j) {
                const float4 b = *reinterpret_cast<const float4 *>(&sb[li][c + 4 * j]);
                v[4 * j] += b.x;
                v[4 * j + 1] += b.y;
                v[4 * j + 2] += b.z;
                v[4 * j + 3] += b.w;
            }
            if (last) {
                for (int j = 0; j < 8; ++j) {
                    const float4 w = *reinterpret_cast<const float4 *>(&sw4[c + 4 * j]);
                    acc = fmaf(fmaxf(v[4 * j], 0.0f), w.x, acc);
                    acc = fmaf(fmaxf(v[4 * j + 1], 0.0f), w.y, acc);
                    acc = fmaf(fmaxf(v[4 * j + 2], 0.0f), w.z, acc);
                    acc = fmaf(fmaxf(v[4 * j + 3], 0.0f), w.w, acc);
                }
            } else {
                for (int q = 0; q < 4; ++q) {
                    uint4 o;
                    o.x = relu_bf16x2(v[8 * q], v[8 * q + 1]);
                    o.y = relu_bf16x2(v[8 * q + 2], v[8 * q + 3]);
                    o.z = relu_bf16x2(v[8 * q + 4], v[8 * q + 5]);
                    o.w = relu_bf16x2(v[8 * q + 6], v[8 * q + 7]);
                    *reinterpret_cast<uint4 *>(sA + core_off(row, c + 8 * q)) = o;
                }
            }
        }
        return acc;
    };
    // the features of tile t, row `row`, as FP32 (zero past N and past F)
    auto load_x = [&](long long t, float *v) {
        const long long m = t * kH + row;
        for (int k = 0; k < 16; ++k) v[k] = (m < N && k < F) ? x[m * F + k] : 0.0f;
    };
    auto sync_group = [&]() {
        fence_async_smem();
        fence_before();
        group_sync(g);
    };

    const long long tiles = ((long long)N + kH - 1) / kH, stride = (long long)gridDim.x * kGroups;
    long long t = (long long)blockIdx.x * kGroups + g;
    float v[16];
    if (t < tiles) load_x(t, v);
    for (; t < tiles && ok; t += stride) {
        store8_bf16(sX, row, 0, v);
        store8_bf16(sX, row, 8, v + 8);
        if (t + stride < tiles) load_x(t + stride, v);  // in flight while this tile's products run
        sync_group();
        ok = layer(sX, sW1, 1);
        if (!ok) break;
        epilogue(0, false);
        sync_group();
        ok = layer(sA, sW2, kH / 16);
        if (!ok) break;
        // every thread has read its accumulators before sA is overwritten:
        // the epilogue reads tensor memory only after the product that read sA is done
        epilogue(1, false);
        sync_group();
        ok = layer(sA, sW3, kH / 16);
        if (!ok) break;
        const float out = epilogue(2, true);
        const long long m = t * kH + row;
        if (m < N) y[m] = out + b4;
        fence_before();
        group_sync(g);
    }
    if (!ok && issuer) {
        atomicExch(err, 1);
        mbar_wait(mb, phase ^ 1u);          // the products in flight (the phase that gave up), bounded
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_holder), "r"(kGroups * kH)
                     : "memory");
}

size_t mlp_forward_tc_smem() { return 2 * (size_t)kRegion + kRegion16 + kGroups * (size_t)(kRegion + kRegion16); }

cudaError_t mlp_forward_tc(const MlpBufs &b, const float *x, int N, float *y, int *err, int num_sms, cudaStream_t st) {
    const size_t smem = mlp_forward_tc_smem();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long tiles = ((long long)N + kH - 1) / kH, groups = (tiles + kGroups - 1) / kGroups;
    const int grid = groups < num_sms ? (int)groups : num_sms;
    k_mlp_forward_tc<<<grid, kThreads, smem, st>>>(x, N, b.F, b.theta, b.w1, b.w2, b.w3, b.w4, y, err);
    return cudaGetLastError();
}

}  // namespace okr
