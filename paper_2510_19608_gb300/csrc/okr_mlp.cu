// okr_mlp.cu -- the learned candidate scorer: a three-hidden-layer perceptron
// (128 units, ReLU) that predicts a candidate's normalised score change from
// local feeder features, with hand-written forward, backward and Adam kernels.
//
// Numerics: weights are held in FP32 (the Adam master copy) and used as
// bfloat16 copies in every product; products are accumulated in FP32 in a
// fixed order, and every reduction over samples is deterministic (fixed
// segments summed in a fixed order), so that training is reproducible.
//
// Parameter vector (FP32), in this order: W1 (F x H, row-major), b1 (H),
// W2 (H x H), b2, W3 (H x H), b3, w4 (H), b4 (1).
//
// The layers are 128 wide and the feature vector at most 16 long, so the
// products are small: one CTA of 128 threads (one per unit) carries a tile of
// 32 samples through all layers with the weights resident in shared memory.
#include "okr_internal.cuh"
#include "okr_kernels.cuh"

#include <cuda_bf16.h>

namespace okr {

namespace {

constexpr int kH = kMlpHidden;
constexpr int kTile = 32;                    // samples per CTA tile
constexpr int kSeg = 2048;                   // samples per partial sum of a weight gradient

struct Off {
    int w1, b1, w2, b2, w3, b3, w4, b4, total;
};

__host__ __device__ inline Off offsets(int F) {
    Off o;
    o.w1 = 0;
    o.b1 = o.w1 + F * kH;
    o.w2 = o.b1 + kH;
    o.b2 = o.w2 + kH * kH;
    o.w3 = o.b2 + kH;
    o.b3 = o.w3 + kH * kH;
    o.w4 = o.b3 + kH;
    o.b4 = o.w4 + kH;
    o.total = o.b4 + 1;
    return o;
}

}  // namespace

int mlp_param_count(int F) { return offsets(F).total; }

// FP32 master weights -> bfloat16 copies used by the products.
__global__ void k_mlp_to_bf16(const float *theta, int F, __nv_bfloat16 *w1, __nv_bfloat16 *w2, __nv_bfloat16 *w3,
                              __nv_bfloat16 *w4) {
    const Off o = offsets(F);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kH * kH; e += gridDim.x * blockDim.x) {
        w2[e] = __float2bfloat16_rn(theta[o.w2 + e]);
        w3[e] = __float2bfloat16_rn(theta[o.w3 + e]);
        if (e < F * kH) w1[e] = __float2bfloat16_rn(theta[o.w1 + e]);
        if (e < kH) w4[e] = __float2bfloat16_rn(theta[o.w4 + e]);
    }
}

// Forward pass.  x: [N][F]; optional outputs h1, h2, h3: [N][H] (post-ReLU), y: [N].
__global__ void __launch_bounds__(kH) k_mlp_forward(const float *__restrict__ x, int N, int F,
                                                    const float *__restrict__ theta, const __nv_bfloat16 *__restrict__ w1,
                                                    const __nv_bfloat16 *__restrict__ w2,
                                                    const __nv_bfloat16 *__restrict__ w3,
                                                    const __nv_bfloat16 *__restrict__ w4, float *h1, float *h2,
                                                    float *h3, float *y) {
    extern __shared__ unsigned char mlp_sm[];
    __nv_bfloat16 *W2 = reinterpret_cast<__nv_bfloat16 *>(mlp_sm);
    __nv_bfloat16 *W3 = W2 + kH * kH;
    __nv_bfloat16 *W1 = W3 + kH * kH;                       // [kMlpMaxF][H]
    float *A = reinterpret_cast<float *>(W1 + kMlpMaxF * kH);  // [kTile][H]
    float *B = A + kTile * kH;
    float *xs = B + kTile * kH;                               // [kTile][kMlpMaxF]
    const int j = threadIdx.x;
    const Off o = offsets(F);
    for (int e = j; e < kH * kH; e += kH) {
        W2[e] = w2[e];
        W3[e] = w3[e];
    }
    for (int e = j; e < F * kH; e += kH) W1[e] = w1[e];
    const float bj1 = theta[o.b1 + j], bj2 = theta[o.b2 + j], bj3 = theta[o.b3 + j];
    const float w4j = __bfloat162float(w4[j]), b4 = theta[o.b4];
    __syncthreads();
    for (int base = blockIdx.x * kTile; base < N; base += gridDim.x * kTile) {
        const int S = min(kTile, N - base);
        for (int e = j; e < kTile * F; e += kH) {
            const int s = e / F, k = e % F;
            xs[s * kMlpMaxF + k] = s < S ? x[(size_t)(base + s) * F + k] : 0.0f;
        }
        __syncthreads();
        for (int s = 0; s < kTile; ++s) {
            float z = bj1;
            for (int k = 0; k < F; ++k) z = fmaf(xs[s * kMlpMaxF + k], __bfloat162float(W1[k * kH + j]), z);
            A[s * kH + j] = fmaxf(z, 0.0f);
        }
        __syncthreads();
        for (int s = 0; s < kTile; ++s) {
            float z = bj2;
            for (int k = 0; k < kH; ++k) z = fmaf(A[s * kH + k], __bfloat162float(W2[k * kH + j]), z);
            B[s * kH + j] = fmaxf(z, 0.0f);
        }
        __syncthreads();
        for (int s = 0; s < kTile; ++s) {
            float z = bj3;
            for (int k = 0; k < kH; ++k) z = fmaf(B[s * kH + k], __bfloat162float(W3[k * kH + j]), z);
            const float h = fmaxf(z, 0.0f);
            if (s < S) {
                if (h1) h1[(size_t)(base + s) * kH + j] = A[s * kH + j];
                if (h2) h2[(size_t)(base + s) * kH + j] = B[s * kH + j];
                if (h3) h3[(size_t)(base + s) * kH + j] = h;
            }
            A[s * kH + j] = h * w4j;                            // the output layer's products
        }
        __syncthreads();
        // y = b4 + sum_j h3_j w4_j: warp w sums samples w, w + 4, ... over j in a fixed order
        const int lane = j & 31, warp = j >> 5;
        for (int s = warp; s < S; s += kH / 32) {
            float acc = A[s * kH + lane] + A[s * kH + lane + 32] + A[s * kH + lane + 64] + A[s * kH + lane + 96];
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) y[base + s] = acc + b4;
        }
        __syncthreads();
    }
}

// Backward through the activations.  dy = scale (y - t); d3 = dy w4 * [h3 > 0];
// d2 = (d3 W3^T) * [h2 > 0]; d1 = (d2 W2^T) * [h1 > 0].  All [N][H] except dy [N].
__global__ void __launch_bounds__(kH) k_mlp_backward(int N, const __nv_bfloat16 *__restrict__ w2,
                                                     const __nv_bfloat16 *__restrict__ w3,
                                                     const __nv_bfloat16 *__restrict__ w4, const float *__restrict__ h1,
                                                     const float *__restrict__ h2, const float *__restrict__ h3,
                                                     const float *__restrict__ y, const float *__restrict__ t,
                                                     float scale, float *d1, float *d2, float *d3, float *dy) {
    extern __shared__ unsigned char mlp_sm[];
    __nv_bfloat16 *W2T = reinterpret_cast<__nv_bfloat16 *>(mlp_sm);   // W2T[j][k] = W2[k][j]
    __nv_bfloat16 *W3T = W2T + kH * kH;
    float *D = reinterpret_cast<float *>(W3T + kH * kH);             // [kTile][H]
    float *E = D + kTile * kH;
    float *dys = E + kTile * kH;                                       // [kTile]
    const int j = threadIdx.x;
    for (int e = j; e < kH * kH; e += kH) {
        const int k = e / kH, c = e % kH;
        W2T[c * kH + k] = w2[e];
        W3T[c * kH + k] = w3[e];
    }
    const float w4j = __bfloat162float(w4[j]);
    __syncthreads();
    for (int base = blockIdx.x * kTile; base < N; base += gridDim.x * kTile) {
        const int S = min(kTile, N - base);
        if (j < kTile) dys[j] = j < S ? scale * (y[base + j] - t[base + j]) : 0.0f;
        __syncthreads();
        for (int s = 0; s < kTile; ++s) {
            const float h = s < S ? h3[(size_t)(base + s) * kH + j] : 0.0f;
            D[s * kH + j] = h > 0.0f ? dys[s] * w4j : 0.0f;
        }
        __syncthreads();
        for (int s = 0; s < kTile; ++s) {                               // d2, thread = unit k of layer 2
            float z = 0.0f;
            for (int c = 0; c < kH; ++c) z = fmaf(D[s * kH + c], __bfloat162float(W3T[c * kH + j]), z);
            const float h = s < S ? h2[(size_t)(base + s) * kH + j] : 0.0f;
            E[s * kH + j] = h > 0.0f ? z : 0.0f;
        }
        __syncthreads();
        for (int s = 0; s < S; ++s) {
            d3[(size_t)(base + s) * kH + j] = D[s * kH + j];
            d2[(size_t)(base + s) * kH + j] = E[s * kH + j];
        }
        for (int s = 0; s < kTile; ++s) {                               // d1
            float z = 0.0f;
            for (int c = 0; c < kH; ++c) z = fmaf(E[s * kH + c], __bfloat162float(W2T[c * kH + j]), z);
            const float h = s < S ? h1[(size_t)(base + s) * kH + j] : 0.0f;
            if (s < S) d1[(size_t)(base + s) * kH + j] = h > 0.0f ? z : 0.0f;
        }
        if (j < S) dy[base + j] = dys[j];
        __syncthreads();
    }
}

// Partial weight gradients over one segment of kSeg samples:
//   part[seg][k][c] = sum over the segment of A[n][k] * D[n][c]   (k < K, c < C)
// and, if with_bias, part[seg][K][c] = sum of D[n][c].  One thread per output, the
// samples in increasing order.
__global__ void k_mlp_wgrad_part(const float *__restrict__ A, int lda, int K, const float *__restrict__ D, int C,
                                 int N, int with_bias, float *part) {
    const int rows = K + (with_bias ? 1 : 0);
    const int seg = blockIdx.y;
    const int n0 = seg * kSeg, n1 = min(N, n0 + kSeg);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * C; e += gridDim.x * blockDim.x) {
        const int k = e / C, c = e % C;
        float acc = 0.0f;
        if (k < K)
            for (int n = n0; n < n1; ++n) acc = fmaf(A[(size_t)n * lda + k], D[(size_t)n * C + c], acc);
        else
            for (int n = n0; n < n1; ++n) acc += D[(size_t)n * C + c];
        part[(size_t)seg * rows * C + e] = acc;
    }
}

// grad[e] = sum over segments (in order) of part[seg][e].
__global__ void k_mlp_sum_parts(const float *__restrict__ part, int nseg, int len, float *grad) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int s = 0; s < nseg; ++s) acc += part[(size_t)s * len + e];
        grad[e] = acc;
    }
}

// Adam (bias-corrected) on the FP32 master weights.
__global__ void k_mlp_adam(float *theta, const float *__restrict__ g, float *m, float *v, int P, float lr, float beta1,
                           float beta2, float eps, float c1, float c2) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P; e += gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = beta1 * m[e] + (1.0f - beta1) * ge;
        const float ve = beta2 * v[e] + (1.0f - beta2) * ge * ge;
        m[e] = me;
        v[e] = ve;
        theta[e] -= lr * (me / c1) / (sqrtf(ve / c2) + eps);
    }
}

// Squared error sums per segment (deterministic loss).
__global__ void k_mlp_sqerr_part(const float *__restrict__ y, const float *__restrict__ t, int N, float *part) {
    const int seg = blockIdx.x;
    const int n0 = seg * kSeg, n1 = min(N, n0 + kSeg);
    __shared__ float red[32];
    float acc = 0.0f;
    for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
        const float d = y[n] - t[n];
        acc = fmaf(d, d, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[seg] = s;
    }
}

// ---------------------------------------------------------------- host launches
size_t mlp_forward_smem() {
    return sizeof(__nv_bfloat16) * (2 * kH * kH + kMlpMaxF * kH) + sizeof(float) * (2 * kTile * kH + kTile * kMlpMaxF);
}

size_t mlp_backward_smem() { return sizeof(__nv_bfloat16) * 2 * kH * kH + sizeof(float) * (2 * kTile * kH + kTile); }

int mlp_segments(int N) { return (N + kSeg - 1) / kSeg; }

cudaError_t mlp_sync_bf16(const MlpBufs &b, cudaStream_t st) {
    k_mlp_to_bf16<<<64, 256, 0, st>>>(b.theta, b.F, b.w1, b.w2, b.w3, b.w4);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const MlpBufs &b, const float *x, int N, float *h1, float *h2, float *h3, float *y, int num_sms,
                        cudaStream_t st) {
    const size_t smem = mlp_forward_smem();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = (N + kTile - 1) / kTile;
    if (grid > num_sms * 2) grid = num_sms * 2;
    if (grid < 1) grid = 1;
    k_mlp_forward<<<grid, kH, smem, st>>>(x, N, b.F, b.theta, b.w1, b.w2, b.w3, b.w4, h1, h2, h3, y);
    return cudaGetLastError();
}

// Gradient of the mean squared error at the current weights into b.grad
// (uses the work buffers, which must hold N samples).
cudaError_t mlp_gradient(const MlpBufs &b, const MlpWork &w, const float *x, const float *t, int N, int num_sms,
                         cudaStream_t st) {
    cudaError_t e = mlp_forward(b, x, N, w.h1, w.h2, w.h3, w.y, num_sms, st);
    if (e != cudaSuccess) return e;
    const size_t smem = mlp_backward_smem();
    e = cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = (N + kTile - 1) / kTile;
    if (grid > num_sms * 2) grid = num_sms * 2;
    if (grid < 1) grid = 1;
    k_mlp_backward<<<grid, kH, smem, st>>>(N, b.w2, b.w3, b.w4, w.h1, w.h2, w.h3, w.y, t, 2.0f / (float)N, w.d1, w.d2,
                                           w.d3, w.dy);
    const Off o = offsets(b.F);
    const int nseg = mlp_segments(N);
    struct Job {
        const float *A;
        int lda, K;
        const float *D;
        int C, off;
    } jobs[4] = {{x, b.F, b.F, w.d1, kH, o.w1},
                 {w.h1, kH, kH, w.d2, kH, o.w2},
                 {w.h2, kH, kH, w.d3, kH, o.w3},
                 {w.h3, kH, kH, w.dy, 1, o.w4}};
    for (const Job &jb : jobs) {
        // weights and bias are adjacent in the parameter vector (W then b), except
        // for the output layer whose bias b4 follows w4: both come out in order
        const int rows = jb.K + 1;
        const int len = rows * jb.C;
        dim3 grid2((len + 255) / 256, nseg);
        k_mlp_wgrad_part<<<grid2, 256, 0, st>>>(jb.A, jb.lda, jb.K, jb.D, jb.C, N, 1, w.part);
        k_mlp_sum_parts<<<(len + 255) / 256, 256, 0, st>>>(w.part, nseg, len, b.grad + jb.off);
    }
    return cudaGetLastError();
}

cudaError_t mlp_adam(const MlpBufs &b, float lr, int step, cudaStream_t st) {
    const int P = offsets(b.F).total;
    const float beta1 = 0.9f, beta2 = 0.999f;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    k_mlp_adam<<<(P + 255) / 256, 256, 0, st>>>(b.theta, b.grad, b.m, b.v, P, lr, beta1, beta2, 1e-8f, c1, c2);
    return mlp_sync_bf16(b, st);
}

cudaError_t mlp_sqerr(const float *y, const float *t, int N, float *part, cudaStream_t st) {
    k_mlp_sqerr_part<<<mlp_segments(N), 256, 0, st>>>(y, t, N, part);
    return cudaGetLastError();
}

}  // namespace okr
