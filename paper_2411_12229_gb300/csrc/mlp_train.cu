// mlp_train.cu -- training kernels of the learned early stop (not in the
// paper): a 16 -> 64 -> 64 -> 1 ReLU MLP over search-state features,
// trained with weighted binary cross-entropy and Adam.
//
// One block takes a tile of 128 samples and runs the batch as small dense
// products in shared memory:
//   forward  A1 = X W1^T + b1, H1 = relu(A1), A2 = H1 W2^T + b2,
//            H2 = relu(A2), z = H2 W3 + b3
//   backward dz = w (sigmoid(z) - y) / sum(w), D2 = (dz W3^T) .* [A2 > 0],
//            D1 = (D2 W2) .* [A1 > 0]
//   grads    W3: H2^T dz, W2: D2^T H1, W1: D1^T X, biases: column sums
// and adds its partial gradient into the global gradient with atomics.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sqg.h"

namespace {

constexpr int kIn = SQG_MLP_IN, kH = SQG_MLP_HIDDEN, kTile = 128, kThreads = 256;
constexpr int oW1 = 0, ob1 = kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH, ob3 = oW3 + kH;

struct TileSmem {
    float W[SQG_MLP_NPARAM];
    float X[kTile][kIn];
    float A1[kTile][kH + 1];  // pre-activation, later D1
    float A2[kTile][kH + 1];  // pre-activation, later D2
    float H1[kTile][kH + 1];
    float dz[kTile];
    float lossp[kThreads / 32];
};

__device__ __forceinline__ float softplus(float z) { return z > 0.f ? z + log1pf(expf(-z)) : log1pf(expf(z)); }

// sum of the sample weights (one block)
__global__ void weight_sum_kernel(const float *w, int n, float *out) {
    __shared__ float part[kThreads / 32];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += w[i];
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < kThreads / 32; ++i) t += part[i];
        *out = t;
    }
}

__global__ void __launch_bounds__(kThreads) mlp_grad_kernel(const float *__restrict__ P, const float *__restrict__ X,
                                                            const float *__restrict__ y, const float *__restrict__ w,
                                                            int n, const float *__restrict__ wsum,
                                                            float *__restrict__ G, float *__restrict__ loss) {
    extern __shared__ __align__(16) unsigned char raw[];
    TileSmem &s = *reinterpret_cast<TileSmem *>(raw);
    const int tid = threadIdx.x, base = blockIdx.x * kTile;
    const int rows = min(kTile, n - base);
    for (int i = tid; i < SQG_MLP_NPARAM; i += kThreads) s.W[i] = P[i];
    for (int i = tid; i < kTile * kIn; i += kThreads) {
        int r = i / kIn, c = i % kIn;
        s.X[r][c] = r < rows ? X[(size_t)(base + r) * kIn + c] : 0.f;
    }
    __syncthreads();
    const float inv_w = 1.0f / *wsum;
    // A1 = X W1^T + b1
    for (int i = tid; i < kTile * kH; i += kThreads) {
        int r = i / kH, o = i % kH;
        float a = s.W[ob1 + o];
        for (int c = 0; c < kIn; ++c) a = fmaf(s.W[oW1 + o * kIn + c], s.X[r][c], a);
        s.A1[r][o] = a;
        s.H1[r][o] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    // A2 = H1 W2^T + b2
    for (int i = tid; i < kTile * kH; i += kThreads) {
        int r = i / kH, o = i % kH;
        float a = s.W[ob2 + o];
        for (int c = 0; c < kH; ++c) a = fmaf(s.W[oW2 + o * kH + c], s.H1[r][c], a);
        s.A2[r][o] = a;
    }
    __syncthreads();
    // z, loss, dz: one warp per 16 samples, lanes over the 64 hidden units
    {
        const int lane = tid & 31, wp = tid >> 5;
        float lsum = 0.f;
        for (int r = wp; r < kTile; r += kThreads / 32) {
            float a0 = s.A2[r][lane], a1 = s.A2[r][lane + 32];
            float p = s.W[oW3 + lane] * (a0 > 0.f ? a0 : 0.f) + s.W[oW3 + lane + 32] * (a1 > 0.f ? a1 : 0.f);
            for (int o = 16; o >= 1; o >>= 1) p += __shfl_xor_sync(0xFFFFFFFFu, p, o);
            const float z = p + s.W[ob3];
            float dz = 0.f;
            if (r < rows) {
                const float yy = y[base + r], ww = w[base + r] * inv_w;
                lsum += ww * (softplus(z) - yy * z);
                dz = ww * (1.0f / (1.0f + expf(-z)) - yy);
            }
            if (lane == 0) s.dz[r] = dz;
        }
        if (lane == 0) s.lossp[wp] = lsum;
    }
    __syncthreads();
    if (tid == 0 && loss) {
        float t = 0.f;
        for (int i = 0; i < kThreads / 32; ++i) t += s.lossp[i];
        atomicAdd(loss, t);
    }
    // gW3, gb3 (before A2 is overwritten by D2)
    if (tid < kH) {
        float g = 0.f;
        for (int r = 0; r < kTile; ++r) {
            float a = s.A2[r][tid];
            g = fmaf(s.dz[r], a > 0.f ? a : 0.f, g);
        }
        atomicAdd(&G[oW3 + tid], g);
    } else if (tid == kH) {
        float g = 0.f;
        for (int r = 0; r < kTile; ++r) g += s.dz[r];
        atomicAdd(&G[ob3], g);
    }
    __syncthreads();
    // D2 = dz W3 .* [A2 > 0]   (in place of A2)
    for (int i = tid; i < kTile * kH; i += kThreads) {
        int r = i / kH, o = i % kH;
        s.A2[r][o] = s.A2[r][o] > 0.f ? s.dz[r] * s.W[oW3 + o] : 0.f;
    }
    __syncthreads();
    // gW2 = D2^T H1 (64 x 64), gb2 = colsum D2
    for (int i = tid; i < kH * kH; i += kThreads) {
        int o = i / kH, c = i % kH;
        float g = 0.f;
        for (int r = 0; r < kTile; ++r) g = fmaf(s.A2[r][o], s.H1[r][c], g);
        atomicAdd(&G[oW2 + i], g);
    }
    if (tid < kH) {
        float g = 0.f;
        for (int r = 0; r < kTile; ++r) g += s.A2[r][tid];
        atomicAdd(&G[ob2 + tid], g);
    }
    __syncthreads();  // H1 is read above and overwritten below
    // D1 = (D2 W2) .* [A1 > 0]   (into H1)
    for (int i = tid; i < kTile * kH; i += kThreads) {
        int r = i / kH, c = i % kH;
        float a = 0.f;
        for (int o = 0; o < kH; ++o) a = fmaf(s.A2[r][o], s.W[oW2 + o * kH + c], a);
        s.H1[r][c] = s.A1[r][c] > 0.f ? a : 0.f;  // H1 no longer needed: holds D1
    }
    __syncthreads();
    // gW1 = D1^T X (64 x 16), gb1 = colsum D1
    for (int i = tid; i < kH * kIn; i += kThreads) {
        int o = i / kIn, c = i % kIn;
        float g = 0.f;
        for (int r = 0; r < kTile; ++r) g = fmaf(s.H1[r][o], s.X[r][c], g);
        atomicAdd(&G[oW1 + i], g);
    }
    if (tid < kH) {
        float g = 0.f;
        for (int r = 0; r < kTile; ++r) g += s.H1[r][tid];
        atomicAdd(&G[ob1 + tid], g);
    }
}

__global__ void adam_kernel(float *P, const float *G, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void __launch_bounds__(kThreads) mlp_forward_kernel(const float *__restrict__ P,
                                                               const float *__restrict__ X, int n,
                                                               float *__restrict__ z) {
    __shared__ float W[SQG_MLP_NPARAM];
    for (int i = threadIdx.x; i < SQG_MLP_NPARAM; i += blockDim.x) W[i] = P[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n) return;
    float x[kIn];
    for (int c = 0; c < kIn; ++c) x[c] = X[(size_t)r * kIn + c];
    float ha = W[ob1 + lane], hb = W[ob1 + lane + 32];
    for (int c = 0; c < kIn; ++c) {
        ha = fmaf(W[oW1 + lane * kIn + c], x[c], ha);
        hb = fmaf(W[oW1 + (lane + 32) * kIn + c], x[c], hb);
    }
    ha = fmaxf(ha, 0.f);
    hb = fmaxf(hb, 0.f);
    float ga = W[ob2 + lane], gb = W[ob2 + lane + 32];
    for (int c = 0; c < kH; ++c) {
        float h = __shfl_sync(0xFFFFFFFFu, c < 32 ? ha : hb, c & 31);
        ga = fmaf(W[oW2 + lane * kH + c], h, ga);
        gb = fmaf(W[oW2 + (lane + 32) * kH + c], h, gb);
    }
    float p = W[oW3 + lane] * fmaxf(ga, 0.f) + W[oW3 + lane + 32] * fmaxf(gb, 0.f);
    for (int o = 16; o >= 1; o >>= 1) p += __shfl_xor_sync(0xFFFFFFFFu, p, o);
    if (lane == 0) z[r] = p + W[ob3];
}

}  // namespace

extern "C" int sqg_mlp_grad(const float *params, const float *x, const float *y, const float *w, int n,
                            float *grad, float *loss, float *scratch, sqg_stream_t stream_) {
    if (!params || !x || !y || !w || !grad || !scratch || n < 1) return SQG_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const size_t smem = sizeof(TileSmem);
    if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SQG_ERR_CUDA;
    if (cudaMemsetAsync(grad, 0, sizeof(float) * SQG_MLP_NPARAM, stream) != cudaSuccess) return SQG_ERR_CUDA;
    if (loss && cudaMemsetAsync(loss, 0, sizeof(float), stream) != cudaSuccess) return SQG_ERR_CUDA;
    weight_sum_kernel<<<1, kThreads, 0, stream>>>(w, n, scratch);
    mlp_grad_kernel<<<(n + kTile - 1) / kTile, kThreads, smem, stream>>>(params, x, y, w, n, scratch, grad, loss);
    return cudaGetLastError() == cudaSuccess ? SQG_OK : SQG_ERR_CUDA;
}

extern "C" int sqg_mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr, float beta1,
                            float beta2, float eps, sqg_stream_t stream_) {
    if (!params || !grad || !m || !v || step < 1 || !(lr > 0.f)) return SQG_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<(SQG_MLP_NPARAM + 255) / 256, 256, 0, stream>>>(params, grad, m, v, SQG_MLP_NPARAM, lr, beta1,
                                                                  beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? SQG_OK : SQG_ERR_CUDA;
}

extern "C" int sqg_mlp_forward(const float *params, const float *x, int n, float *logits, sqg_stream_t stream_) {
    if (!params || !x || !logits || n < 0) return SQG_ERR_INVALID_ARG;
    if (n == 0) return SQG_OK;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const int wpb = kThreads / 32;
    mlp_forward_kernel<<<(n + wpb - 1) / wpb, kThreads, 0, stream>>>(params, x, n, logits);
    return cudaGetLastError() == cudaSuccess ? SQG_OK : SQG_ERR_CUDA;
}
