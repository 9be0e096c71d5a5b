// fjlt.cu -- the query side of the fast Johnson-Lindenstrauss transform
// (Sec. 3.1.4: the random rotation applied with the fast Hadamard
// transform in O(d log d) instead of a dense d x d product).
//
// q' = c H S_3 c H S_2 c H S_1 q for d a power of 2, S_r the diagonal signs
// of the index (derived from its rotation seed), H the Walsh-Hadamard
// transform (+1/-1 entries) and c = fl(1/sqrt(d)).  One warp per query; the
// query's element 32e + lane sits in register e of that lane, so the
// transform's stages h = 1 .. 16 are lane shuffles and h = 32 .. d/2 pair
// registers.  Every stage replaces (y_j, y_j+h), j without bit h, by
// (y_j + y_j+h, y_j - y_j+h) in fp32 with round-to-nearest, the stages run
// in the order h = 1, 2, 4, ..., so the result is bit for bit the one an
// in-order sequential transform gives.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kWarps = 4;

template <int E>  // d = 32 E
__global__ void __launch_bounds__(kWarps * 32)
    fjlt_kernel(const float *__restrict__ q, const float *__restrict__ signs, float *__restrict__ out, int nq) {
    constexpr int d = 32 * E;
    const int lane = threadIdx.x & 31;
    const int qi = blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (qi >= nq) return;
    const float *src = q + (size_t)qi * d;
    float x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = __ldg(src + e * 32 + lane);
    const float c = __fdiv_rn(1.0f, __fsqrt_rn((float)d));
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = __fmul_rn(x[e], __ldg(signs + r * d + e * 32 + lane));
#pragma unroll
        for (int h = 1; h < 32; h <<= 1) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float v = __shfl_xor_sync(0xFFFFFFFFu, x[e], h);
                x[e] = (lane & h) ? __fsub_rn(v, x[e]) : __fadd_rn(x[e], v);
            }
        }
#pragma unroll
        for (int m = 1; m < E; m <<= 1) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (e & m) continue;
                const float a = x[e], b = x[e | m];
                x[e] = __fadd_rn(a, b);
                x[e | m] = __fsub_rn(a, b);
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = __fmul_rn(x[e], c);
    }
    float *dst = out + (size_t)qi * d;
#pragma unroll
    for (int e = 0; e < E; ++e) dst[e * 32 + lane] = x[e];
}

template <int E>
cudaError_t launch_e(const float *q, const float *signs, float *out, int nq, cudaStream_t s) {
    fjlt_kernel<E><<<(nq + kWarps - 1) / kWarps, kWarps * 32, 0, s>>>(q, signs, out, nq);
    return cudaGetLastError();
}

}  // namespace

namespace sqg {

// q' for nq queries (nq x d, row-major) into out; d a power of 2 in 32..2048.
cudaError_t launch_fjlt(const float *q, const float *signs, float *out, int nq, int d, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    switch (d) {
        case 32: return launch_e<1>(q, signs, out, nq, s);
        case 64: return launch_e<2>(q, signs, out, nq, s);
        case 128: return launch_e<4>(q, signs, out, nq, s);
        case 256: return launch_e<8>(q, signs, out, nq, s);
        case 512: return launch_e<16>(q, signs, out, nq, s);
        case 1024: return launch_e<32>(q, signs, out, nq, s);
        case 2048: return launch_e<64>(q, signs, out, nq, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sqg
