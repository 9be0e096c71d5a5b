// sqg_api.cu -- the C ABI of libsqg: index loading, launch planning and the
// query-preparation kernels (rotation q' = P^-1 q, Eq. (4); 4-bit
// quantization; per-query output offsets).  The search kernel itself is in
// search.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/sqg.h"
#include "index_format.h"
#include "search.cuh"

using namespace sqg;

struct sqg_index {
    int device;
    sqg_fmt::Layout lay;
    uint32_t entry;
    unsigned char *d_blocks;
    float *d_rot;
    float *d_rot_hi, *d_rot_lo;  // tf32 split of the rotation for the tensor-core path
    bool fjlt;                   // version 2: queries are rotated by the fast JLT
    bool cosine;                 // metric 1: queries are scaled to unit norm first
    uint32_t version;
    float *d_signs;              // its 3 x d signs
    uint32_t *d_status;
    int num_sms;
    size_t smem_optin;
};

namespace {

constexpr int kPlanThreads = 1024;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
// The kernels read query rows as float4 and workspace regions as uint4.
inline bool aligned(const void *p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

// ---------------------------------------------------------------- kernels

// Output offsets (exclusive prefix sum of each query's slot count) and the
// largest valid k / ef of the batch.  One block; each thread scans
// kPlanItems consecutive queries of a tile, so a 10k batch takes two tiles.
constexpr int kPlanItems = 16;
__global__ void plan_kernel(const int32_t *k, const int32_t *ef, int nq, long long *offsets, int *maxes) {
    __shared__ long long warp_sums[kPlanThreads / 32];
    __shared__ long long carry;
    __shared__ int smax_k, smax_ef;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) { carry = 0; smax_k = 0; smax_ef = 0; }
    __syncthreads();
    int mk = 0, me = 0;
    for (int base = 0; base < nq; base += kPlanThreads * kPlanItems) {
        const int i0 = base + tid * kPlanItems;
        int c[kPlanItems];
        long long tsum = 0;
#pragma unroll
        for (int j = 0; j < kPlanItems; ++j) {
            const int i = i0 + j;
            c[j] = 0;
            if (i < nq) {
                const int kk = k[i], ee = ef[i];
                c[j] = kk < 0 ? 0 : (kk > SQG_MAX_K ? SQG_MAX_K : kk);
                if (kk >= 1 && kk <= SQG_MAX_K && ee >= kk && ee <= SQG_MAX_EF) {
                    mk = max(mk, kk);
                    me = max(me, ee);
                }
            }
            tsum += c[j];
        }
        long long x = tsum;  // inclusive scan of the threads' sums within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            long long s = lane < kPlanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xFFFFFFFFu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;  // inclusive over warps
        }
        __syncthreads();
        long long run = carry + (w > 0 ? warp_sums[w - 1] : 0) + x - tsum;
#pragma unroll
        for (int j = 0; j < kPlanItems; ++j) {
            if (i0 + j < nq) offsets[i0 + j] = run;
            run += c[j];
        }
        __syncthreads();
        if (tid == kPlanThreads - 1) carry = run;
        __syncthreads();
    }
    atomicMax(&smax_k, mk);
    atomicMax(&smax_ef, me);
    __syncthreads();
    if (tid == 0) {
        maxes[0] = smax_k;
        maxes[1] = smax_ef;
    }
}

// The stop network's parameters (W1 [64][16], b1, W2 [64][64], b2, W3, b3)
// in the packed layout mlp_logit_warp reads: for lane l and input pair i2,
// the weights of neurons l and l + 32 for inputs 2 i2 and 2 i2 + 1 side by
// side (one 16-byte load), the biases and output weights of l and l + 32 as
// pairs, then b3.
__global__ void mlp_transpose_kernel(const float *__restrict__ src, float *__restrict__ dst) {
    const float *W1 = src, *b1 = W1 + 64 * SQG_MLP_IN, *W2 = b1 + 64, *b2 = W2 + 64 * 64, *W3 = b2 + 64;
    float *t = dst;
    for (int e = threadIdx.x; e < 8 * 32; e += blockDim.x) {  // W1p[i2][l]
        const int i2 = e / 32, l = e % 32;
        t[4 * e + 0] = W1[l * SQG_MLP_IN + 2 * i2];
        t[4 * e + 1] = W1[(l + 32) * SQG_MLP_IN + 2 * i2];
        t[4 * e + 2] = W1[l * SQG_MLP_IN + 2 * i2 + 1];
        t[4 * e + 3] = W1[(l + 32) * SQG_MLP_IN + 2 * i2 + 1];
    }
    t += 8 * 32 * 4;
    for (int l = threadIdx.x; l < 32; l += blockDim.x) {
        t[2 * l] = b1[l];
        t[2 * l + 1] = b1[l + 32];
    }
    t += 64;
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {  // W2p[i2][l]
        const int i2 = e / 32, l = e % 32;
        t[4 * e + 0] = W2[l * 64 + 2 * i2];
        t[4 * e + 1] = W2[(l + 32) * 64 + 2 * i2];
        t[4 * e + 2] = W2[l * 64 + 2 * i2 + 1];
        t[4 * e + 3] = W2[(l + 32) * 64 + 2 * i2 + 1];
    }
    t += 32 * 32 * 4;
    for (int l = threadIdx.x; l < 32; l += blockDim.x) {
        t[2 * l] = b2[l];
        t[2 * l + 1] = b2[l + 32];
        t[64 + 2 * l] = W3[l];
        t[64 + 2 * l + 1] = W3[l + 32];
    }
    if (threadIdx.x == 0) t[128] = W3[64];  // b3
}

// q' = P^-1 q for a batch (Eq. (4)) in the canonical chunked order:
// out[r][i] = (((0 + s_0) + s_1) + ...) over the d/32 chunks, s_c the fmaf
// chain of rot[i][j] * q[r][j] over j = 32c .. 32c+31 from 0.  64 x 64 output
// tiles, 256 threads with 4 x 4 outputs each; one 32-wide chunk of q and of
// P^-1 per step, double-buffered in shared memory (the next chunk's global
// loads are in flight while this one is multiplied), so every output walks
// j in order with one chunk accumulator and one total and the tiling changes
// no bit.
constexpr int kRotT = 64, kRotK = 32;
__global__ void __launch_bounds__(256) rotate_kernel(const float *__restrict__ q, const float *__restrict__ rot,
                                                     float *__restrict__ out, int nq, int d) {
    __shared__ __align__(16) float As[2][kRotK][kRotT + 4];  // [buffer][j][row]
    __shared__ __align__(16) float Bs[2][kRotK][kRotT + 4];  // [buffer][j][col]
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int r0 = blockIdx.y * kRotT, c0 = blockIdx.x * kRotT;
    constexpr int kPer = kRotT * kRotK / 256;  // elements of each tile a thread moves
    float ra[kPer], rb[kPer];
    auto load = [&](int j0) {
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            const int e = tid + 256 * t, rr = e / kRotK, jj = e % kRotK;
            const int gr = r0 + rr, gc = c0 + rr;
            ra[t] = gr < nq ? q[(size_t)gr * d + j0 + jj] : 0.0f;
            rb[t] = gc < d ? rot[(size_t)gc * d + j0 + jj] : 0.0f;
        }
    };
    auto store = [&](int b) {
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            const int e = tid + 256 * t, rr = e / kRotK, jj = e % kRotK;
            As[b][jj][rr] = ra[t];
            Bs[b][jj][rr] = rb[t];
        }
    };
    float acc[4][4], tot[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) tot[a][b] = 0.0f;
    load(0);
    store(0);
    __syncthreads();
    const int nchunk = d / kRotK;
    for (int c = 0; c < nchunk; ++c) {
        const int buf = c & 1;
        if (c + 1 < nchunk) load((c + 1) * kRotK);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
#pragma unroll 8
        for (int jj = 0; jj < kRotK; ++jj) {
            const float4 av = *reinterpret_cast<const float4 *>(&As[buf][jj][ty * 4]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[buf][jj][tx * 4]);
            const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = __fmaf_rn(b4[b], a4[a], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) tot[a][b] = __fadd_rn(tot[a][b], acc[a][b]);
        if (c + 1 < nchunk) store(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int gr = r0 + ty * 4 + a;
        if (gr >= nq) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int gc = c0 + tx * 4 + b;
            if (gc < d) out[(size_t)gr * d + gc] = tot[a][b];
        }
    }
}

// Cosine similarity as Euclidean search between unit vectors: q / ||q||,
// one warp per query.  ||q||^2 in the exact distance's order (lane l sums
// float4 chunks l, l+32, ... with fmaf(x, x, acc), then the xor butterfly
// 16, 8, 4, 2, 1), then each coordinate divided by fl(sqrt(||q||^2)); a
// query whose squared norm is 0 or not finite is copied as it is.
constexpr int kNormWarps = 8;
__global__ void __launch_bounds__(kNormWarps * 32) normalize_kernel(const float *__restrict__ q,
                                                                    float *__restrict__ out, int nq, uint32_t d) {
    const int lane = threadIdx.x & 31;
    const long long qi = (long long)blockIdx.x * kNormWarps + (threadIdx.x >> 5);
    if (qi >= nq) return;  // uniform over the warp
    const float4 *src = reinterpret_cast<const float4 *>(q + (size_t)qi * d);
    float4 *dst = reinterpret_cast<float4 *>(out + (size_t)qi * d);
    const uint32_t nch = d / 4;
    float acc = 0.0f;
    for (uint32_t c = lane; c < nch; c += 32) {
        const float4 x = src[c];
        acc = __fmaf_rn(x.x, x.x, acc);
        acc = __fmaf_rn(x.y, x.y, acc);
        acc = __fmaf_rn(x.z, x.z, acc);
        acc = __fmaf_rn(x.w, x.w, acc);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    const bool scale = acc > 0.0f && acc <= 3.40282347e38f;
    const float r = __fsqrt_rn(acc);
    for (uint32_t c = lane; c < nch; c += 32) {
        float4 x = src[c];
        if (scale) {
            x.x = __fdiv_rn(x.x, r);
            x.y = __fdiv_rn(x.y, r);
            x.z = __fdiv_rn(x.z, r);
            x.w = __fdiv_rn(x.w, r);
        }
        dst[c] = x;
    }
}

// Quantized query export (test entry point): one warp per query.
__global__ void quantize_kernel(const float *qrot, int nq, int d, uint32_t *planes, float *scal) {
    const int lane = threadIdx.x & 31;
    const int qi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (qi >= nq) return;
    extern __shared__ __align__(16) uint32_t pl_smem[];
    uint32_t *pl = pl_smem + (threadIdx.x >> 5) * (4 * (d / 32));
    const QuerySide qs = quantize_warp(qrot + (size_t)qi * d, (uint32_t)d, pl, lane);
    __syncwarp();
    // shared layout is word-major ([w][b]); the export is plane-major ([b][w])
    for (int i = lane; i < 4 * (d / 32); i += 32) {
        const int b = i / (d / 32), w = i % (d / 32);
        planes[(size_t)qi * 4 * (d / 32) + i] = pl[4 * w + b];
    }
    if (lane == 0) {
        scal[qi * 4 + 0] = qs.vl;
        scal[qi * 4 + 1] = qs.delta;
        scal[qi * 4 + 2] = (float)qs.sq;
        scal[qi * 4 + 3] = qs.inv_sqrt_d;
    }
}

// Estimates of one block per query with the search kernel's own device
// functions (test entry point).  One warp per query; the block is staged in
// shared memory with plain 16-byte loads.
__global__ void estimate_block_kernel(SearchArgs a, const uint32_t *v, int32_t *out_S, float *out_est,
                                      float *out_key, float *out_dist_c) {
    extern __shared__ __align__(16) unsigned char eb_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int qi = blockIdx.x * (blockDim.x >> 5) + w;
    if (qi >= a.nq) return;
    const uint32_t d = a.d, R = a.R;
    unsigned char *blk = eb_smem + (size_t)w * a.warp_bytes;
    uint32_t *planes = reinterpret_cast<uint32_t *>(blk + a.block_bytes);
    const uint32_t vv = v[qi];
    if (vv >= a.n) {  // out-of-range vertex: NaN outputs, no access
        for (uint32_t j = lane; j < R; j += 32) {
            out_S[(size_t)qi * R + j] = 0;
            out_est[(size_t)qi * R + j] = __int_as_float(0x7fc00000);
            out_key[(size_t)qi * R + j] = __int_as_float(0x7fc00000);
        }
        if (lane == 0) out_dist_c[qi] = __int_as_float(0x7fc00000);
        return;
    }
    const uint4 *src = reinterpret_cast<const uint4 *>(a.blocks + (size_t)vv * a.block_bytes);
    for (uint32_t i = lane; i < a.block_bytes / 16; i += 32) reinterpret_cast<uint4 *>(blk)[i] = src[i];
    float4 qv[16];
    const float *q = a.queries + (size_t)qi * d;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        uint32_t c = lane + 32 * t;
        qv[t] = c < d / 4 ? reinterpret_cast<const float4 *>(q)[c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const QuerySide qs = quantize_warp(a.qrot + (size_t)qi * d, d, planes, lane);
    __syncwarp();
    const float dist_c = exact_dist<16>(qv, reinterpret_cast<const float *>(blk), d / 4, lane);
    const float sqrt_dc = __fsqrt_rn(dist_c);
    for (uint32_t j = lane; j < R; j += 32) {
        const Est e = estimate(blk, a, planes, qs, j, dist_c, sqrt_dc);
        out_S[(size_t)qi * R + j] = e.S;
        out_est[(size_t)qi * R + j] = e.est;
        out_key[(size_t)qi * R + j] = e.key;
    }
    if (lane == 0) out_dist_c[qi] = dist_c;
}

// ---------------------------------------------------------------- planning

int pick_ch(uint32_t d) {
    const uint32_t need = (d / 4 + 31) / 32;
    for (int c : {1, 2, 4, 8, 12, 16})
        if ((uint32_t)c >= need) return c;
    return -1;
}

struct LaunchPlan {
    int ch, nb, team, warps, grid;
    bool compact;  // the compact kernel (search_compact.cu)
    int cbnb;      // its beam slots per lane: 2 (ef <= 64), 4 (ef <= 128) or 8 (ef <= 256, d <= 256)
    int crk;       // its result slots per lane: 1 (k <= 32) or 4 (k <= 128, d <= 256)
    size_t smem;
    SearchArgs a;  // layout fields filled in
    bool ghash;
    // workspace layout
    size_t ws_offsets, ws_qrot, ws_queue, ws_maxes, ws_stats, ws_ghash, ws_planes, ws_scal, ws_mlp, ws_qnorm,
        ws_total;
};

int make_plan(const sqg_index *ix, int nq, int max_k, int max_ef, const sqg_search_params &p, LaunchPlan &pl,
              bool traced = false) {
    const uint32_t d = ix->lay.d, R = ix->lay.R, bb = ix->lay.block_bytes;
    pl.ch = pick_ch(d);
    pl.nb = (int)(R / 32);
    if (pl.ch < 0 || (pl.nb != 1 && pl.nb != 2)) return SQG_ERR_UNSUPPORTED;
    pl.team = p.team == 0 ? 32 : p.team;
    const int V = 32 / pl.team;  // queries per warp
    // the compact kernel's range: k <= 32 and ef <= 128, for d <= 256 k <= 128
    // and ef <= 256
    const bool small_d = pl.ch <= 2;
    pl.compact = p.kernel != 1 && pl.team == 32 && pl.ch <= 8 && max_k <= (small_d ? 128 : 32) &&
                 max_ef <= (small_d ? 256 : 128) && p.multi_estimate && !traced && p.prefetch != 2 && p.lean != 2;
    if (p.kernel == 2 && !pl.compact) return SQG_ERR_UNSUPPORTED;
    pl.cbnb = max_ef <= 64 ? 2 : max_ef <= 128 ? 4 : 8;
    pl.crk = max_k <= 32 ? 1 : 4;
    const bool big = pl.compact && (pl.cbnb == 8 || pl.crk == 4);  // search_compact_big.cu
    if (pl.compact) {
    } else if (pl.team < 32) {
        // smaller teams: d <= 256, the 96-register build, no fused stop network
        if (pl.ch > 2 || p.stop_mlp) return SQG_ERR_UNSUPPORTED;
    } else if (p.lean != 2 && pl.ch <= 2) {
        // the 64-register build for d <= 256 unless asked for the full one
        // (measured faster at d = 128: more resident warps hide more latency)
        pl.ch = -pl.ch;
    }
    const long long cap = p.hop_cap > 0 ? p.hop_cap : 4LL * max_ef + 64;
    uint32_t bits = 5;
    while ((1ull << bits) < 2ull * (unsigned long long)cap + 1) ++bits;
    if (bits > 26) return SQG_ERR_CAPACITY;
    SearchArgs &a = pl.a;
    std::memset(&a, 0, sizeof(a));
    a.hash_bits = bits;
    const size_t hash_bytes = (size_t)4 << bits;
    size_t o = 0;
    // one block buffer: every read of a block (raw vector, codes, factors,
    // ids) is done before the next block's copy is issued into it, and at
    // most one copy is in flight, so the two mbarrier phases of the kernel's
    // double-buffer protocol can share it -- half the shared memory, twice
    // the resident warps at d = 960 / 1536
    a.o_buf0 = (uint32_t)o; o += bb;
    a.o_buf1 = a.o_buf0;
    a.o_bar = (uint32_t)o; o += 32;  // the mbarrier(s); the compact kernel keeps its stop state after the first
    a.o_planes = (uint32_t)o; o = align_up(o + 16 * (d / 32), 16);
    if (pl.compact) {
        // two beam buffers of 32 cbnb packed entries, the step's candidates
        // by rank (R packed entries); the results live in registers
        a.o_beam = (uint32_t)o; o += 2 * 32 * (size_t)pl.cbnb * 8;
        a.o_res = (uint32_t)o;
        a.o_spos = (uint32_t)o; o += (size_t)R * 8;
    } else {
        a.o_beam = (uint32_t)o; o = align_up(o + 8 * (size_t)max_ef, 16);
        a.o_res = (uint32_t)o; o = align_up(o + 8 * (size_t)max_k, 16);
        // the admitted candidates' positions; also the stop network's 64
        // hidden values between its layers
        a.o_spos = (uint32_t)o; o = align_up(o + std::max<size_t>(4 * (size_t)R, 256), 16);
    }
    // visited set: up to 2^10 slots in shared memory; a longer search moves
    // to its warp's full-size table in the workspace
    const uint32_t smem_bits_default = 9u;  // 2^10 measured slower at large beams (less residency)
    a.shash_bits =
        std::min<uint32_t>(bits, p.visited_smem_log2 > 0 ? (uint32_t)p.visited_smem_log2 : smem_bits_default);
    pl.ghash = a.shash_bits < bits;
    a.o_hash = (uint32_t)o;
    const size_t warp_bytes = align_up(o + ((size_t)4 << a.shash_bits), 128);
    const size_t cta = 0;  // the stop network's weights are read from the workspace (L1-cached)
    // one slot of warp_bytes per query in flight: V per warp
    auto occupancy = [&](int w, int *blocks) -> cudaError_t {
        const size_t sm = cta + (size_t)w * V * warp_bytes;
        *blocks = 0;
        if (sm > ix->smem_optin) return cudaSuccess;
        return big ? search_occupancy_compact_big(pl.ch, pl.nb, pl.cbnb, pl.crk, p.stop_mlp != nullptr, w * 32, sm,
                                                  blocks)
             : pl.compact && p.stop_mlp ? search_occupancy_compact_stop(pl.ch, pl.nb, pl.cbnb, w * 32, sm, blocks)
             : pl.compact     ? search_occupancy_compact(pl.ch, pl.nb, pl.cbnb, p.lean, w * 32, sm, blocks)
             : pl.team < 32 ? search_occupancy_team(pl.ch, pl.nb, pl.team, w * 32, sm, blocks)
             : pl.nb == 1   ? search_occupancy_nb1(pl.ch, w * 32, sm, blocks)
                            : search_occupancy_nb2(pl.ch, w * 32, sm, blocks);
    };
    int warps = 0, per_sm = 0;
    if (p.warps_per_block > 0) {
        warps = std::min(p.warps_per_block, 4);
        while (warps > 1 && cta + warps * V * warp_bytes > ix->smem_optin) --warps;
        if (occupancy(warps, &per_sm) != cudaSuccess) return SQG_ERR_CUDA;
    } else {
        // the block size with the most resident warps per SM (shared memory
        // limits large d, registers small d); larger blocks on a tie
        for (int w : {4, 2, 1}) {
            int b = 0;
            if (occupancy(w, &b) != cudaSuccess) return SQG_ERR_CUDA;
            if (b * w > per_sm * warps) {
                warps = w;
                per_sm = b;
            }
        }
    }
    if (warps < 1 || per_sm < 1) return SQG_ERR_CAPACITY;
    a.warp_bytes = (uint32_t)warp_bytes;
    a.cta_bytes = (uint32_t)cta;
    pl.warps = warps;
    pl.smem = cta + warps * V * warp_bytes;
    const long long want = ((long long)nq + warps * V - 1) / (warps * V);
    pl.grid = (int)std::max(1LL, std::min<long long>((long long)per_sm * ix->num_sms, want));
    // workspace
    size_t w = 0;
    pl.ws_offsets = w; w = align_up(w + 8 * (size_t)std::max(nq, 1), 256);
    pl.ws_qrot = w; w = align_up(w + 4 * (size_t)std::max(nq, 1) * d, 256);
    pl.ws_queue = w; w = align_up(w + 4, 256);
    pl.ws_maxes = w; w = align_up(w + 8, 256);
    pl.ws_stats = w; w = align_up(w + sizeof(sqg_query_stats) * (size_t)std::max(nq, 1), 256);
    pl.ws_ghash = w;
    if (pl.ghash) w = align_up(w + hash_bytes * (size_t)pl.grid * warps * V, 256);
    // the exactly quantized query after a tensor-core rotation
    pl.ws_planes = w; w = align_up(w + 16 * (size_t)(d / 32) * (size_t)std::max(nq, 1), 256);
    pl.ws_scal = w; w = align_up(w + 16 * (size_t)std::max(nq, 1), 256);
    // the stop network, its two weight matrices transposed to [in][out]
    pl.ws_mlp = w;
    if (p.stop_mlp) w = align_up(w + sizeof(float) * SQG_MLP_NPARAM, 256);
    // the unit-norm queries of a cosine index
    pl.ws_qnorm = w;
    if (ix->cosine) w = align_up(w + 4 * (size_t)std::max(nq, 1) * d, 256);
    pl.ws_total = w;
    return SQG_OK;
}

// The queries every later step reads: on a cosine index their unit-norm
// copies, written to `scratch` (nq x d floats), else the caller's.
const float *queries_for(const sqg_index *ix, const float *queries, int nq, float *scratch, cudaStream_t stream,
                         cudaError_t *e) {
    *e = cudaSuccess;
    if (!ix->cosine) return queries;
    const long long blocks = ((long long)nq + kNormWarps - 1) / kNormWarps;
    normalize_kernel<<<(unsigned)blocks, kNormWarps * 32, 0, stream>>>(queries, scratch, nq, ix->lay.d);
    *e = cudaGetLastError();
    return scratch;
}

// q' on the CUDA cores: the fast JLT for a version-2 index, else the dense
// P^-1 q in the canonical chunked order.
cudaError_t rotate_simt(const sqg_index *ix, const float *queries, float *out, int nq, cudaStream_t stream) {
    const int d = (int)ix->lay.d;
    if (ix->fjlt) return launch_fjlt(queries, ix->d_signs, out, nq, d, stream);
    dim3 rg((d + kRotT - 1) / kRotT, (nq + kRotT - 1) / kRotT);
    rotate_kernel<<<rg, 256, 0, stream>>>(queries, ix->d_rot, out, nq, d);
    return cudaGetLastError();
}

// Rotation path: 1 = the CUDA-core kernel in the canonical order, 2 = tensor
// cores plus the exact quantization pass (same codes bit for bit); 0 = tensor
// cores from d = 512 up (2.5x faster there; at d = 128 the two tie).
bool use_tc_rotation(const sqg_index *ix, const sqg_search_params &p) {
    if (ix->fjlt || p.rotation == 1) return false;  // the fast JLT needs no contraction
    if (p.rotation == 2) return true;
    return ix->lay.d >= 512;
}

sqg_search_params default_params() {
    sqg_search_params p;
    std::memset(&p, 0, sizeof(p));
    p.multi_estimate = 1;
    p.stop_every = 1;
    return p;
}

int check_params(const sqg_search_params &p) {
    if (p.hop_cap < 0 || p.max_k < 0 || p.max_ef < 0 || p.max_k > SQG_MAX_K || p.max_ef > SQG_MAX_EF ||
        (p.max_k > 0 && p.max_ef > 0 && p.max_ef < p.max_k) || p.stop_every < 0 ||
        (p.team != 0 && p.team != 8 && p.team != 16 && p.team != 32) || p.warps_per_block < 0 ||
        !std::isfinite(p.eps0) ||
        (p.visited_smem_log2 != 0 && (p.visited_smem_log2 < 5 || p.visited_smem_log2 > 12)) ||
        p.prefetch < 0 || p.prefetch > 2 || p.lean < 0 || p.lean > 2 || p.rotation < 0 || p.rotation > 2 ||
        p.kernel < 0 || p.kernel > 2 || p.uniform_k < 0 || p.uniform_k > SQG_MAX_K ||
        (p.stop_mlp && p.stop_every < 1))
        return SQG_ERR_INVALID_ARG;
    return SQG_OK;
}

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" const char *sqg_error_string(int code) {
    switch (code) {
        case SQG_OK: return "ok";
        case SQG_ERR_INVALID_ARG: return "invalid argument";
        case SQG_ERR_IO: return "i/o error";
        case SQG_ERR_FORMAT: return "bad index file format";
        case SQG_ERR_OOM: return "out of memory";
        case SQG_ERR_CUDA: return "CUDA error";
        case SQG_ERR_TIMEOUT: return "bounded device wait expired";
        case SQG_ERR_CAPACITY: return "capacity exceeded";
        case SQG_ERR_UNSUPPORTED: return "unsupported index shape";
        default: return "unknown error";
    }
}

extern "C" int sqg_index_load(const char *path, int device, sqg_index **out) {
    if (!path || !out || device < 0) return SQG_ERR_INVALID_ARG;
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return SQG_ERR_IO;
    std::fseek(f, 0, SEEK_END);
    const long long fsize = std::ftell(f);
    std::fseek(f, 0, SEEK_SET);
    unsigned char hdr[sqg_fmt::kHeaderBytes];
    if (fsize < (long long)sizeof(hdr) || std::fread(hdr, 1, sizeof(hdr), f) != sizeof(hdr)) {
        std::fclose(f);
        return fsize < (long long)sizeof(hdr) ? SQG_ERR_FORMAT : SQG_ERR_IO;
    }
    sqg_fmt::Header h;
    if (!sqg_fmt::parse_header(hdr, (uint64_t)fsize, h)) {
        std::fclose(f);
        return SQG_ERR_FORMAT;
    }
    const sqg_fmt::Layout &L = h.l;
    if (L.n > 0x7FFFFFFFull) { std::fclose(f); return SQG_ERR_UNSUPPORTED; }
    if (pick_ch(L.d) < 0 || (L.R != 32 && L.R != 64)) { std::fclose(f); return SQG_ERR_UNSUPPORTED; }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) {
        cudaGetLastError();
        std::fclose(f);
        return SQG_ERR_INVALID_ARG;
    }
    DeviceGuard g(device);
    sqg_index *ix = new (std::nothrow) sqg_index();
    if (!ix) { std::fclose(f); return SQG_ERR_OOM; }
    ix->device = device;
    ix->lay = L;
    ix->entry = h.entry;
    ix->fjlt = h.version == sqg_fmt::kVersionFjlt;
    ix->cosine = h.metric == sqg_fmt::kMetricCosine;
    ix->version = h.version;
    cudaDeviceGetAttribute(&ix->num_sms, cudaDevAttrMultiProcessorCount, device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    ix->smem_optin = (size_t)optin;
    const size_t block_bytes_total = (size_t)L.n * L.block_bytes;
    if (cudaMalloc(&ix->d_blocks, block_bytes_total) != cudaSuccess ||
        cudaMalloc(&ix->d_rot, sizeof(float) * (size_t)L.d * L.d) != cudaSuccess ||
        cudaMalloc(&ix->d_rot_hi, sizeof(float) * (size_t)L.d * L.d) != cudaSuccess ||
        cudaMalloc(&ix->d_rot_lo, sizeof(float) * (size_t)L.d * L.d) != cudaSuccess ||
        cudaMalloc(&ix->d_status, sizeof(uint32_t)) != cudaSuccess) {
        std::fclose(f);
        sqg_index_free(ix);
        cudaGetLastError();
        return SQG_ERR_OOM;
    }
    cudaMemset(ix->d_status, 0, sizeof(uint32_t));
    if (ix->fjlt) {  // the fast JLT's signs, from the rotation seed
        std::vector<float> sg(3 * (size_t)L.d);
        for (uint32_t r = 0; r < 3; ++r)
            for (uint32_t i = 0; i < L.d; ++i) sg[(size_t)r * L.d + i] = sqg_fmt::fjlt_sign(h.seed_rot, r, i);
        if (L.d > 2048 || cudaMalloc(&ix->d_signs, sizeof(float) * sg.size()) != cudaSuccess ||
            cudaMemcpy(ix->d_signs, sg.data(), sizeof(float) * sg.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            std::fclose(f);
            sqg_index_free(ix);
            cudaGetLastError();
            return SQG_ERR_UNSUPPORTED;
        }
    }
    // stream the payload through a pinned buffer, hashing and checking ids
    const size_t chunk = (size_t)64 << 20;
    unsigned char *stage = nullptr;
    if (cudaMallocHost(&stage, chunk) != cudaSuccess) {
        std::fclose(f);
        sqg_index_free(ix);
        return SQG_ERR_OOM;
    }
    uint64_t hash = sqg_fmt::kFnvBasis;
    int rc = SQG_OK;
    // rotation + padding
    {
        const size_t nbytes = L.blocks_offset - L.rot_offset;
        std::vector<unsigned char> buf(nbytes);
        if (std::fread(buf.data(), 1, nbytes, f) != nbytes) rc = SQG_ERR_IO;
        else {
            hash = sqg_fmt::fnv_words(hash, buf.data(), nbytes);
            if (cudaMemcpy(ix->d_rot, buf.data(), sizeof(float) * (size_t)L.d * L.d, cudaMemcpyHostToDevice) !=
                    cudaSuccess ||
                launch_split_tf32(ix->d_rot, ix->d_rot_hi, ix->d_rot_lo, (size_t)L.d * L.d, 0) != cudaSuccess ||
                cudaDeviceSynchronize() != cudaSuccess)
                rc = SQG_ERR_CUDA;
        }
    }
    const size_t per_chunk = std::max<size_t>(1, chunk / L.block_bytes);
    std::vector<uint32_t> ids(L.R);
    for (uint64_t v0 = 0; rc == SQG_OK && v0 < L.n; v0 += per_chunk) {
        const uint64_t nv = std::min<uint64_t>(per_chunk, L.n - v0);
        const size_t nbytes = nv * L.block_bytes;
        if (std::fread(stage, 1, nbytes, f) != nbytes) { rc = SQG_ERR_IO; break; }
        hash = sqg_fmt::fnv_words(hash, stage, nbytes);
        for (uint64_t t = 0; t < nv && rc == SQG_OK; ++t) {
            const unsigned char *b = stage + t * L.block_bytes + L.off_ids;
            for (uint32_t j = 0; j < L.R; ++j) ids[j] = sqg_fmt::load_u32(b + 4 * j);
            std::sort(ids.begin(), ids.end());
            for (uint32_t j = 0; j < L.R; ++j)  // SQG_NO_ID (sorted last, repeats allowed): an empty slot
                if (ids[j] != SQG_NO_ID &&
                    (ids[j] >= L.n || ids[j] == v0 + t || (j > 0 && ids[j] == ids[j - 1])))
                    rc = SQG_ERR_FORMAT;
        }
        if (rc == SQG_OK && cudaMemcpy(ix->d_blocks + v0 * L.block_bytes, stage, nbytes, cudaMemcpyHostToDevice) !=
                                cudaSuccess)
            rc = SQG_ERR_CUDA;
    }
    cudaFreeHost(stage);
    std::fclose(f);
    if (rc == SQG_OK && hash != h.payload_hash) rc = SQG_ERR_FORMAT;
    if (rc != SQG_OK) {
        sqg_index_free(ix);
        return rc;
    }
    *out = ix;
    return SQG_OK;
}

extern "C" void sqg_index_free(sqg_index *ix) {
    if (!ix) return;
    DeviceGuard g(ix->device);
    cudaDeviceSynchronize();
    if (ix->d_blocks) cudaFree(ix->d_blocks);
    if (ix->d_rot) cudaFree(ix->d_rot);
    if (ix->d_rot_hi) cudaFree(ix->d_rot_hi);
    if (ix->d_rot_lo) cudaFree(ix->d_rot_lo);
    if (ix->d_signs) cudaFree(ix->d_signs);
    if (ix->d_status) cudaFree(ix->d_status);
    delete ix;
}

extern "C" int sqg_index_info(const sqg_index *ix, sqg_info *out) {
    if (!ix || !out) return SQG_ERR_INVALID_ARG;
    out->n = ix->lay.n;
    out->d = ix->lay.d;
    out->degree = ix->lay.R;
    out->block_bytes = ix->lay.block_bytes;
    out->entry = ix->entry;
    out->off_codes = ix->lay.off_codes;
    out->off_factors = ix->lay.off_factors;
    out->off_ids = ix->lay.off_ids;
    out->device = ix->device;
    out->device_bytes = (uint64_t)ix->lay.n * ix->lay.block_bytes + 4ull * ix->lay.d * ix->lay.d + 4;
    out->metric = ix->cosine ? sqg_fmt::kMetricCosine : sqg_fmt::kMetricL2;
    out->version = ix->version;
    return SQG_OK;
}

extern "C" size_t sqg_workspace_size(const sqg_index *ix, int nq, int max_k, int max_ef) {
    if (!ix || nq < 0 || max_k < 1 || max_k > SQG_MAX_K || max_ef < max_k || max_ef > SQG_MAX_EF) return 0;
    DeviceGuard g(ix->device);
    // the larger of the plans without and with the learned stop's weights
    LaunchPlan pl;
    sqg_search_params p = default_params();
    if (make_plan(ix, nq, max_k, max_ef, p, pl) != SQG_OK) return 0;
    size_t need = pl.ws_total;
    p.kernel = 1;  // the general kernel (its visited tables follow its own residency)
    if (make_plan(ix, nq, max_k, max_ef, p, pl) == SQG_OK) need = std::max(need, pl.ws_total);
    p.stop_mlp = reinterpret_cast<const float *>(16);  // any non-null: only the layout is planned
    if (make_plan(ix, nq, max_k, max_ef, p, pl) == SQG_OK) need = std::max(need, pl.ws_total);
    p.kernel = 0;  // the compact kernel's build with the stop fused
    if (make_plan(ix, nq, max_k, max_ef, p, pl) == SQG_OK) need = std::max(need, pl.ws_total);
    return need;
}

extern "C" size_t sqg_workspace_size_ex(const sqg_index *ix, int nq, int max_k, int max_ef,
                                        const sqg_search_params *params) {
    if (!ix || nq < 0 || max_k < 1 || max_k > SQG_MAX_K || max_ef < max_k || max_ef > SQG_MAX_EF) return 0;
    sqg_search_params p = params ? *params : default_params();
    if (params && p.stop_every == 0) p.stop_every = 1;
    if (check_params(p) != SQG_OK) return 0;
    DeviceGuard g(ix->device);
    LaunchPlan pl;
    if (make_plan(ix, nq, max_k, max_ef, p, pl) != SQG_OK) return 0;
    return pl.ws_total;
}

static int search_impl(const sqg_index *ix, const float *queries, int nq, const int32_t *k, const int32_t *ef,
                       uint32_t *out_ids, float *out_dists, const sqg_search_params *params, void *workspace,
                       size_t ws_bytes, sqg_query_stats *stats, cudaStream_t stream, float *trace_feat,
                       int32_t *trace_hit, int32_t *trace_n, int trace_cap, const uint32_t *gt, int gt_k,
                       uint32_t *path = nullptr, int path_cap = 0) {
    if (!ix || nq < 0) return SQG_ERR_INVALID_ARG;
    if (nq == 0) return SQG_OK;
    if (!queries || !k || !ef || !out_ids || !out_dists) return SQG_ERR_INVALID_ARG;
    if (!aligned(queries, 16) || (workspace && !aligned(workspace, 256))) return SQG_ERR_INVALID_ARG;
    sqg_search_params p = params ? *params : default_params();
    if (params && p.stop_every == 0) p.stop_every = 1;
    if (check_params(p) != SQG_OK) return SQG_ERR_INVALID_ARG;
    if (trace_feat && p.team != 0 && p.team != 32) return SQG_ERR_UNSUPPORTED;  // the trace uses whole warps
    DeviceGuard g(ix->device);
    cudaError_t e;
    int max_k = p.max_k, max_ef = p.max_ef;
    if (p.uniform_k > 0) {
        if (max_k == 0) max_k = p.uniform_k;
        if (max_k != p.uniform_k) return SQG_ERR_INVALID_ARG;
    }
    if (max_k == 0 || max_ef == 0) {  // read the batch's bounds (one stream sync)
        void *tmp = nullptr;
        if (cudaMallocAsync(&tmp, 8 * (size_t)nq + 256, stream) != cudaSuccess) return SQG_ERR_OOM;
        int *maxes = reinterpret_cast<int *>(reinterpret_cast<char *>(tmp) + align_up(8 * (size_t)nq, 256));
        plan_kernel<<<1, kPlanThreads, 0, stream>>>(k, ef, nq, reinterpret_cast<long long *>(tmp), maxes);
        int hm[2] = {0, 0};
        e = cudaMemcpyAsync(hm, maxes, sizeof(hm), cudaMemcpyDeviceToHost, stream);
        cudaError_t e2 = cudaStreamSynchronize(stream);
        cudaFreeAsync(tmp, stream);
        if (e != cudaSuccess || e2 != cudaSuccess) return SQG_ERR_CUDA;
        if (max_k == 0) max_k = std::max(1, hm[0]);
        if (max_ef == 0) max_ef = std::max(max_k, hm[1]);
    }
    LaunchPlan pl;
    int rc = make_plan(ix, nq, max_k, max_ef, p, pl, trace_feat != nullptr || path != nullptr);
    if (rc != SQG_OK) return rc;
    bool own_ws = false;
    if (!workspace) {
        if (cudaMallocAsync(&workspace, pl.ws_total, stream) != cudaSuccess) return SQG_ERR_OOM;
        own_ws = true;
    } else if (ws_bytes < pl.ws_total) {
        return SQG_ERR_CAPACITY;
    }
    char *ws = reinterpret_cast<char *>(workspace);
    queries = queries_for(ix, queries, nq, reinterpret_cast<float *>(ws + pl.ws_qnorm), stream, &e);
    if (e != cudaSuccess) {
        if (own_ws) cudaFreeAsync(workspace, stream);
        return SQG_ERR_CUDA;
    }
    SearchArgs &a = pl.a;
    a.blocks = ix->d_blocks;
    a.block_bytes = ix->lay.block_bytes;
    a.n = (uint32_t)ix->lay.n;
    a.d = ix->lay.d;
    a.R = ix->lay.R;
    a.entry = ix->entry;
    a.off_codes = ix->lay.off_codes;
    a.off_factors = ix->lay.off_factors;
    a.off_ids = ix->lay.off_ids;
    a.queries = queries;
    a.qrot = reinterpret_cast<float *>(ws + pl.ws_qrot);
    a.nq = nq;
    a.k = k;
    a.ef = ef;
    a.offsets = reinterpret_cast<long long *>(ws + pl.ws_offsets);
    a.out_ids = out_ids;
    a.out_dists = out_dists;
    a.stats = stats ? stats : reinterpret_cast<sqg_query_stats *>(ws + pl.ws_stats);
    a.status_word = ix->d_status;
    a.queue_head = reinterpret_cast<unsigned int *>(ws + pl.ws_queue);
    a.max_k = max_k;
    a.max_ef = max_ef;
    a.hop_cap = p.hop_cap;
    a.ghash = pl.ghash ? reinterpret_cast<uint32_t *>(ws + pl.ws_ghash) : nullptr;
    a.eps0 = p.eps0;
    a.multi_estimate = p.multi_estimate;
    a.mlp = nullptr;
    if (p.stop_mlp) {
        float *t = reinterpret_cast<float *>(ws + pl.ws_mlp);
        mlp_transpose_kernel<<<1, 256, 0, stream>>>(p.stop_mlp, t);
        a.mlp = t;
    }
    a.stop_logit = p.stop_logit;
    a.stop_every = p.stop_every;
    a.stop_magic = p.stop_every >= 2 ? ~0ull / (uint64_t)p.stop_every + 1ull : 0ull;
    a.prefetch = p.prefetch == 0 ? 1 : p.prefetch;
    a.trace_feat = trace_feat;
    a.trace_hit = trace_hit;
    a.trace_n = trace_n;
    a.trace_cap = trace_cap;
    a.gt = gt;
    a.gt_k = gt_k;
    a.path = path;
    a.path_cap = path_cap;
    a.uniform_k = p.uniform_k;

    if (p.uniform_k == 0)  // ragged outputs: the offsets are the prefix sum of k[]
        plan_kernel<<<1, kPlanThreads, 0, stream>>>(k, ef, nq, const_cast<long long *>(a.offsets),
                                                    reinterpret_cast<int *>(ws + pl.ws_maxes));
    if (use_tc_rotation(ix, p)) {  // tensor cores, then the exact quantization
        a.qplanes = reinterpret_cast<uint32_t *>(ws + pl.ws_planes);
        a.qscal = reinterpret_cast<float4 *>(ws + pl.ws_scal);
        e = launch_rotate_tc(queries, ix->d_rot_hi, ix->d_rot_lo, const_cast<float *>(a.qrot), nq, (int)ix->lay.d,
                             ix->d_status, stream);
        if (e == cudaSuccess)
            e = launch_quantize_exact(queries, ix->d_rot, a.qrot, nq, (int)ix->lay.d,
                                      const_cast<uint32_t *>(a.qplanes), const_cast<float4 *>(a.qscal), nullptr,
                                      false, stream);
        if (e != cudaSuccess) {
            if (own_ws) cudaFreeAsync(workspace, stream);
            return SQG_ERR_CUDA;
        }
    } else if (rotate_simt(ix, queries, const_cast<float *>(a.qrot), nq, stream) != cudaSuccess) {
        if (own_ws) cudaFreeAsync(workspace, stream);
        return SQG_ERR_CUDA;
    }
    e = cudaMemsetAsync(a.queue_head, 0, sizeof(unsigned int), stream);
    if (e == cudaSuccess && p.timing_events[0])
        e = cudaEventRecord(reinterpret_cast<cudaEvent_t>(p.timing_events[0]), stream);
    if (e == cudaSuccess) {
        e = pl.compact && (pl.cbnb == 8 || pl.crk == 4)
                ? launch_search_compact_big(pl.ch, pl.nb, pl.cbnb, pl.crk, p.stop_mlp != nullptr, dim3(pl.grid),
                                            dim3(pl.warps * 32), pl.smem, stream, a)
            : pl.compact && p.stop_mlp
                ? launch_search_compact_stop(pl.ch, pl.nb, pl.cbnb, dim3(pl.grid), dim3(pl.warps * 32), pl.smem,
                                             stream, a)
            : pl.compact ? launch_search_compact(pl.ch, pl.nb, pl.cbnb, p.lean, dim3(pl.grid), dim3(pl.warps * 32),
                                                 pl.smem, stream, a)
            : pl.team < 32 ? launch_search_team(pl.ch, pl.nb, pl.team, dim3(pl.grid), dim3(pl.warps * 32), pl.smem,
                                                stream, a)
            : pl.nb == 1 ? launch_search_nb1(pl.ch, dim3(pl.grid), dim3(pl.warps * 32), pl.smem, stream, a)
                         : launch_search_nb2(pl.ch, dim3(pl.grid), dim3(pl.warps * 32), pl.smem, stream, a);
    }
    if (e == cudaSuccess && p.timing_events[1])
        e = cudaEventRecord(reinterpret_cast<cudaEvent_t>(p.timing_events[1]), stream);
    if (own_ws) cudaFreeAsync(workspace, stream);
    if (e != cudaSuccess) return SQG_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? SQG_OK : SQG_ERR_CUDA;
}

extern "C" int sqg_search(const sqg_index *ix, const float *queries, int nq, const int32_t *k, const int32_t *ef,
                          uint32_t *out_ids, float *out_dists, sqg_stream_t stream) {
    return search_impl(ix, queries, nq, k, ef, out_ids, out_dists, nullptr, nullptr, 0, nullptr,
                       reinterpret_cast<cudaStream_t>(stream), nullptr, nullptr, nullptr, 0, nullptr, 0);
}

extern "C" int sqg_search_ex(const sqg_index *ix, const float *queries, int nq, const int32_t *k,
                             const int32_t *ef, uint32_t *out_ids, float *out_dists,
                             const sqg_search_params *params, void *workspace, size_t ws_bytes,
                             sqg_query_stats *stats, sqg_stream_t stream) {
    return search_impl(ix, queries, nq, k, ef, out_ids, out_dists, params, workspace, ws_bytes, stats,
                       reinterpret_cast<cudaStream_t>(stream), nullptr, nullptr, nullptr, 0, nullptr, 0);
}

extern "C" int sqg_search_trace(const sqg_index *ix, const float *queries, int nq, const int32_t *k,
                                const int32_t *ef, uint32_t *out_ids, float *out_dists,
                                const sqg_search_params *params, sqg_query_stats *stats, const uint32_t *gt,
                                int gt_k, float *trace_feat, int32_t *trace_hit, int32_t *trace_n, int trace_cap,
                                uint32_t *path, int path_cap, sqg_stream_t stream) {
    if (trace_feat && (!trace_n || trace_cap < 1)) return SQG_ERR_INVALID_ARG;
    if (gt && (!trace_feat || !trace_hit || gt_k < 1)) return SQG_ERR_INVALID_ARG;
    if ((path && path_cap < 1) || (!path && !trace_feat)) return SQG_ERR_INVALID_ARG;
    if (!trace_feat) trace_cap = 0;
    return search_impl(ix, queries, nq, k, ef, out_ids, out_dists, params, nullptr, 0, stats,
                       reinterpret_cast<cudaStream_t>(stream), trace_feat, trace_hit, trace_n, trace_cap, gt, gt_k,
                       path, path ? path_cap : 0);
}

extern "C" int sqg_prepare_queries(const sqg_index *ix, const float *queries, int nq, float *out_qrot,
                                   uint32_t *out_planes, float *out_scal, sqg_stream_t stream_) {
    if (!ix || nq < 0) return SQG_ERR_INVALID_ARG;
    if (nq == 0) return SQG_OK;
    if (!queries || !out_qrot || !out_planes || !out_scal) return SQG_ERR_INVALID_ARG;
    if (!aligned(queries, 16) || !aligned(out_qrot, 16) || !aligned(out_planes, 16) || !aligned(out_scal, 16))
        return SQG_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    DeviceGuard g(ix->device);
    const int d = (int)ix->lay.d;
    float *qn = nullptr;
    if (ix->cosine && cudaMallocAsync(&qn, sizeof(float) * (size_t)nq * d, stream) != cudaSuccess)
        return SQG_ERR_OOM;
    cudaError_t e;
    queries = queries_for(ix, queries, nq, qn, stream, &e);
    if (e == cudaSuccess) e = rotate_simt(ix, queries, out_qrot, nq, stream);
    if (qn) cudaFreeAsync(qn, stream);
    if (e != cudaSuccess) return SQG_ERR_CUDA;
    const int wpb = 4;
    quantize_kernel<<<(nq + wpb - 1) / wpb, wpb * 32, sizeof(uint32_t) * wpb * 4 * (d / 32), stream>>>(
        out_qrot, nq, d, out_planes, out_scal);
    return cudaGetLastError() == cudaSuccess ? SQG_OK : SQG_ERR_CUDA;
}

extern "C" int sqg_prepare_queries_tc(const sqg_index *ix, const float *queries, int nq, float *out_qrot,
                                      uint32_t *out_planes, float *out_scal, uint32_t *recomputed,
                                      sqg_stream_t stream_) {
    if (!ix || nq < 0) return SQG_ERR_INVALID_ARG;
    if (nq == 0) return SQG_OK;
    if (!queries || !out_qrot || !out_planes || !out_scal || !recomputed) return SQG_ERR_INVALID_ARG;
    if (!aligned(queries, 16) || !aligned(out_qrot, 16) || !aligned(out_planes, 16) || !aligned(out_scal, 16))
        return SQG_ERR_INVALID_ARG;
    if (ix->fjlt) return SQG_ERR_UNSUPPORTED;  // the fast JLT has no dense contraction to put on tensor cores
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    DeviceGuard g(ix->device);
    const int d = (int)ix->lay.d;
    float *qn = nullptr;
    if (ix->cosine && cudaMallocAsync(&qn, sizeof(float) * (size_t)nq * d, stream) != cudaSuccess)
        return SQG_ERR_OOM;
    cudaError_t e;
    queries = queries_for(ix, queries, nq, qn, stream, &e);
    if (e == cudaSuccess)
        e = launch_rotate_tc(queries, ix->d_rot_hi, ix->d_rot_lo, out_qrot, nq, d, ix->d_status, stream);
    if (e == cudaSuccess)
        e = launch_quantize_exact(queries, ix->d_rot, out_qrot, nq, d, out_planes,
                                  reinterpret_cast<float4 *>(out_scal), recomputed, true, stream);
    if (qn) cudaFreeAsync(qn, stream);
    return e == cudaSuccess ? SQG_OK : SQG_ERR_CUDA;
}

extern "C" int sqg_estimate_block(const sqg_index *ix, const float *queries, int nq, const uint32_t *v,
                                  float eps0, int32_t *out_S, float *out_est, float *out_key, float *out_dist_c,
                                  sqg_stream_t stream_) {
    if (!ix || nq < 0 || !std::isfinite(eps0)) return SQG_ERR_INVALID_ARG;
    if (nq == 0) return SQG_OK;
    if (!queries || !v || !out_S || !out_est || !out_key || !out_dist_c) return SQG_ERR_INVALID_ARG;
    if (!aligned(queries, 16)) return SQG_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    DeviceGuard g(ix->device);
    const int d = (int)ix->lay.d;
    float *qrot = nullptr;  // q', then on a cosine index the unit-norm queries after it
    const size_t qbytes = sizeof(float) * (size_t)nq * d;
    if (cudaMallocAsync(&qrot, ix->cosine ? 2 * qbytes : qbytes, stream) != cudaSuccess) return SQG_ERR_OOM;
    cudaError_t qe;
    queries = queries_for(ix, queries, nq, qrot + (size_t)nq * d, stream, &qe);
    if (qe != cudaSuccess || rotate_simt(ix, queries, qrot, nq, stream) != cudaSuccess) {
        cudaFreeAsync(qrot, stream);
        return SQG_ERR_CUDA;
    }
    SearchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.blocks = ix->d_blocks;
    a.block_bytes = ix->lay.block_bytes;
    a.n = (uint32_t)ix->lay.n;
    a.d = ix->lay.d;
    a.R = ix->lay.R;
    a.off_codes = ix->lay.off_codes;
    a.off_factors = ix->lay.off_factors;
    a.off_ids = ix->lay.off_ids;
    a.queries = queries;
    a.qrot = qrot;
    a.nq = nq;
    a.eps0 = eps0;
    a.warp_bytes = (uint32_t)align_up(ix->lay.block_bytes + 16 * (d / 32), 16);
    const int wpb = 2;
    const size_t smem = (size_t)wpb * a.warp_bytes;
    cudaError_t e = cudaFuncSetAttribute(estimate_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        estimate_block_kernel<<<(nq + wpb - 1) / wpb, wpb * 32, smem, stream>>>(a, v, out_S, out_est, out_key,
                                                                               out_dist_c);
        e = cudaGetLastError();
    }
    cudaFreeAsync(qrot, stream);
    return e == cudaSuccess ? SQG_OK : SQG_ERR_CUDA;
}

extern "C" int sqg_get_status(const sqg_index *ix, sqg_stream_t stream_, uint32_t *status) {
    if (!ix || !status) return SQG_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    DeviceGuard g(ix->device);
    uint32_t h = 0;
    if (cudaMemcpyAsync(&h, ix->d_status, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaMemsetAsync(ix->d_status, 0, sizeof(uint32_t), stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return SQG_ERR_CUDA;
    *status = h;
    return SQG_OK;
}
