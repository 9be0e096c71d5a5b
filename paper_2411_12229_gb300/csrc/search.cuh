// search.cuh -- device code of the SymphonyQG query phase for sm_103a.
//
// One warp serves one query at a time and pulls the next query index from a
// device work queue (persistent kernel).  Per query it runs Algorithm 1
// (Querying, Sec. 3.1.3) with multiple estimated distances and implicit
// re-ranking (Sec. 3.1.2):
//
//   select   the first unvisited beam entry (beam sorted by (key, id));
//   fetch    the vertex's block -- raw vector, neighbour codes and factors,
//            neighbour ids (Sec. 3.1.3) -- by one 1-D bulk copy
//            (cp.async.bulk) into shared memory; the NEXT vertex's block is
//            copied while the current one is merged (memory prefetching,
//            Sec. 3.1.4); the kernel alternates two buffer slots with their
//            own mbarriers, which the launch plan may point at one buffer
//            (every read of a block precedes the next copy);
//   exact    the squared distance from the raw vector updates the result
//            set (implicit re-ranking);
//   estimate every neighbour's distance: S = sum_i b_i qbar_i by AND +
//            __popc against 4 bit-planes of the quantized rotated query,
//            est = f_add + dist_c + f_rescale * ip (Eq. (2) with Eq. (5)-(6));
//   admit    every unvisited neighbour enters the beam, duplicates of an id
//            included, and the beam is cut to ef (Algorithm 1, line 6).
//
// Float decisions follow a fixed operation order (explicit __f*_rn
// intrinsics; the file is built with -fmad=false), so that the CPU oracle
// can take the same decisions bit for bit.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sqg.h"

namespace sqg {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kVisited = 0x80000000u;
constexpr uint32_t kIdMask = 0x7FFFFFFFu;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s per bounded wait

struct SearchArgs {
    const unsigned char *blocks;
    uint32_t block_bytes, n, d, R, entry;
    uint32_t off_codes, off_factors, off_ids;
    const float *queries;  // nq x d
    const float *qrot;     // nq x d, P^-1 q
    int nq;
    const int32_t *k, *ef;
    const long long *offsets;  // nq: output offset of each query
    uint32_t *out_ids;
    float *out_dists;
    sqg_query_stats *stats;  // nq or null
    uint32_t *status_word;   // OR of all status bits
    unsigned int *queue_head;
    int max_k, max_ef, hop_cap;
    int uniform_k;        // > 0: every k[i] equals it, outputs at i * uniform_k (offsets unused)
    uint32_t hash_bits;   // full visited table: 2^hash_bits >= 2 * hop cap + 1
    uint32_t shash_bits;  // shared-memory table (<= hash_bits)
    uint32_t *ghash;      // per-warp full tables in global memory when shash_bits < hash_bits
    float eps0;
    int multi_estimate;
    const float *mlp;       // the stop network with W1, W2 transposed to [in][out], or null
    float stop_logit;
    int stop_every;
    uint64_t stop_magic;  // 2^64 / stop_every + 1 for stop_every >= 2 (hops mod stop_every by a multiply)
    int prefetch;       // 1: next block only; 2: also L2-prefetch the runner-up
    float *trace_feat;  // nq x trace_cap x 16, or null
    int32_t *trace_hit; // nq x trace_cap
    int32_t *trace_n;   // nq
    int trace_cap;
    const uint32_t *gt; // nq x gt_k ground-truth ids (trace mode)
    int gt_k;
    const uint32_t *qplanes;  // nq x d/32 x 4 precomputed bit-planes ([w][b]), or null: quantize qrot
    const float4 *qscal;      // nq: (v_l, delta, Sq, 1/sqrt(d)) with qplanes
    uint32_t *path;     // nq x path_cap: ids of the first expanded vertices, or null
    int path_cap;
    uint32_t warp_bytes, cta_bytes;
    uint32_t o_buf0, o_buf1, o_bar, o_beam, o_hash, o_res, o_planes, o_spos;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Lane 0 only: arm the barrier for `bytes` and start the 1-D bulk copy.
__device__ __forceinline__ void bulk_fetch(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// try_wait that may suspend the warp for up to `hint_ns` (it resumes as soon
// as the phase completes), so a waiting warp does not spin on issue slots.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of `bar`; false on timeout (never hangs).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait_suspend(bar, parity, 200000u)) return true;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
}

// ---------------------------------------------------------------- ordering
__device__ __forceinline__ bool kless(float ka, uint32_t ia, float kb, uint32_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// ---------------------------------------------------------------- hash set
__device__ __forceinline__ uint32_t hslot(uint32_t id, uint32_t bits) { return (id * 0x9E3779B1u) >> (32 - bits); }
__device__ __forceinline__ void hash_insert(uint32_t *H, uint32_t bits, uint32_t id) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t s = hslot(id, bits);
    for (;;) {
        uint32_t v = H[s];
        if (v == id) return;
        if (v == kEmpty) { H[s] = id; return; }
        s = (s + 1) & mask;
    }
}
// ---------------------------------------------------------------- teams
// A team of T lanes (T = 32, 16 or 8) serves one query; a warp holds 32/T
// teams that run side by side.  Every collective below is scoped to the
// team: ballots return the team's T bits, shuffles address lanes within it.
template <int T>
struct Team {
    static_assert(T == 32 || T == 16 || T == 8, "team of 32, 16 or 8 lanes");
    static constexpr int V = 32 / T;  // lanes of the canonical 32-lane order each lane stands for
    uint32_t mask;  // the team's lanes in the warp
    int tl;         // lane within the team
    int base;       // the team's first lane
    __device__ __forceinline__ explicit Team(int lane) {
        tl = lane & (T - 1);
        base = lane & ~(T - 1);
        if constexpr (T == 32) mask = kFull;
        else mask = ((1u << T) - 1u) << base;
    }
    __device__ __forceinline__ uint32_t ballot(bool p) const {
        const uint32_t b = __ballot_sync(mask, p);
        if constexpr (T == 32) return b;
        else return (b >> base) & ((1u << T) - 1u);
    }
    template <class X>
    __device__ __forceinline__ X shfl(X v, int src) const {
        return __shfl_sync(mask, v, src, T);
    }
    template <class X>
    __device__ __forceinline__ X shfl_xor(X v, int o) const {
        return __shfl_xor_sync(mask, v, o, T);
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    __device__ __forceinline__ int reduce_min(int v) const { return __reduce_min_sync(mask, v); }
    __device__ __forceinline__ int reduce_add(int v) const { return __reduce_add_sync(mask, v); }
};

// Team: move every id of the shared table `S` into the cleared global table
// `G` (concurrent inserts by compare-and-swap).
template <int T>
__device__ __forceinline__ void hash_migrate(const uint32_t *S, uint32_t sbits, uint32_t *G, uint32_t gbits,
                                             const Team<T> &tm) {
    const uint32_t gsize = 1u << gbits, gmask = gsize - 1u;
    for (uint32_t i = tm.tl; i < gsize; i += T) G[i] = kEmpty;
    tm.sync();
    for (uint32_t i = tm.tl; i < (1u << sbits); i += T) {
        const uint32_t id = S[i];
        if (id == kEmpty) continue;
        uint32_t s = hslot(id, gbits);
        while (atomicCAS(&G[s], kEmpty, id) != kEmpty) s = (s + 1) & gmask;
    }
    tm.sync();
}
__device__ __forceinline__ bool hash_contains(const uint32_t *H, uint32_t bits, uint32_t id) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t s = hslot(id, bits);
    for (;;) {
        uint32_t v = H[s];
        if (v == id) return true;
        if (v == kEmpty) return false;
        s = (s + 1) & mask;
    }
}

// ---------------------------------------------------------------- query side
// 4-bit uniform quantization of q' = P^-1 q over [v_l, v_r] (Sec. 3.1.1 with
// the 4-bit reading): qbar_i = min(15, trunc((q'_i - v_l)*15/(v_r-v_l) + 0.5));
// bit b of every qbar_i is packed into plane b by a warp ballot.
struct QuerySide {
    float vl, delta, inv_sqrt_d;
    int sq;
};
// Team T: coordinate 32w + tl + T v belongs to lane tl (v < 32/T); the
// planes' word w is assembled from the 32/T team ballots.
template <int T>
__device__ __forceinline__ QuerySide quantize_team(const float *qr, uint32_t d, uint32_t *planes, const Team<T> &tm) {
    constexpr int V = Team<T>::V;
    const uint32_t nw = d / 32;
    float vl = __int_as_float(0x7f800000), vr = -vl;
    for (uint32_t w = 0; w < nw; ++w) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float x = qr[w * 32 + tm.tl + T * v];
            vl = x < vl ? x : vl;
            vr = x > vr ? x : vr;
        }
    }
#pragma unroll
    for (int o = T / 2; o >= 1; o >>= 1) {
        const float a = tm.shfl_xor(vl, o), b = tm.shfl_xor(vr, o);
        vl = a < vl ? a : vl;
        vr = b > vr ? b : vr;
    }
    const float range = __fsub_rn(vr, vl);
    QuerySide qs;
    qs.vl = vl;
    qs.delta = range > 0.0f ? __fdiv_rn(range, 15.0f) : 0.0f;
    const float inv = range > 0.0f ? __fdiv_rn(15.0f, range) : 0.0f;
    qs.inv_sqrt_d = __fdiv_rn(1.0f, __fsqrt_rn((float)d));
    int sq = 0;
    for (uint32_t w = 0; w < nw; ++w) {
        uint32_t b0 = 0, b1 = 0, b2 = 0, b3 = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            int t = 0;
            if (range > 0.0f) {
                float x = __fsub_rn(qr[w * 32 + tm.tl + T * v], vl);
                x = __fmul_rn(x, inv);
                x = __fadd_rn(x, 0.5f);
                t = __float2int_rz(x);
                t = t > 15 ? 15 : t;
            }
            sq += t;
            b0 |= tm.ballot(t & 1) << (T * v);
            b1 |= tm.ballot(t & 2) << (T * v);
            b2 |= tm.ballot(t & 4) << (T * v);
            b3 |= tm.ballot(t & 8) << (T * v);
        }
        if (tm.tl == 0) {
            // word-major: the 4 planes of word w share one 16-byte slot
            reinterpret_cast<uint4 *>(planes)[w] = make_uint4(b0, b1, b2, b3);
        }
    }
    qs.sq = tm.reduce_add(sq);
    return qs;
}
__device__ __forceinline__ QuerySide quantize_warp(const float *qr, uint32_t d, uint32_t *planes, int lane) {
    return quantize_team<32>(qr, d, planes, Team<32>(lane));
}

// Exact squared distance in the canonical order: lane l of 32 sums float4
// chunks l, l+32, ... (x, y, z, w; fmaf(d, d, acc) from 0), then an xor
// butterfly adds partials l and l^16, ^8, ^4, ^2, ^1.  A team of T lanes
// keeps the 32/T partials of lanes tl + T v in registers: butterfly steps of
// at least T combine registers, the smaller ones shuffle, and every step
// adds the same two partials as the 32-lane order, so the result is equal.
template <int CH, int T>
__device__ __forceinline__ void exact_partial(const float4 (&qv)[32 / T][CH], const float *raw, uint32_t nch,
                                              const Team<T> &tm, float (&acc)[32 / T]) {
    constexpr int V = 32 / T;
    const float4 *r4 = reinterpret_cast<const float4 *>(raw);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        acc[v] = 0.0f;
#pragma unroll
        for (int t = 0; t < CH; ++t) {
            const uint32_t c = tm.tl + T * v + 32 * t;
            if (c < nch) {
                const float4 x = r4[c];
                const float dx = __fsub_rn(qv[v][t].x, x.x), dy = __fsub_rn(qv[v][t].y, x.y);
                const float dz = __fsub_rn(qv[v][t].z, x.z), dw = __fsub_rn(qv[v][t].w, x.w);
                acc[v] = __fmaf_rn(dx, dx, acc[v]);
                acc[v] = __fmaf_rn(dy, dy, acc[v]);
                acc[v] = __fmaf_rn(dz, dz, acc[v]);
                acc[v] = __fmaf_rn(dw, dw, acc[v]);
            }
        }
    }
}
template <int T>
__device__ __forceinline__ float exact_reduce(float (&acc)[32 / T], const Team<T> &tm) {
    constexpr int V = 32 / T;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (o >= T) {
            float nx[V];
#pragma unroll
            for (int v = 0; v < V; ++v) nx[v] = __fadd_rn(acc[v], acc[v ^ (o / T)]);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = nx[v];
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = __fadd_rn(acc[v], tm.shfl_xor(acc[v], o));
        }
    }
    return acc[0];
}
template <int CH, int T>
__device__ __forceinline__ float exact_dist_team(const float4 (&qv)[32 / T][CH], const float *raw, uint32_t nch,
                                                 const Team<T> &tm) {
    float acc[32 / T];
    exact_partial<CH, T>(qv, raw, nch, tm, acc);
    return exact_reduce<T>(acc, tm);
}
template <int CH>
__device__ __forceinline__ float exact_dist(const float4 (&qv)[CH], const float *raw, uint32_t nch, int lane) {
    return exact_dist_team<CH, 32>(reinterpret_cast<const float4(&)[1][CH]>(qv), raw, nch, Team<32>(lane));
}

// RaBitQ estimate of neighbour j from its block (Sec. 3.1.1):
// S = sum_b 2^b popc(code & plane_b); ip = fmaf(delta, 2S-Sq, v_l(2pc-d))/sqrt(d);
// est = fmaf(f_rescale, ip, f_add + dist_c); key = est - eps0 * f_err sqrt(dist_c).
struct Est {
    int S;
    float est, key;
};
// S of neighbour j: integer, independent of dist_c, so a caller can overlap
// it with the exact distance's butterfly.  Up to d = 256 the word loop is
// unrolled and predicated (one basic block).
template <int CH>
__device__ __forceinline__ int estimate_S(const unsigned char *blk, const SearchArgs &a, const uint32_t *planes,
                                          uint32_t j) {
    const uint32_t nw = a.d / 32, R = a.R;
    const uint32_t *codes = reinterpret_cast<const uint32_t *>(blk + a.off_codes) + j;
    int s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    if constexpr (CH <= 2) {
#pragma unroll
        for (uint32_t w = 0; w < 4 * CH; ++w) {
            if (w < nw) {
                const uint32_t c = codes[w * R];
                const uint4 pl = reinterpret_cast<const uint4 *>(planes)[w];
                s0 += __popc(c & pl.x);
                s1 += __popc(c & pl.y);
                s2 += __popc(c & pl.z);
                s3 += __popc(c & pl.w);
            }
        }
    } else {
#pragma unroll 4
        for (uint32_t w = 0; w < nw; ++w) {
            const uint32_t c = codes[w * R];
            const uint4 pl = reinterpret_cast<const uint4 *>(planes)[w];
            s0 += __popc(c & pl.x);
            s1 += __popc(c & pl.y);
            s2 += __popc(c & pl.z);
            s3 += __popc(c & pl.w);
        }
    }
    return s0 + 2 * s1 + 4 * s2 + 8 * s3;
}
// The estimate and key of neighbour j from its S.
// sqrt_dc = sqrtf(dist_c), computed once per expansion (used only when eps0 != 0).
__device__ __forceinline__ Est estimate_from_S(const unsigned char *blk, const SearchArgs &a, const QuerySide &qs,
                                               uint32_t j, int S, float dist_c, float sqrt_dc) {
    const uint32_t R = a.R;
    const float *fac = reinterpret_cast<const float *>(blk + a.off_factors);
    const float f_add = fac[j], f_rescale = fac[R + j];
    const int pc = (int)reinterpret_cast<const uint32_t *>(fac)[3 * R + j];
    const float A = (float)(2 * S - qs.sq);
    const float B = __fmul_rn(qs.vl, (float)(2 * pc - (int)a.d));
    const float ip = __fmul_rn(__fmaf_rn(qs.delta, A, B), qs.inv_sqrt_d);
    Est e;
    e.S = S;
    e.est = __fmaf_rn(f_rescale, ip, __fadd_rn(f_add, dist_c));
    if (a.eps0 == 0.0f) {
        e.key = e.est;  // est - 0 * bound, bound finite and >= 0
    } else {
        const float bound = __fmul_rn(fac[2 * R + j], sqrt_dc);
        e.key = __fsub_rn(e.est, __fmul_rn(a.eps0, bound));
    }
    return e;
}
__device__ __forceinline__ Est estimate(const unsigned char *blk, const SearchArgs &a, const uint32_t *planes,
                                        const QuerySide &qs, uint32_t j, float dist_c, float sqrt_dc) {
    return estimate_from_S(blk, a, qs, j, estimate_S<16>(blk, a, planes, j), dist_c, sqrt_dc);
}

// ---------------------------------------------------------------- learned stop
// Features of the search state (all IEEE +,-,*,/ so both sides agree).
struct StopState {
    int hops, last_improve, inserted_last;
    float ema_improve, ema_insert, dist_c;
};
__device__ __forceinline__ float clamp8(float x) { return x < -8.0f ? -8.0f : (x > 8.0f ? 8.0f : x); }

// MLP 16 -> 64 -> 64 -> 1 on one warp; lane l computes hidden neurons l and
// l + 32 of both layers.  The parameters are read from global memory (the
// same 21 KB for every warp, so they stay in L1) in a packed layout made once
// per call (mlp_pack_kernel), so that one 16-byte load gives a lane the
// weights of its two neurons for two consecutive inputs:
//   W1p[i2][l] = (W1[l][2i2], W1[l+32][2i2], W1[l][2i2+1], W1[l+32][2i2+1]),
//   b1p[l] = (b1[l], b1[l+32]), W2p[i2][l] likewise over the 64 inputs,
//   b2p[l], W3p[l] = (W3[l], W3[l+32]), then b3.
// Hidden neuron o is an fmaf chain over its inputs in order starting from
// its bias; the first layer's outputs pass to the second through `hbuf`
// (64 floats of the warp's shared memory); the output adds
// p_l = fmaf(W3[l+32], h[l+32], W3[l] h[l]) by xor butterfly, then b3.
// The features f come from registers (an array) or from shared memory (a
// pointer to SQG_MLP_IN floats the warp wrote before a __syncwarp); the
// arithmetic is the same.  From shared memory the loops are not unrolled,
// so that few registers are in flight (for builds at their register
// limit); from registers they are, for more loads in flight.
template <typename FV>
__device__ __forceinline__ float mlp_logit_warp(const float *w, const FV &f, int lane, float *hbuf) {
    constexpr bool kLean = std::is_pointer<FV>::value;
    const float4 *W1p = reinterpret_cast<const float4 *>(w);               // [8][32]
    const float2 *b1p = reinterpret_cast<const float2 *>(w + 8 * 32 * 4);  // [32]
    const float4 *W2p = reinterpret_cast<const float4 *>(w + 8 * 32 * 4 + 64);        // [32][32]
    const float2 *b2p = reinterpret_cast<const float2 *>(w + 8 * 32 * 4 + 64 + 32 * 32 * 4);
    const float2 *W3p = b2p + 32;
    const float *b3 = reinterpret_cast<const float *>(W3p + 32);
    const float2 bb1 = __ldg(b1p + lane);
    float ha = bb1.x, hb = bb1.y;
    auto layer1 = [&](int i2) {
        const float4 wv = __ldg(W1p + i2 * 32 + lane);
        ha = __fmaf_rn(wv.x, f[2 * i2], ha);
        hb = __fmaf_rn(wv.y, f[2 * i2], hb);
        ha = __fmaf_rn(wv.z, f[2 * i2 + 1], ha);
        hb = __fmaf_rn(wv.w, f[2 * i2 + 1], hb);
    };
    if constexpr (kLean) {
#pragma unroll 1
        for (int i2 = 0; i2 < SQG_MLP_IN / 2; ++i2) layer1(i2);
    } else {  // a register array: constant indices only
#pragma unroll
        for (int i2 = 0; i2 < SQG_MLP_IN / 2; ++i2) layer1(i2);
    }
    hbuf[lane] = ha > 0.0f ? ha : 0.0f;
    hbuf[lane + 32] = hb > 0.0f ? hb : 0.0f;
    __syncwarp();
    const float2 bb2 = __ldg(b2p + lane);
    float ga = bb2.x, gb = bb2.y;
    const float4 *h4 = reinterpret_cast<const float4 *>(hbuf);
    auto layer2 = [&](int i4) {
        const float4 h = h4[i4];
        const float4 w0 = __ldg(W2p + (2 * i4) * 32 + lane), w1 = __ldg(W2p + (2 * i4 + 1) * 32 + lane);
        ga = __fmaf_rn(w0.x, h.x, ga);
        gb = __fmaf_rn(w0.y, h.x, gb);
        ga = __fmaf_rn(w0.z, h.y, ga);
        gb = __fmaf_rn(w0.w, h.y, gb);
        ga = __fmaf_rn(w1.x, h.z, ga);
        gb = __fmaf_rn(w1.y, h.z, gb);
        ga = __fmaf_rn(w1.z, h.w, ga);
        gb = __fmaf_rn(w1.w, h.w, gb);
    };
    if constexpr (kLean) {
#pragma unroll 1
        for (int i4 = 0; i4 < 16; ++i4) layer2(i4);
    } else {
#pragma unroll 4
        for (int i4 = 0; i4 < 16; ++i4) layer2(i4);
    }
    __syncwarp();  // hbuf may be reused after this
    ga = ga > 0.0f ? ga : 0.0f;
    gb = gb > 0.0f ? gb : 0.0f;
    const float2 w3 = __ldg(W3p + lane);
    float p = __fmaf_rn(w3.y, gb, __fmul_rn(w3.x, ga));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) p = __fadd_rn(p, __shfl_xor_sync(kFull, p, o));
    return __fadd_rn(p, __ldg(b3));
}

// ---------------------------------------------------------------- the kernel
// LEAN: a build capped at 64 registers (8 resident blocks of 4 warps) for
// d <= 256, trading a few spills for more warps in flight.  T: lanes per
// query; a warp runs 32/T queries side by side, each team with its own
// shared-memory slot, work-queue loop and visited set, so the per-query
// serial steps (select, hash insert, merge bookkeeping) are shared by the
// warp's queries instead of idling lanes.
template <int CH, int NB, bool LEAN = false, int T = 32>
__global__ void __launch_bounds__(128, (LEAN ? 8 : (CH <= 2 ? 5 : 3))) search_kernel(const SearchArgs a) {
    constexpr int V = 32 / T;   // teams (queries) per warp
    constexpr int NT = NB * V;  // neighbours per lane
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Team<T> tm(lane);
    const int tl = tm.tl, team = lane / T;
    const uint32_t R = a.R, d = a.d, nch = d / 4;
    const float inv_R = __fdiv_rn(1.0f, (float)R);

    const float *wts = a.mlp;  // the stop network in its packed layout (global, L1-cached)

    unsigned char *ws = smem + a.cta_bytes + (size_t)(warp * V + team) * a.warp_bytes;
    unsigned char *buf[2] = {ws + a.o_buf0, ws + a.o_buf1};
    uint64_t *bar = reinterpret_cast<uint64_t *>(ws + a.o_bar);
    // beam and result: (key bits, id) pairs; bit 31 of a beam id marks an
    // expanded vertex
    uint2 *beam = reinterpret_cast<uint2 *>(ws + a.o_beam);
    uint2 *res = reinterpret_cast<uint2 *>(ws + a.o_res);
    uint32_t *planes = reinterpret_cast<uint32_t *>(ws + a.o_planes);
    const uint32_t gteam = (blockIdx.x * (blockDim.x >> 5) + warp) * V + team;
    // visited set: a shared-memory table, moved once to this team's global
    // table if a query's expansions fill half of it
    uint32_t *const Hs = reinterpret_cast<uint32_t *>(ws + a.o_hash);
    uint32_t *const Hg = a.ghash ? a.ghash + ((size_t)gteam << a.hash_bits) : nullptr;

    if (tl == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    fence_mbar_init();
    tm.sync();
    uint32_t phase = 0;     // bit b: parity of the next completion of bar[b]
    bool healthy = true;    // false after an unrecovered copy timeout

    while (healthy) {
        int qi = 0;
        if (tl == 0) qi = (int)atomicAdd(a.queue_head, 1u);
        qi = tm.shfl(qi, 0);
        if (qi >= a.nq) break;

        const int k = a.k[qi], ef = a.ef[qi];
        const long long off = a.uniform_k ? (long long)qi * a.uniform_k : a.offsets[qi];
        uint32_t status = 0;
        if (!(k >= 1 && k <= a.max_k && ef >= k && ef <= a.max_ef && (!a.uniform_k || k == a.uniform_k))) {
            const int kk = a.uniform_k ? a.uniform_k : (k < 0 ? 0 : (k > SQG_MAX_K ? SQG_MAX_K : k));
            for (int t = tl; t < kk; t += T) {
                a.out_ids[off + t] = SQG_NO_ID;
                a.out_dists[off + t] = __int_as_float(0x7f800000);
            }
            if (tl == 0) {
                if (a.stats) a.stats[qi] = sqg_query_stats{0u, SQG_STATUS_BAD_PARAM};
                atomicOr(a.status_word, SQG_STATUS_BAD_PARAM);
                if (a.trace_n) a.trace_n[qi] = 0;
            }
            continue;
        }
        const int hop_cap = a.hop_cap > 0 ? a.hop_cap : 4 * ef + 64;

        // ---- query setup: raw query in registers, quantized rotated query planes
        float4 qv[V][CH];
        const float *q = a.queries + (size_t)qi * d;
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int t = 0; t < CH; ++t) {
                const uint32_t c = tl + T * v + 32 * t;
                qv[v][t] = c < nch ? reinterpret_cast<const float4 *>(q)[c] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        QuerySide qs;
        if (a.qplanes) {  // quantized by the exact pass after the tensor-core rotation
            const uint4 *src = reinterpret_cast<const uint4 *>(a.qplanes + (size_t)qi * 4 * (d / 32));
            for (uint32_t w = tl; w < d / 32; w += T) reinterpret_cast<uint4 *>(planes)[w] = src[w];
            const float4 sc = a.qscal[qi];
            qs.vl = sc.x;
            qs.delta = sc.y;
            qs.sq = (int)sc.z;
            qs.inv_sqrt_d = sc.w;
        } else {
            qs = quantize_team<T>(a.qrot + (size_t)qi * d, d, planes, tm);
        }
        uint32_t *H = Hs;
        uint32_t hbits = a.shash_bits;
        for (uint32_t i = tl; i < (1u << hbits); i += T) H[i] = kEmpty;

        // ---- Algorithm 1, line 1: the beam and the result start from the entry
        int m = 1, cur = 0, rc = 0;
        if (tl == 0) {
            beam[0] = make_uint2(0u, a.entry);  // key: the entry's exact distance, set at its expansion
        }
        int cb = 0;                          // buffer holding the block to expand next
        uint32_t pend = a.entry;             // id whose block is in flight into buf[cb]
        bool inflight = true;
        tm.sync();
        if (tl == 0) {
            fence_proxy_async();
            bulk_fetch(buf[0], a.blocks + (size_t)a.entry * a.block_bytes, a.block_bytes, &bar[0]);
        }
        StopState st{0, 0, 0, 0.0f, 0.0f, 0.0f};
        int tn = 0;
        int hops = 0;

        while (cur < m) {
            if (hops >= hop_cap) { status |= SQG_STATUS_CAPACITY; break; }
            const uint32_t p = beam[cur].y & kIdMask;
            // one pass over [cur, m): mark every copy of p visited (copies lie
            // after cur, which is the first unvisited entry) and find the next
            // unvisited entry after cur
            int nxt = m;
            for (int base = cur; base < m; base += T) {
                const int i = base + tl;
                uint32_t v = kVisited;
                if (i < m) {
                    v = beam[i].y;
                    if ((v & kIdMask) == p) {
                        v = p | kVisited;
                        beam[i].y = v;
                    }
                }
                if (nxt == m) {
                    const uint32_t b = tm.ballot(i > cur && !(v & kVisited));
                    if (b) nxt = base + __ffs(b) - 1;
                }
            }
            if (tl == 0) {
                hash_insert(H, hbits, p);
                if (a.path && hops < a.path_cap) a.path[(size_t)qi * a.path_cap + hops] = p;
            }
            tm.sync();
            ++hops;
            if (Hg && H == Hs && (uint32_t)hops >= (1u << hbits) / 2) {
                hash_migrate<T>(Hs, hbits, Hg, a.hash_bits, tm);
                H = Hg;
                hbits = a.hash_bits;
            }
            if (!inflight || pend != p) {  // the prefetch always targets p; kept as a safeguard
                if (inflight) {
                    if (!mbar_wait_bounded(&bar[cb], (phase >> cb) & 1u)) { status |= SQG_STATUS_TIMEOUT; healthy = false; break; }
                    phase ^= 1u << cb;
                }
                tm.sync();
                if (tl == 0) {
                    fence_proxy_async();
                    bulk_fetch(buf[cb], a.blocks + (size_t)p * a.block_bytes, a.block_bytes, &bar[cb]);
                }
                pend = p;
                inflight = true;
            }
            if (!mbar_wait_bounded(&bar[cb], (phase >> cb) & 1u)) {
                status |= SQG_STATUS_TIMEOUT;
                healthy = false;
                break;
            }
            phase ^= 1u << cb;
            inflight = false;
            const unsigned char *blk = buf[cb];

            // ---- line 4: exact distance, implicit re-ranking
            // exact distance partials, then the neighbours' integer sums S while
            // the partials' butterfly is in flight, then the butterfly
            float dacc[V];
            exact_partial<CH, T>(qv, reinterpret_cast<const float *>(blk), nch, tm, dacc);
            const uint32_t *ids = reinterpret_cast<const uint32_t *>(blk + a.off_ids);
            int Sv[NT];
            uint32_t cid[NT];
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const uint32_t j = tl + T * t;
                cid[t] = ids[j];
                Sv[t] = estimate_S<CH>(blk, a, planes, j);
            }
            const float dist_c = exact_reduce<T>(dacc, tm);
            if (hops == 1 && tl == 0) beam[0].x = __float_as_uint(dist_c);
            bool improved = false;
            {
                const bool full = rc == k;
                if (!full || kless(dist_c, p, __uint_as_float(res[k - 1].x), res[k - 1].y)) {
                    improved = true;
                    int pos = 0;
                    for (int base = 0; base < rc; base += T) {
                        int i = base + tl;
                        const uint2 e = i < rc ? res[i] : make_uint2(0u, 0u);
                        pos += __popc(tm.ballot(i < rc && kless(__uint_as_float(e.x), e.y, dist_c, p)));
                    }
                    const int top = full ? k - 1 : rc;  // entries [pos, top) move up one
                    for (int base = ((top - 1) & ~(T - 1)); base >= (pos & ~(T - 1)) && top > pos; base -= T) {
                        int i = base + tl;
                        bool mv = i >= pos && i < top;
                        const uint2 e = mv ? res[i] : make_uint2(0u, 0u);
                        tm.sync();
                        if (mv) res[i + 1] = e;
                        tm.sync();
                    }
                    if (tl == 0) res[pos] = make_uint2(__float_as_uint(dist_c), p);
                    rc = full ? k : rc + 1;
                }
            }

            // ---- line 5: estimates for all R neighbours from the same block
            const bool full = m == ef;
            const uint2 we = beam[ef - 1 < m ? ef - 1 : 0];
            const float wk = __uint_as_float(we.x);
            const uint32_t wi = we.y & kIdMask;
            float ck[NT];
            int cpos[NT];
            bool adm[NT];
            const float sqrt_dc = a.eps0 == 0.0f ? 0.0f : __fsqrt_rn(dist_c);
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const uint32_t j = tl + T * t;
                const Est e = estimate_from_S(blk, a, qs, j, Sv[t], dist_c, sqrt_dc);
                ck[t] = e.key;
                // line 6: only unvisited neighbours enter; an entry that the cut
                // to ef would drop at once is skipped early
                adm[t] = cid[t] != kEmpty && (!full || kless(ck[t], cid[t], wk, wi));  // kEmpty: an empty slot
                if (adm[t]) adm[t] = !hash_contains(H, hbits, cid[t]);
            }
            if (!a.multi_estimate) {  // ablation w/o ME: skip ids already in the beam
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    bool in = false;
                    for (int i = 0; i < m && adm[t]; ++i) in |= (beam[i].y & kIdMask) == cid[t];
                    adm[t] = adm[t] && !in;
                }
            }
            // position in the beam; an identical (key, id) already there is dropped
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                cpos[t] = 0;
                if (adm[t]) {
                    int lo = 0, hi = m;
                    while (lo < hi) {
                        int mid = (lo + hi) >> 1;
                        const uint2 e = beam[mid];
                        if (kless(__uint_as_float(e.x), e.y & kIdMask, ck[t], cid[t])) lo = mid + 1;
                        else hi = mid;
                    }
                    cpos[t] = lo;
                    if (lo < m) {
                        const uint2 e = beam[lo];
                        if (__uint_as_float(e.x) == ck[t] && (e.y & kIdMask) == cid[t]) adm[t] = false;
                    }
                }
            }
            uint32_t am[NT];
            int nadm = 0;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                am[t] = tm.ballot(adm[t]);
                nadm += __popc(am[t]);
            }
            // rank among the admitted candidates (ids in a block are distinct)
            int rank[NT];
#pragma unroll
            for (int t = 0; t < NT; ++t) rank[t] = 0;
            const float kInf = __int_as_float(0x7f800000);
            float bk = kInf, b2k = kInf;  // best and second-best admitted candidates
            uint32_t bi = kEmpty, b2i = kEmpty;
#pragma unroll
            for (int t2 = 0; t2 < NT; ++t2) {
                uint32_t mm = am[t2];
                while (mm) {
                    const int src = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const float ok = tm.shfl(ck[t2], src);
                    const uint32_t oi = tm.shfl(cid[t2], src);
#pragma unroll
                    for (int t = 0; t < NT; ++t) rank[t] += kless(ok, oi, ck[t], cid[t]) ? 1 : 0;
                }
            }
            // the best admitted candidate has rank 0 (ranks are distinct), the
            // runner-up rank 1 (needed for the speculative prefetch only)
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const uint32_t m0 = tm.ballot(adm[t] && rank[t] == 0);
                if (m0) {
                    const int s = __ffs(m0) - 1;
                    bk = tm.shfl(ck[t], s);
                    bi = tm.shfl(cid[t], s);
                }
                if (a.prefetch == 2) {
                    const uint32_t m1 = tm.ballot(adm[t] && rank[t] == 1);
                    if (m1) {
                        const int s = __ffs(m1) - 1;
                        b2k = tm.shfl(ck[t], s);
                        b2i = tm.shfl(cid[t], s);
                    }
                }
            }
            // ---- memory prefetching (Sec. 3.1.4): the next vertex is the smaller
            // of the first unvisited beam entry and the best admitted candidate
            uint32_t next_id = kEmpty, runner_id = kEmpty;
            {
                const uint2 ne = nxt < m ? beam[nxt] : make_uint2(__float_as_uint(kInf), kEmpty);
                const float nk = __uint_as_float(ne.x);
                const uint32_t ni = nxt < m ? (ne.y & kIdMask) : kEmpty;
                const bool cand_first = nadm > 0 && kless(bk, bi, nk, ni);
                next_id = cand_first ? bi : ni;
                if (a.prefetch == 2) {  // speculative: the runner-up, if no better candidate appears
                    float rk = cand_first ? nk : bk;
                    uint32_t ri = cand_first ? ni : bi;
                    if (cand_first) {
                        if (kless(b2k, b2i, rk, ri)) { rk = b2k; ri = b2i; }
                    } else {
                        int n2 = m;  // the unvisited beam entry after nxt
                        for (int base = nxt + 1; base < m; base += T) {
                            const int i = base + tl;
                            const uint32_t bb2 = tm.ballot(i < m && !(beam[i].y & kVisited));
                            if (bb2) { n2 = base + __ffs(bb2) - 1; break; }
                        }
                        if (n2 < m) {
                            const uint2 e2 = beam[n2];
                            if (kless(__uint_as_float(e2.x), e2.y & kIdMask, rk, ri)) {
                                rk = __uint_as_float(e2.x);
                                ri = e2.y & kIdMask;
                            }
                        }
                    }
                    runner_id = ri;
                }
            }
            tm.sync();
            if (runner_id != kEmpty && tl == 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                                 a.blocks + (size_t)runner_id * a.block_bytes),
                             "r"(a.block_bytes)
                             : "memory");
            if (next_id != kEmpty) {
                const int nb = cb ^ 1;
                if (tl == 0) {
                    fence_proxy_async();
                    bulk_fetch(buf[nb], a.blocks + (size_t)next_id * a.block_bytes, a.block_bytes, &bar[nb]);
                }
                cb = nb;
                pend = next_id;
                inflight = true;
            }

            // ---- line 6: merge the admitted candidates and cut the beam to ef
            int inserted = 0;
            if (nadm > 0) {
                // beam positions of the admitted candidates in rank order: a
                // smaller key never has a larger position, so this is sorted
                int *spos = reinterpret_cast<int *>(ws + a.o_spos);
#pragma unroll
                for (int t = 0; t < NT; ++t)
                    if (adm[t]) spos[rank[t]] = cpos[t];
                tm.sync();
                const int minpos = spos[0];
                // number of admitted candidates placed at or before beam entry i
                auto count_le = [&](int i) {
                    int lo = 0, hi = nadm;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (spos[mid] <= i) lo = mid + 1;
                        else hi = mid;
                    }
                    return lo;
                };
                for (int base = ((m - 1) & ~(T - 1)); base >= (minpos & ~(T - 1)); base -= T) {
                    const int i = base + tl;
                    const bool valid = i >= minpos && i < m;
                    const int cnt = valid ? count_le(i) : 0;
                    const uint2 e = valid ? beam[i] : make_uint2(0u, 0u);
                    tm.sync();
                    if (valid && cnt > 0 && i + cnt < ef) beam[i + cnt] = e;
                    tm.sync();
                }
                const int nxt_shift = nxt < m ? count_le(nxt) : 0;
                int newcur = m + nadm;  // "none"
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const int fp = cpos[t] + rank[t];
                    const bool keep = adm[t] && fp < ef;
                    if (keep) {
                        beam[fp] = make_uint2(__float_as_uint(ck[t]), cid[t]);
                        newcur = min(newcur, fp);
                    }
                    inserted += __popc(tm.ballot(keep));
                }
                newcur = tm.reduce_min(newcur);
                if (nxt < m && nxt >= minpos) {
                    if (nxt + nxt_shift < ef) newcur = min(newcur, nxt + nxt_shift);
                } else if (nxt < m) {
                    newcur = min(newcur, nxt);
                }
                m = min(ef, m + nadm);
                cur = newcur < m ? newcur : m;
            } else {
                cur = nxt;
            }
            tm.sync();

            // ---- learned early stop (not in the paper) / trace
            // (teams of 32 lanes only: the fused network and the trace use the whole warp)
            const bool stop_on = T == 32 && (a.mlp || a.trace_feat);  // the state below feeds the stop only
            if (stop_on) {
                st.hops = hops;
                st.inserted_last = inserted;
                st.dist_c = dist_c;
                if (improved) st.last_improve = hops;
                st.ema_improve =
                    __fadd_rn(__fmul_rn(0.75f, st.ema_improve), __fmul_rn(0.25f, improved ? 1.0f : 0.0f));
                st.ema_insert = __fadd_rn(__fmul_rn(0.75f, st.ema_insert),
                                          __fmul_rn(0.25f, __fmul_rn((float)inserted, inv_R)));
            }
            if constexpr (T == 32) if (stop_on && a.stop_every > 0 && hops % a.stop_every == 0 && rc == k) {
                const float rk = __uint_as_float(res[k - 1].x);
                const float rk2 = __fmul_rn(1.25f, rk);
                int u = 0, near1 = 0, near2 = 0;  // unvisited; of them with key <= rk, <= 1.25 rk
                for (int base = 0; base < m; base += T) {
                    const int i = base + tl;
                    const uint2 e = i < m ? beam[i] : make_uint2(0u, kVisited);
                    const bool un = !(e.y & kVisited);
                    const float kk = un ? __uint_as_float(e.x) : 0.0f;
                    u += __popc(tm.ballot(un));
                    near1 += __popc(tm.ballot(un && kk <= rk));
                    near2 += __popc(tm.ballot(un && kk <= rk2));
                }
                const float den = rk > 1e-20f ? rk : 1e-20f;
                const float fef = (float)ef;
                const float since = (float)(hops - st.last_improve);
                // ratios as products with four reciprocals
                const float inv_ef = __fdiv_rn(1.0f, fef), inv_den = __fdiv_rn(1.0f, den);
                const float inv_k = __fdiv_rn(1.0f, (float)k);
                const float inv_h1 = __fdiv_rn(1.0f, __fadd_rn((float)hops, 1.0f));
                float f[SQG_MLP_IN];
                f[0] = __fmul_rn((float)hops, inv_ef);
                f[1] = __fmul_rn(since, inv_ef);
                f[2] = __fmul_rn((float)u, inv_ef);
                f[3] = __fmul_rn((float)m, inv_ef);
                f[4] = __fmul_rn(__uint_as_float(res[0].x), inv_den);
                f[5] = u > 0 ? __fmul_rn(__uint_as_float(beam[cur].x), inv_den) : 0.0f;
                f[6] = __fmul_rn(dist_c, inv_den);
                f[7] = __fmul_rn((float)inserted, __fdiv_rn(1.0f, (float)R));
                f[8] = __fmul_rn((float)k, inv_ef);
                f[9] = st.ema_improve;
                f[10] = st.ema_insert;
                f[11] = __fmul_rn((float)near1, inv_k);
                f[12] = __fmul_rn((float)near2, inv_k);
                f[13] = __fmul_rn(since, inv_h1);
                f[14] = dist_c <= rk ? 1.0f : 0.0f;
                f[15] = __fmul_rn((float)k, 0.01f);
#pragma unroll
                for (int i = 0; i < SQG_MLP_IN; ++i) f[i] = clamp8(f[i]);
                if (a.trace_feat && tn < a.trace_cap) {
                    float *dst = a.trace_feat + ((size_t)qi * a.trace_cap + tn) * SQG_MLP_IN;
                    if (lane < SQG_MLP_IN) {
                        float v = f[0];
#pragma unroll
                        for (int i = 1; i < SQG_MLP_IN; ++i) v = lane == i ? f[i] : v;
                        dst[lane] = v;
                    }
                    if (a.gt) {
                        int hit = 0;
                        const uint32_t *g = a.gt + (size_t)qi * a.gt_k;
                        for (int i = tl; i < rc; i += 32) {
                            const uint32_t x = res[i].y;
                            for (int b = 0; b < k; ++b) hit += g[b] == x ? 1 : 0;
                        }
#pragma unroll
                        for (int o = 16; o >= 1; o >>= 1) hit += tm.shfl_xor(hit, o);
                        if (tl == 0) a.trace_hit[(size_t)qi * a.trace_cap + tn] = hit;
                    }
                    ++tn;
                }
                if (a.mlp && mlp_logit_warp(wts, f, lane, reinterpret_cast<float *>(ws + a.o_spos)) >
                                 a.stop_logit) {
                    status |= SQG_STATUS_LEARNED_STOP;
                    break;
                }
            }
        }
        // drain a prefetch that will not be used
        if (inflight) {
            if (mbar_wait_bounded(&bar[cb], (phase >> cb) & 1u)) {
                phase ^= 1u << cb;
            } else {
                status |= SQG_STATUS_TIMEOUT;
                healthy = false;
            }
        }
        tm.sync();
        // ---- line 8: the k nearest expanded vertices by exact distance
        const bool ok = !(status & SQG_STATUS_TIMEOUT);
        for (int t = tl; t < k; t += T) {
            const bool have = ok && t < rc;
            const uint2 e = have ? res[t] : make_uint2(0x7f800000u, SQG_NO_ID);
            a.out_ids[off + t] = e.y;
            a.out_dists[off + t] = __uint_as_float(e.x);
        }
        if (tl == 0) {
            if (a.stats) a.stats[qi] = sqg_query_stats{(uint32_t)hops, status};
            if (status) atomicOr(a.status_word, status);
            if (a.trace_n) a.trace_n[qi] = tn;
        }
        tm.sync();
    }
}

// Host-side launch helpers, defined in the instantiation units.
// Tensor-core rotation and the exact quantization after it (rotate_tc.cu).
float rotate_tc_err_scale(int d);
cudaError_t launch_split_tf32(const float *x, float *hi, float *lo, size_t n, cudaStream_t s);
// The fast JLT on the query side (fjlt.cu); d a power of 2 in 32..2048.
cudaError_t launch_fjlt(const float *q, const float *signs, float *out, int nq, int d, cudaStream_t s);
cudaError_t launch_rotate_tc(const float *q, const float *rot_hi, const float *rot_lo, float *out, int nq, int d,
                             uint32_t *status, cudaStream_t s);
cudaError_t launch_quantize_exact(const float *q, const float *rot, const float *qa, int nq, int d, uint32_t *planes,
                                  float4 *scal, uint32_t *recomputed, bool plane_major, cudaStream_t s);
cudaError_t launch_search_nb1(int ch, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const SearchArgs &a);
cudaError_t launch_search_nb2(int ch, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const SearchArgs &a);
cudaError_t search_occupancy_nb1(int ch, int block, size_t smem, int *blocks_per_sm);
// teams of 16 or 8 lanes (search_team.cu): ch 1 or 2, nb 1 or 2
cudaError_t launch_search_team(int ch, int nb, int team, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                               const SearchArgs &a);
cudaError_t search_occupancy_team(int ch, int nb, int team, int block, size_t smem, int *blocks_per_sm);
cudaError_t search_occupancy_nb2(int ch, int block, size_t smem, int *blocks_per_sm);
// the compact kernel (search_compact.cuh): d <= 1024 (ch 1, 2, 4, 8),
// out-degree 32 (nr 1) or 64 (nr 2), k <= 32, ef <= 64 (bnb 2) or 128 (bnb
// 4) beam entries (for d <= 256 also k <= 128 and ef <= 256: the big
// builds below), whole warps, multiple estimates, no trace
// (lean 1, d <= 256 and out-degree 32: the build for one more resident block
// of 4 warps per SM: 9 / 8, else 8 / 7)
cudaError_t launch_search_compact(int ch, int nr, int bnb, int lean, dim3 grid, dim3 block, size_t smem,
                                  cudaStream_t s, const SearchArgs &a);
cudaError_t search_occupancy_compact(int ch, int nr, int bnb, int lean, int block, size_t smem, int *blocks_per_sm);
// its builds for d > 256 (search_compact_wide.cu)
cudaError_t launch_search_compact_wide(int ch, int nr, int bnb, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                       const SearchArgs &a);
cudaError_t search_occupancy_compact_wide(int ch, int nr, int bnb, int block, size_t smem, int *blocks_per_sm);
// its builds with the learned early stop fused (search_compact_stop.cu)
cudaError_t launch_search_compact_stop(int ch, int nr, int bnb, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                       const SearchArgs &a);
cudaError_t search_occupancy_compact_stop(int ch, int nr, int bnb, int block, size_t smem, int *blocks_per_sm);
// its builds for d <= 256 with 256-entry beams (bnb 8) or k <= 128 (rk 4),
// plain or with the stop fused (search_compact_big.cu)
cudaError_t launch_search_compact_big(int ch, int nr, int bnb, int rk, bool stop, dim3 grid, dim3 block, size_t smem,
                                      cudaStream_t s, const SearchArgs &a);
cudaError_t search_occupancy_compact_big(int ch, int nr, int bnb, int rk, bool stop, int block, size_t smem,
                                         int *blocks_per_sm);

}  // namespace sqg
