// rotate_tc.cu -- the batched query rotation q' = P^-1 q (Eq. (4)) on the
// 5th-generation tensor cores, and the exact 4-bit quantization built on it.
//
// The canonical fp32 rotation (the one the CUDA-core kernel and the oracle
// compute) is chunked: q'_i = (((0 + s_0) + s_1) + ... ) over the d/32
// chunks, s_c an fmaf chain over j = 32c .. 32c+31 started from 0.
//
// rotate_tc_kernel: persistent, one CTA per SM, walking 128-query x 128-output
// tiles D = A B^T with A = the queries and B = the rows of P^-1, both K-major,
// with tcgen05.mma kind::tf32.  fp32 accuracy comes from the 3xTF32 split
// a.b ~ hi(a)hi(b) + hi(a)lo(b) + lo(a)hi(b), hi = tf32(x), lo = tf32(x - hi).
// Warp roles:
//   warp 0      TMA producer: per 32-wide K chunk, the raw query tile and the
//               pre-split hi/lo tiles of P^-1 (cp.async.bulk.tensor, 128-byte
//               swizzle) into a 3-stage ring;
//   warp 1      MMA issuer: 12 MMAs per chunk into one of two TMEM buffers;
//   warps 2-5   split the query tile into hi (in place) and lo;
//   warps 6-21  drain each chunk's 128 x 128 result from TMEM (tcgen05.ld)
//               and add it to fp32 registers: 4 warps per 32-lane quarter
//               of TMEM, 32 columns of one tile row per thread, so one
//               load round-trip per chunk.
// Draining per chunk keeps the tensor cores' accumulation short (96 products
// per accumulator), which is what makes the error bound below tight.
//
// quantize_exact_kernel: the search's decisions depend on the 4-bit codes,
// v_l and Delta being exactly those of the canonical rotation.  The
// tensor-core q' differs from it by at most err = c(d) * ||q||, so every
// coordinate whose code or whose role as min/max could change within err is
// recomputed in the canonical order (one warp per coordinate, its row staged
// through shared memory, one chunk per lane); the rest are decided from q'.
// The result is bit-identical to quantizing the canonical rotation.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/sqg.h"

namespace {

constexpr int BM = 128, BN = 128, BK = 32;  // BK fp32 = one 128-byte swizzled row
constexpr int kStages = 3;
constexpr int kTile = BM * BK * 4;          // 16 KB
constexpr int kStageBytes = 4 * kTile;      // query raw->hi, query lo, P hi, P lo
constexpr int kConvWarp0 = 2, kConvWarps = 4, kDrainWarp0 = 6, kDrainWarps = 16;
constexpr int kWarps = kDrainWarp0 + kDrainWarps, kThreads = kWarps * 32;
constexpr int kDrainCols = BN / (kDrainWarps / 4);  // accumulator columns per drain thread
constexpr uint32_t kTmemCols = 2 * BN;
constexpr int kSmemBytes = kStages * kStageBytes + 1024;  // + alignment slack
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; give up after
// kWaitNs or as soon as another role has given up (abort flag).
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    const unsigned long long t0 = gtime();
    for (;;) {
        if (bar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtime() - t0 > kWaitNs) {
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor for a K-major operand in the 128-byte
// swizzle layout written by the tensor map: 8-row groups 1024 B apart
// (stride byte offset), leading byte offset unused (1), the fixed 0b001 at
// bits 46-48, layout type 2 (128-byte swizzle) at bits 61-63.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// instruction descriptor, kind::tf32: D f32 (bits 4-5 = 1), A and B tf32
// (bits 7-9 and 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(addr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
    rotate_tc_kernel(const __grid_constant__ CUtensorMap qmap, const __grid_constant__ CUtensorMap phimap,
                     const __grid_constant__ CUtensorMap plomap, float *__restrict__ out, int nq, int d,
                     uint32_t *status) {
    extern __shared__ unsigned char smraw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                                          ~static_cast<uintptr_t>(1023));
    __shared__ __align__(8) uint64_t full_bar[kStages], conv_bar[kStages], empty_bar[kStages];
    __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    volatile int *abort_v = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nchunk = d / BK;
    // persistent: this CTA takes tiles blockIdx.x, + gridDim.x, ...; column
    // tiles vary fastest, so CTAs running together share query tiles in L2
    const int ncol_tiles = (d + BN - 1) / BN;
    const int ntiles = ncol_tiles * ((nq + BM - 1) / BM);
    const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int total = my_tiles * nchunk;  // chunks this CTA streams, across its tiles
    auto tile_of = [&](int g, int &r0, int &c0) {
        const int t = (int)blockIdx.x + (g / nchunk) * (int)gridDim.x;
        r0 = (t / ncol_tiles) * BM;
        c0 = (t % ncol_tiles) * BN;
    };

    if (warp == 0) {  // two 128-column fp32 accumulators in tensor memory
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(saddr(&full_bar[s]), 1);
            bar_init(saddr(&conv_bar[s]), kConvWarps);
            bar_init(saddr(&empty_bar[s]), 1);
        }
        for (int t = 0; t < 2; ++t) {
            bar_init(saddr(&tfull_bar[t]), 1);
            bar_init(saddr(&tempty_bar[t]), kDrainWarps);
        }
        bar_init(saddr(&done_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t base = saddr(sm);
    // stage s: [query hi | query lo | P hi | P lo], each 1024-byte aligned
    auto tile = [&](int s, int which) -> uint32_t { return base + (uint32_t)(s * kStageBytes + which * kTile); };

    if (warp == 0) {
        if (lane == 0) {
            for (int g = 0; g < total; ++g) {
                const int s = g % kStages, n = g / kStages, k = g % nchunk;
                int r0, c0;
                tile_of(g, r0, c0);
                if (n >= 1 && !bar_wait(saddr(&empty_bar[s]), (uint32_t)((n - 1) & 1), abort_v)) break;
                bar_arrive_tx(saddr(&full_bar[s]), 3 * kTile);
                tma_load_2d(tile(s, 0), &qmap, k * BK, r0, saddr(&full_bar[s]));
                tma_load_2d(tile(s, 2), &phimap, k * BK, c0, saddr(&full_bar[s]));
                tma_load_2d(tile(s, 3), &plomap, k * BK, c0, saddr(&full_bar[s]));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int g = 0; g < total; ++g) {
                const int s = g % kStages, n = g / kStages, t = g & 1, m = g >> 1;
                if (!bar_wait(saddr(&full_bar[s]), (uint32_t)(n & 1), abort_v)) break;
                if (!bar_wait(saddr(&conv_bar[s]), (uint32_t)(n & 1), abort_v)) break;
                if (m >= 1 && !bar_wait(saddr(&tempty_bar[t]), (uint32_t)((m - 1) & 1), abort_v)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dt = tmem + (uint32_t)(t * BN);
#pragma unroll
                for (int st = 0; st < BK / 8; ++st) {  // K = 8 per MMA = 32 bytes along the swizzled row
                    const uint32_t ko = (uint32_t)st * 32;
                    const uint64_t ah = desc_sw128(tile(s, 0) + ko), al = desc_sw128(tile(s, 1) + ko);
                    const uint64_t bh = desc_sw128(tile(s, 2) + ko), bl = desc_sw128(tile(s, 3) + ko);
                    mma_tf32(dt, ah, bh, st > 0 ? 1u : 0u);
                    mma_tf32(dt, ah, bl, 1u);
                    mma_tf32(dt, al, bh, 1u);
                }
                mma_commit(saddr(&empty_bar[s]));
                mma_commit(saddr(&tfull_bar[t]));
            }
            // every MMA this thread issued has finished before TMEM is freed
            mma_commit(saddr(&done_bar));
            if (!bar_wait(saddr(&done_bar), 0u, abort_v)) {
                const unsigned long long t0 = gtime();
                while (!bar_try_wait(saddr(&done_bar), 0u) && gtime() - t0 < kWaitNs) {
                }
            }
        }
    } else if (warp < kDrainWarp0) {
        const int ct = tid - kConvWarp0 * 32;
        for (int g = 0; g < total; ++g) {
            const int s = g % kStages, n = g / kStages;
            if (!bar_wait(saddr(&full_bar[s]), (uint32_t)(n & 1), abort_v)) break;
            float4 *raw = reinterpret_cast<float4 *>(sm + s * kStageBytes);
            float4 *lo = reinterpret_cast<float4 *>(sm + s * kStageBytes + kTile);
            // elementwise, so the swizzled positions need no decoding
            for (int i = ct; i < kTile / 16; i += kConvWarps * 32) {
                const float4 x = raw[i];
                float4 h, l;
                h.x = tf32_round(x.x); l.x = tf32_round(__fsub_rn(x.x, h.x));
                h.y = tf32_round(x.y); l.y = tf32_round(__fsub_rn(x.y, h.y));
                h.z = tf32_round(x.z); l.z = tf32_round(__fsub_rn(x.z, h.z));
                h.w = tf32_round(x.w); l.w = tf32_round(__fsub_rn(x.w, h.w));
                raw[i] = h;
                lo[i] = l;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(saddr(&conv_bar[s]));
        }
    } else {
        const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31 = tile rows
        const int col0 = ((warp - kDrainWarp0) >> 2) * kDrainCols;
        float acc[kDrainCols];
        for (int g = 0; g < total; ++g) {
            const int t = g & 1, m = g >> 1, k = g % nchunk;
            if (k == 0) {
#pragma unroll
                for (int j = 0; j < kDrainCols; ++j) acc[j] = 0.0f;
            }
            if (!bar_wait(saddr(&tfull_bar[t]), (uint32_t)(m & 1), abort_v)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int cc = 0; cc < kDrainCols; cc += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * BN + col0 + cc), v);
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[cc + j] = __fadd_rn(acc[cc + j], __uint_as_float(v[j]));
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(saddr(&tempty_bar[t]));
            if (k == nchunk - 1) {  // the tile is complete: write this thread's part of its row
                int r0, c0;
                tile_of(g, r0, c0);
                const int row = r0 + quarter * 32 + lane;
                if (row < nq && c0 + col0 < d) {  // d - c0 is a multiple of 32
                    float4 *o = reinterpret_cast<float4 *>(out + (size_t)row * d + c0 + col0);
#pragma unroll
                    for (int j = 0; j < kDrainCols / 4; ++j)  // streaming stores: read once by the exact pass
                        __stcs(o + j, make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
    if (tid == 0 && *abort_v) atomicOr(status, SQG_STATUS_TIMEOUT);
}

// hi = tf32(x), lo = tf32(x - hi), elementwise (the rows of P^-1, once per index)
__global__ void split_tf32_kernel(const float *__restrict__ x, float *__restrict__ hi, float *__restrict__ lo,
                                  size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float h = tf32_round(x[i]);
        hi[i] = h;
        lo[i] = tf32_round(__fsub_rn(x[i], h));
    }
}

constexpr int kMaxD = 2048;
constexpr int kQxWarps = 4;
constexpr int kPadChunk = 36;  // floats per 32-float chunk in shared memory: 144 B, conflict-free float4 reads

// Per-warp shared memory of the exact pass: the query and one row of P^-1,
// chunk c at [c * kPadChunk, +32).
struct QxLayout {
    size_t q, row, warp;
    __host__ __device__ explicit QxLayout(int d) {
        const size_t chunks = (size_t)(d / 32) * kPadChunk * 4;
        q = 0;
        row = chunks;
        warp = 2 * chunks;
    }
};

// d floats from global (16-byte aligned) into the padded chunk layout; the
// loads of a batch are all issued before its stores.
__device__ __forceinline__ void stage_padded(float *dst, const float *__restrict__ src, int d, int lane) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    const int n4 = d / 4;
    for (int i0 = lane; i0 < n4; i0 += 32 * 8) {
        float4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (i0 + 32 * j < n4) v[j] = __ldg(s4 + i0 + 32 * j);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = i0 + 32 * j;
            if (i < n4) *reinterpret_cast<float4 *>(dst + (i >> 3) * kPadChunk + (i & 7) * 4) = v[j];
        }
    }
}

// s_c = fmaf chain over the 32 columns of chunk c, from 0.
__device__ __forceinline__ float chunk_chain(const float *row, const float *q) {
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 r = *reinterpret_cast<const float4 *>(row + 4 * j);
        const float4 v = *reinterpret_cast<const float4 *>(q + 4 * j);
        s = __fmaf_rn(r.x, v.x, s);
        s = __fmaf_rn(r.y, v.y, s);
        s = __fmaf_rn(r.z, v.z, s);
        s = __fmaf_rn(r.w, v.w, s);
    }
    return s;
}

// The canonical rotated coordinate i, by the whole warp: the row is staged
// (coalesced), lane c runs chunk c (and c + 32), and every lane adds the
// chunk sums to the total in order c = 0, 1, ...; all lanes return it.
__device__ float warp_canonical(const float *__restrict__ rot, int i, const float *qpad, float *rowpad, int d,
                                int lane) {
    const int nc = d / 32;
    __syncwarp();  // the previous call's reads of rowpad are done
    stage_padded(rowpad, rot + (size_t)i * d, d, lane);
    __syncwarp();
    const float s0 = lane < nc ? chunk_chain(rowpad + lane * kPadChunk, qpad + lane * kPadChunk) : 0.0f;
    const float s1 =
        lane + 32 < nc ? chunk_chain(rowpad + (lane + 32) * kPadChunk, qpad + (lane + 32) * kPadChunk) : 0.0f;
    float tot = 0.0f;
#pragma unroll 8
    for (int c = 0; c < nc; ++c) tot = __fadd_rn(tot, __shfl_sync(0xFFFFFFFFu, c < 32 ? s0 : s1, c & 31));
    return tot;
}

constexpr int kMaxWords = kMaxD / 32;

// One warp per query.  qa = the tensor-core q'; err_scale * ||q|| bounds
// |qa_i - canonical_i| for every i.  Writes planes (per word w the four
// planes b as one uint4 -- [w][b] -- or, with plane_major, [b][w]) and
// (v_l, delta, Sq, 1/sqrt(d)) exactly as the canonical rotation would give.
__global__ void __launch_bounds__(kQxWarps * 32)
    quantize_exact_kernel(const float *__restrict__ q, const float *__restrict__ rot, const float *__restrict__ qa,
                          int nq, int d, float err_scale, uint32_t *__restrict__ planes, float4 *__restrict__ scal,
                          uint32_t *__restrict__ recomputed, int plane_major) {
    extern __shared__ __align__(16) unsigned char qxsm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int qi = blockIdx.x * kQxWarps + wib;
    if (qi >= nq) return;
    const QxLayout L(d);
    float *qpad = reinterpret_cast<float *>(qxsm + wib * L.warp + L.q);
    float *rowpad = reinterpret_cast<float *>(qxsm + wib * L.warp + L.row);
    const int nw = d / 32;
    const float *qq = q + (size_t)qi * d;
    const float *qr = qa + (size_t)qi * d;
    stage_padded(qpad, qq, d, lane);
    float x[kMaxWords];  // coordinate 32w + lane
    float ss = 0.0f, lo = __int_as_float(0x7f800000), hi = -lo;
    for (int w0 = 0; w0 < nw; w0 += 8) {  // batches of loads in flight together
        float vq[8], vx[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (w0 + j < nw) {
                vq[j] = __ldcs(qq + (w0 + j) * 32 + lane);  // streamed once: keep P^-1 in L2
                vx[j] = __ldcs(qr + (w0 + j) * 32 + lane);
            }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (w0 + j < nw) {
                x[w0 + j] = vx[j];
                ss = fmaf(vq[j], vq[j], ss);
                lo = fminf(lo, vx[j]);
                hi = fmaxf(hi, vx[j]);
            }
    }
    for (int o = 16; o >= 1; o >>= 1) {
        ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
        lo = fminf(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
    }
    const float err = err_scale * sqrtf(ss) + 1e-30f;
    // candidates for the minimum and the maximum (within 2 err of the
    // tensor-core extremes), one bit per word in each lane
    uint64_t exact = 0;
    for (int w = 0; w < nw; ++w)
        if (x[w] <= lo + 2.0f * err || x[w] >= hi - 2.0f * err) exact |= 1ull << w;
    // recompute them (the extremes are among them); every lane sees each
    // recomputed value, so v_l and v_r come out warp-uniform
    float vl = __int_as_float(0x7f800000), vr = -vl;
    int nrec = 0;
    for (uint32_t owners = __ballot_sync(0xFFFFFFFFu, exact != 0); owners; owners &= owners - 1) {
        const int l = __ffs(owners) - 1;
        for (uint64_t cm = __shfl_sync(0xFFFFFFFFu, exact, l); cm; cm &= cm - 1) {
            const int w = __ffsll((long long)cm) - 1;
            const float v = warp_canonical(rot, w * 32 + l, qpad, rowpad, d, lane);
            if (lane == l) x[w] = v;
            vl = v < vl ? v : vl;
            vr = v > vr ? v : vr;
            ++nrec;
        }
    }
    const float range = __fsub_rn(vr, vl);
    const float delta = range > 0.0f ? __fdiv_rn(range, 15.0f) : 0.0f;
    const float inv = range > 0.0f ? __fdiv_rn(15.0f, range) : 0.0f;
    const float margin = err * inv * 1.01f + 1e-4f;  // in units of the code
    int sq = 0;
    for (int w = 0; w < nw; ++w) {
        float y = 0.0f;
        bool redo = false;
        if (range > 0.0f) {
            y = __fadd_rn(__fmul_rn(__fsub_rn(x[w], vl), inv), 0.5f);
            // an integer boundary (1 .. 15) within the margin: decide exactly
            const float nearest = fminf(fmaxf(rintf(y), 1.0f), 15.0f);
            redo = !(exact >> w & 1ull) && fabsf(y - nearest) <= margin;
        }
        for (uint32_t m = __ballot_sync(0xFFFFFFFFu, redo); m; m &= m - 1) {
            const int l = __ffs(m) - 1;
            const float v = warp_canonical(rot, w * 32 + l, qpad, rowpad, d, lane);
            if (lane == l) y = __fadd_rn(__fmul_rn(__fsub_rn(v, vl), inv), 0.5f);
            ++nrec;
        }
        int t = 0;
        if (range > 0.0f) {
            t = __float2int_rz(y);
            t = t > 15 ? 15 : t;
        }
        sq += t;
        const uint32_t b0 = __ballot_sync(0xFFFFFFFFu, t & 1), b1 = __ballot_sync(0xFFFFFFFFu, t & 2);
        const uint32_t b2 = __ballot_sync(0xFFFFFFFFu, t & 4), b3 = __ballot_sync(0xFFFFFFFFu, t & 8);
        if (lane == 0) {
            uint32_t *pq = planes + (size_t)qi * 4 * nw;
            if (plane_major) {
                pq[w] = b0;
                pq[nw + w] = b1;
                pq[2 * nw + w] = b2;
                pq[3 * nw + w] = b3;
            } else {
                reinterpret_cast<uint4 *>(pq)[w] = make_uint4(b0, b1, b2, b3);
            }
        }
    }
    sq = __reduce_add_sync(0xFFFFFFFFu, sq);
    if (lane == 0) {
        scal[qi] = make_float4(vl, delta, (float)sq, __fdiv_rn(1.0f, __fsqrt_rn((float)d)));
        if (recomputed) atomicAdd(recomputed, (uint32_t)nrec);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// rows x cols fp32, row-major; boxes of 128 rows x 32 columns, 128-byte swizzle,
// rows past the end read as zeros
bool make_tile_map(CUtensorMap *m, const float *base, uint64_t rows, uint64_t cols) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * sizeof(float)};
    cuuint32_t box[2] = {BK, BM};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

namespace sqg {

// Bound on |tensor-core q'_i - canonical q'_i| per unit of ||q||, with
// u = 2^-24, C = d/32 chunks and sum_j |P_ij q_j| <= ||P_i|| ||q|| = ||q||:
//  * the 3xTF32 split drops lo(a)lo(b) and the tf32 rounding of both low
//    parts: at most 3 * 2^-22 = 12u of every |P_ij q_j|;
//  * per chunk the tensor cores add 96 exact tf32 products into a fresh fp32
//    accumulator; every addition is taken to err by at most 2u (one unit in
//    the last place, so truncation is covered) of a partial sum bounded by
//    the chunk's sum of magnitudes: 192u over all chunks;
//  * adding the C chunk results in fp32 registers: C u;
//  * the canonical order: 32-term chains (32u) and C chunk additions (C u).
// The total, (236 + 2C) u, is taken twice and 5 % more, in case the tensor
// cores' internal alignment drops one more bit than this model allows and
// for the rounding of ||q|| itself.
float rotate_tc_err_scale(int d) {
    const double u = 1.0 / 16777216.0;
    const double C = d / 32;
    return (float)(2.1 * (236.0 + 2.0 * C) * u);
}

cudaError_t launch_split_tf32(const float *x, float *hi, float *lo, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t blocks = (n + 255) / 256;
    split_tf32_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(x, hi, lo, n);
    return cudaGetLastError();
}

cudaError_t launch_rotate_tc(const float *q, const float *rot_hi, const float *rot_lo, float *out, int nq, int d,
                             uint32_t *status, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    if (d % BK != 0) return cudaErrorInvalidValue;
    CUtensorMap qm, hm, lm;
    if (!make_tile_map(&qm, q, (uint64_t)nq, (uint64_t)d) || !make_tile_map(&hm, rot_hi, (uint64_t)d, (uint64_t)d) ||
        !make_tile_map(&lm, rot_lo, (uint64_t)d, (uint64_t)d))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(rotate_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const long long tiles = (long long)((d + BN - 1) / BN) * ((nq + BM - 1) / BM);
    const int grid = (int)(tiles < sms ? tiles : sms);  // one persistent CTA per SM
    rotate_tc_kernel<<<grid, kThreads, kSmemBytes, s>>>(qm, hm, lm, out, nq, d, status);
    return cudaGetLastError();
}

cudaError_t launch_quantize_exact(const float *q, const float *rot, const float *qa, int nq, int d, uint32_t *planes,
                                  float4 *scal, uint32_t *recomputed, bool plane_major, cudaStream_t s) {
    if (d > kMaxD || d % 32 != 0) return cudaErrorInvalidValue;
    if (nq <= 0) return cudaSuccess;
    const size_t smem = kQxWarps * QxLayout(d).warp;
    cudaError_t e = cudaFuncSetAttribute(quantize_exact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    quantize_exact_kernel<<<(nq + kQxWarps - 1) / kQxWarps, kQxWarps * 32, smem, s>>>(
        q, rot, qa, nq, d, rotate_tc_err_scale(d), planes, scal, recomputed, plane_major ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace sqg
