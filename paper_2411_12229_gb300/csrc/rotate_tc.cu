// rotate_tc.cu -- the batched query rotation q' = P^-1 q (Eq. (4)) on the
// 5th-generation tensor cores, and the exact 4-bit quantization built on it.
//
// rotate_tc_kernel: one CTA computes a 128-query x 128-output tile as
// D = A B^T with A = the queries (K-major), B = the rows of P^-1 (K-major),
// accumulated in tensor memory by tcgen05.mma kind::tf32.  fp32 accuracy
// comes from splitting every operand into a tf32 high part and a tf32 low
// part: a.b ~ hi(a)hi(b) + hi(a)lo(b) + lo(a)hi(b) (three MMAs per K step).
// Operands are staged in shared memory by the CTA's threads (the split is
// done on the way) in the no-swizzle K-major core-matrix layout; one thread
// issues the MMAs and commits them to an mbarrier; four warps read the
// accumulator back with tcgen05.ld.
//
// quantize_exact_kernel: the search's decisions depend on the 4-bit codes,
// v_l and delta being exactly those of the canonical fp32 rotation (an
// fmaf chain over j = 0..d-1).  The tensor-core q' differs from it by at
// most err = c * ||q|| (a worst-case bound on both accumulations), so every
// coordinate whose code or whose role as min/max could change within err is
// recomputed with the canonical chain; the rest are decided from q'.  The
// result is bit-identical to quantizing the canonical rotation.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sqg.h"

namespace {

constexpr int BM = 128, BN = 128, BK = 32, kThreads = 128;
constexpr int kPiece = BM * BK * 4;                       // one 128 x 32 fp32 operand piece, bytes
constexpr uint32_t kCoreRowGroupBytes = (BK / 4) * 128;   // stride between 8-row groups
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) of a 128 x BK piece in the no-swizzle
// K-major layout: 8 x 16-byte core matrices, K-adjacent ones 128 B apart,
// row groups kCoreRowGroupBytes apart
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    return (uint32_t)((row >> 3) * kCoreRowGroupBytes + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N)
// byte offsets, the fixed 0b001 field at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
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

__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool bar_wait_bounded(uint32_t bar, uint32_t parity) {
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (bar_try_wait(bar, parity)) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > kWaitNs) return false;
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    rotate_tc_kernel(const float *__restrict__ q, const float *__restrict__ rot, float *__restrict__ out, int nq,
                     int d, uint32_t *status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *Ahi = sm, *Alo = sm + kPiece, *Bhi = sm + 2 * kPiece, *Blo = sm + 3 * kPiece;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.x * BM, c0 = blockIdx.y * BN;

    if (warp == 0) {  // 128 fp32 accumulator columns in tensor memory
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = 0; k0 < d && ok; k0 += BK) {
        // stage the four pieces: each thread moves float4 runs (4 consecutive k)
        for (int e = tid; e < BM * (BK / 4); e += kThreads) {
            const int row = e / (BK / 4), k = (e % (BK / 4)) * 4;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (r0 + row < nq) a = *reinterpret_cast<const float4 *>(q + (size_t)(r0 + row) * d + k0 + k);
            if (c0 + row < d) b = *reinterpret_cast<const float4 *>(rot + (size_t)(c0 + row) * d + k0 + k);
            float4 ah, al, bh, bl;
            ah.x = tf32_round(a.x); al.x = tf32_round(a.x - ah.x);
            ah.y = tf32_round(a.y); al.y = tf32_round(a.y - ah.y);
            ah.z = tf32_round(a.z); al.z = tf32_round(a.z - ah.z);
            ah.w = tf32_round(a.w); al.w = tf32_round(a.w - ah.w);
            bh.x = tf32_round(b.x); bl.x = tf32_round(b.x - bh.x);
            bh.y = tf32_round(b.y); bl.y = tf32_round(b.y - bh.y);
            bh.z = tf32_round(b.z); bl.z = tf32_round(b.z - bh.z);
            bh.w = tf32_round(b.w); bl.w = tf32_round(b.w - bh.w);
            const uint32_t off = core_off(row, k);
            *reinterpret_cast<float4 *>(Ahi + off) = ah;
            *reinterpret_cast<float4 *>(Alo + off) = al;
            *reinterpret_cast<float4 *>(Bhi + off) = bh;
            *reinterpret_cast<float4 *>(Blo + off) = bl;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int s = 0; s < BK / 8; ++s) {  // K = 8 per MMA: two core matrices
                const uint32_t ko = (uint32_t)s * 2 * 128;
                const uint64_t ah = smem_desc(saddr(Ahi) + ko, 128, kCoreRowGroupBytes);
                const uint64_t al = smem_desc(saddr(Alo) + ko, 128, kCoreRowGroupBytes);
                const uint64_t bh = smem_desc(saddr(Bhi) + ko, 128, kCoreRowGroupBytes);
                const uint64_t bl = smem_desc(saddr(Blo) + ko, 128, kCoreRowGroupBytes);
                mma_tf32(tmem, ah, bh, (k0 > 0 || s > 0) ? 1u : 0u);
                mma_tf32(tmem, ah, bl, 1u);
                mma_tf32(tmem, al, bh, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             saddr(&bar))
                         : "memory");
        }
        // the pieces are overwritten next: wait for the MMAs that read them
        ok = bar_wait_bounded(saddr(&bar), phase);
        if (!ok) bar_wait_bounded(saddr(&bar), phase);  // once more before giving up
        phase ^= 1u;
        ok = __syncthreads_and(ok);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: warp w holds accumulator rows (TMEM lanes) 32w .. 32w+31
    const int row = r0 + warp * 32 + lane;
#pragma unroll 1
    for (int cc = 0; cc < BN; cc += 32) {
        uint32_t v[32];
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(ta)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (ok && row < nq) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int col = c0 + cc + j;
                if (col < d) out[(size_t)row * d + col] = __uint_as_float(v[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
    if (!ok && tid == 0) atomicOr(status, SQG_STATUS_TIMEOUT);
}

// The canonical rotated coordinate i: fmaf chain over j = 0..d-1 from 0
// (row and query read four at a time; the order of the chain is unchanged).
__device__ __forceinline__ float canonical_coord(const float *__restrict__ rotrow, const float *__restrict__ q,
                                                 int d) {
    const float4 *r4 = reinterpret_cast<const float4 *>(rotrow);
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    float acc = 0.0f;
    for (int j = 0; j < d / 4; ++j) {
        const float4 r = r4[j], v = q4[j];
        acc = __fmaf_rn(r.x, v.x, acc);
        acc = __fmaf_rn(r.y, v.y, acc);
        acc = __fmaf_rn(r.z, v.z, acc);
        acc = __fmaf_rn(r.w, v.w, acc);
    }
    return acc;
}

constexpr int kMaxWords = 64;  // d <= 2048

// One warp per query.  qa = the tensor-core q'; err_scale * ||q|| bounds
// |qa_i - canonical_i| for every i.  Writes planes (per word w the four
// planes b as one uint4 -- [w][b] -- or, with plane_major, [b][w]) and
// (v_l, delta, Sq, 1/sqrt(d)) exactly as the canonical rotation would give.
__global__ void quantize_exact_kernel(const float *__restrict__ q, const float *__restrict__ rot,
                                      const float *__restrict__ qa, int nq, int d, float err_scale,
                                      uint32_t *__restrict__ planes, float4 *__restrict__ scal,
                                      uint32_t *__restrict__ recomputed, int plane_major) {
    const int lane = threadIdx.x & 31;
    const int qi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (qi >= nq) return;
    const int nw = d / 32;
    const float *qq = q + (size_t)qi * d;
    const float *qr = qa + (size_t)qi * d;
    float x[kMaxWords];
    uint64_t exact = 0;  // bit w: x[w] already canonical
    float ss = 0.0f;
    for (int w = 0; w < nw; ++w) {
        x[w] = qr[w * 32 + lane];
        const float v = qq[w * 32 + lane];
        ss = fmaf(v, v, ss);
    }
    for (int o = 16; o >= 1; o >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
    const float err = err_scale * sqrtf(ss) * 1.0001f + 1e-30f;
    int nrec = 0;
    // candidates for the minimum and the maximum: recompute them exactly
    float lo = x[0], hi = x[0];
    for (int w = 1; w < nw; ++w) { lo = fminf(lo, x[w]); hi = fmaxf(hi, x[w]); }
    for (int o = 16; o >= 1; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
    }
    for (int w = 0; w < nw; ++w) {
        if (x[w] <= lo + 2.0f * err || x[w] >= hi - 2.0f * err) {
            x[w] = canonical_coord(rot + (size_t)(w * 32 + lane) * d, qq, d);
            exact |= 1ull << w;
            ++nrec;
        }
    }
    // exact v_l, v_r: the same comparisons as the canonical quantizer
    const float inf = __int_as_float(0x7f800000);
    float vl = inf, vr = -inf;
    for (int w = 0; w < nw; ++w)
        if (exact >> w & 1ull) { vl = x[w] < vl ? x[w] : vl; vr = x[w] > vr ? x[w] : vr; }
    for (int o = 16; o >= 1; o >>= 1) {
        const float a = __shfl_xor_sync(0xFFFFFFFFu, vl, o), b = __shfl_xor_sync(0xFFFFFFFFu, vr, o);
        vl = a < vl ? a : vl;
        vr = b > vr ? b : vr;
    }
    const float range = __fsub_rn(vr, vl);
    const float delta = range > 0.0f ? __fdiv_rn(range, 15.0f) : 0.0f;
    const float inv = range > 0.0f ? __fdiv_rn(15.0f, range) : 0.0f;
    const float margin = err * inv * 1.01f + 1e-4f;  // in units of the code
    int sq = 0;
    for (int w = 0; w < nw; ++w) {
        int t = 0;
        if (range > 0.0f) {
            float y = __fadd_rn(__fmul_rn(__fsub_rn(x[w], vl), inv), 0.5f);
            if (!(exact >> w & 1ull)) {
                // an integer boundary (1 .. 15) within the margin: decide exactly
                const float nearest = fminf(fmaxf(rintf(y), 1.0f), 15.0f);
                if (fabsf(y - nearest) <= margin) {
                    x[w] = canonical_coord(rot + (size_t)(w * 32 + lane) * d, qq, d);
                    ++nrec;
                    y = __fadd_rn(__fmul_rn(__fsub_rn(x[w], vl), inv), 0.5f);
                }
            }
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
    nrec = __reduce_add_sync(0xFFFFFFFFu, nrec);
    if (lane == 0) {
        scal[qi] = make_float4(vl, delta, (float)sq, __fdiv_rn(1.0f, __fsqrt_rn((float)d)));
        if (recomputed) atomicAdd(recomputed, (uint32_t)nrec);
    }
}

}  // namespace

namespace sqg {

// Bound on |tensor-core q'_i - canonical q'_i| per unit of ||q||, with
// u = 2^-24 and sum_j |P_ij q_j| <= ||P_i|| ||q|| = ||q||:
//  * the 3xTF32 split drops lo(a)lo(b) and the tf32 rounding of both low
//    parts: at most 3 * 2^-22 = 12u of every |P_ij q_j|;
//  * the tensor cores add 3d exact tf32 products in fp32; every addition is
//    taken to err by at most 2u (one unit in the last place, so truncation
//    is covered) of a partial sum bounded by the sum of magnitudes: 6d u;
//  * the canonical chain rounds each of its d fmaf once: d u.
// The total, (7d + 12) u, is doubled in case the tensor cores' internal
// alignment drops one more bit than this model allows.
float rotate_tc_err_scale(int d) {
    const double u = 1.0 / 16777216.0;
    return (float)(2.0 * (7.0 * d + 12.0) * u);
}

cudaError_t launch_rotate_tc(const float *q, const float *rot, float *out, int nq, int d, uint32_t *status,
                             cudaStream_t s) {
    const int smem = 4 * kPiece;
    cudaError_t e = cudaFuncSetAttribute(rotate_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((nq + BM - 1) / BM, (d + BN - 1) / BN);
    rotate_tc_kernel<<<grid, kThreads, smem, s>>>(q, rot, out, nq, d, status);
    return cudaGetLastError();
}

cudaError_t launch_quantize_exact(const float *q, const float *rot, const float *qa, int nq, int d, uint32_t *planes,
                                  float4 *scal, uint32_t *recomputed, bool plane_major, cudaStream_t s) {
    if (d / 32 > kMaxWords) return cudaErrorInvalidValue;
    const int wpb = 4;
    quantize_exact_kernel<<<(nq + wpb - 1) / wpb, wpb * 32, 0, s>>>(q, rot, qa, nq, d, rotate_tc_err_scale(d),
                                                                   planes, scal, recomputed, plane_major ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace sqg
