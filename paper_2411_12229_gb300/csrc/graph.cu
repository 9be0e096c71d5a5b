// graph.cu -- Algorithm 2's adjust step (Sec. 3.2) on the GPU.
//
// Steps (1)-(3) of graph_host.h run here, one warp per vertex: the NSG
// pruning of every vertex's own candidates (kernel 1), then the re-pruning
// with the reverse candidates and the adaptive angle rule (kernel 2); the
// reverse-edge lists between them, the random fill, the n x R rows and the
// reachability repair stay on the host.  Every decision is the host's bit
// for bit: the exact distance in its canonical fp32 order (32 lane partial
// sums of fmaf over float4 chunks, then the xor butterfly), the same
// (distance, id) order, the same cosine arithmetic.  A vertex whose lists
// do not fit a warp's shared-memory lists (a hub with many reverse
// candidates) is marked and refined on the host with the same code.  A
// degree-unaligned graph ("w/o GR", Sec. 5) skips the angle rule.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/sqg.h"
#include "graph_host.h"

namespace {

constexpr int kWarps = 4;      // warps (vertices in flight) per block
constexpr int kCap = 512;      // entries of a warp's two long lists
constexpr int kMaxR = 64;      // longest edge list the kernels keep
constexpr int kAll = 256;      // kept + angle-rule candidates: R' + 3R' <= 4 * 64
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kFlagHost = 1u, kFlagAngle = 2u;

typedef unsigned long long u64;

// A candidate (distance, id) as one key whose unsigned order is the
// (distance, id) order: distances are sums of squares from +0, never
// negative, so their bits order like their values.
__device__ __forceinline__ u64 key_di(float d, uint32_t id) { return ((u64)__float_as_uint(d) << 32) | id; }
__device__ __forceinline__ float key_d(u64 k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ uint32_t key_id(u64 k) { return (uint32_t)k; }
// the same candidate keyed by id first (for removing repeated ids)
__device__ __forceinline__ u64 swap_halves(u64 k) { return (k << 32) | (k >> 32); }

__device__ __forceinline__ uint32_t lanes_below(int lane) { return (1u << lane) - 1u; }

// Ascending bitonic sort of a[0, cnt) by one warp; a has room for the
// next power of 2 >= max(cnt, 32), padded with the largest key.
__device__ void warp_sort(u64 *a, int cnt, int lane) {
    int N = 32;
    while (N < cnt) N <<= 1;
    for (int i = cnt + lane; i < N; i += 32) a[i] = ~0ull;
    __syncwarp();
    for (int k = 2; k <= N; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < N; i += 32) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const u64 x = a[i], y = a[ixj];
                    if ((x > y) == ((i & k) == 0)) {
                        a[i] = y;
                        a[ixj] = x;
                    }
                }
            }
            __syncwarp();
        }
}

// a[0, cnt) sorted by id-first keys: copy one entry per id to b, back in
// (distance, id) keys; returns the count.
__device__ int unique_by_id(const u64 *a, int cnt, u64 *b, int lane) {
    int m = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        const bool keep = i < cnt && (i == 0 || (a[i] >> 32) != (a[i - 1] >> 32));
        const uint32_t bal = __ballot_sync(0xffffffffu, keep);
        if (keep) b[m + __popc(bal & lanes_below(lane))] = swap_halves(a[i]);
        m += __popc(bal);
    }
    __syncwarp();
    return m;
}

// Exact squared distance of rows x and y in the canonical order; every lane
// returns the same value.
__device__ __forceinline__ float wdist(const float *x, const float *y, uint32_t nch, int lane) {
    const float4 *a = reinterpret_cast<const float4 *>(x);
    const float4 *b = reinterpret_cast<const float4 *>(y);
    float acc = 0.0f;
    for (uint32_t c = lane; c < nch; c += 32) {
        const float4 p = __ldg(a + c), q = __ldg(b + c);
        const float dx = __fsub_rn(p.x, q.x), dy = __fsub_rn(p.y, q.y);
        const float dz = __fsub_rn(p.z, q.z), dw = __fsub_rn(p.w, q.w);
        acc = __fmaf_rn(dx, dx, acc);
        acc = __fmaf_rn(dy, dy, acc);
        acc = __fmaf_rn(dz, dz, acc);
        acc = __fmaf_rn(dw, dw, acc);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    return acc;
}

// NSG's rule over c[0, m) (sorted): keep c unless a kept w has
// d(w, c) < d(u, c); at most R kept, written to kept[].  Warp-uniform.
__device__ int nsg_prune_warp(const u64 *c, int m, u64 *kept, int R, const float *data, uint32_t d, int lane) {
    const uint32_t nch = d / 4;
    int nk = 0;
    for (int i = 0; i < m && nk < R; ++i) {
        const u64 ci = c[i];
        const float *xc = data + (size_t)key_id(ci) * d;
        bool occluded = false;
        for (int j = 0; j < nk && !occluded; ++j)
            occluded = wdist(data + (size_t)key_id(kept[j]) * d, xc, nch, lane) < key_d(ci);
        if (!occluded) {
            if (lane == 0) kept[nk] = ci;
            ++nk;
            __syncwarp();
        }
    }
    return nk;
}

struct WarpLists {
    u64 a[kCap], b[kCap];
    u64 k[kMaxR];
    float s[kAll];
};

// (1) own candidates of each vertex, kept by NSG's rule.
__global__ void __launch_bounds__(kWarps * 32) adjust_prune_kernel(const float *__restrict__ data, uint64_t n,
                                                                   uint32_t d, const uint32_t *__restrict__ cand,
                                                                   uint32_t L, uint32_t Rr, u64 *c_own,
                                                                   uint32_t *c_cnt, u64 *k1, uint32_t *n1) {
    __shared__ WarpLists lists[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpLists &S = lists[w];
    const uint32_t nch = d / 4;
    for (uint64_t u = (uint64_t)blockIdx.x * kWarps + w; u < n; u += (uint64_t)gridDim.x * kWarps) {
        int m = 0;  // valid ids (L <= kCap), keyed by id
        for (uint32_t base = 0; base < L; base += 32) {
            const uint32_t t = base + lane;
            const uint32_t v = t < L ? cand[u * L + t] : kNone;
            const bool ok = v != kNone && v < n && v != u;
            const uint32_t bal = __ballot_sync(0xffffffffu, ok);
            if (ok) S.a[m + __popc(bal & lanes_below(lane))] = (u64)v << 32;
            m += __popc(bal);
        }
        __syncwarp();
        warp_sort(S.a, m, lane);
        m = unique_by_id(S.a, m, S.b, lane);
        const float *xu = data + (size_t)u * d;
        for (int i = 0; i < m; ++i) {
            const uint32_t v = key_id(S.b[i]);
            const float dd = wdist(xu, data + (size_t)v * d, nch, lane);
            if (lane == 0) S.b[i] = key_di(dd, v);
        }
        __syncwarp();
        warp_sort(S.b, m, lane);
        for (int i = lane; i < m; i += 32) c_own[u * L + i] = S.b[i];
        const int nk = nsg_prune_warp(S.b, m, S.k, (int)Rr, data, d, lane);
        for (int i = lane; i < nk; i += 32) k1[u * Rr + i] = S.k[i];
        if (lane == 0) {
            c_cnt[u] = (uint32_t)m;
            n1[u] = (uint32_t)nk;
        }
        __syncwarp();
    }
}

// (2)-(3) re-prune with the reverse candidates, then the angle rule.
__global__ void __launch_bounds__(kWarps * 32) adjust_refine_kernel(
    const float *__restrict__ data, uint64_t n, uint32_t d, uint32_t L, uint32_t Rr, const u64 *__restrict__ c_own,
    const uint32_t *__restrict__ c_cnt, const u64 *__restrict__ k1, const uint32_t *__restrict__ n1,
    const u64 *__restrict__ rev, const uint64_t *__restrict__ roff, int regular, u64 *k2, uint32_t *n2,
    uint32_t *flag) {
    __shared__ WarpLists lists[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpLists &S = lists[w];
    const uint32_t nch = d / 4;
    const int cap = d >= 512 ? 2 * (int)Rr : 3 * (int)Rr;
    for (uint64_t u = (uint64_t)blockIdx.x * kWarps + w; u < n; u += (uint64_t)gridDim.x * kWarps) {
        const uint64_t r0 = roff[u], nrev = roff[u + 1] - r0;
        const int nk1 = (int)n1[u];
        if ((uint64_t)nk1 + nrev > (uint64_t)kCap || (uint64_t)c_cnt[u] + nrev > (uint64_t)kCap) {
            if (lane == 0) flag[u] = kFlagHost;  // too long for the warp's lists
            continue;
        }
        // pool = kept edges + reverse candidates, one per id, by (distance, id)
        int np = nk1 + (int)nrev;
        for (int i = lane; i < np; i += 32)
            S.a[i] = swap_halves(i < nk1 ? k1[u * Rr + i] : rev[r0 + (i - nk1)]);
        __syncwarp();
        warp_sort(S.a, np, lane);
        np = unique_by_id(S.a, np, S.b, lane);
        warp_sort(S.b, np, lane);
        int nk = nsg_prune_warp(S.b, np, S.k, (int)Rr, data, d, lane);
        uint32_t fl = 0;
        if (regular && nk < (int)Rr) {
            fl = kFlagAngle;
            // own and reverse candidates not kept, the nearest `cap` of them
            const int nc = (int)c_cnt[u];
            int na = nc + (int)nrev;
            for (int i = lane; i < na; i += 32) S.a[i] = swap_halves(i < nc ? c_own[u * L + i] : rev[r0 + (i - nc)]);
            __syncwarp();
            warp_sort(S.a, na, lane);
            na = unique_by_id(S.a, na, S.b, lane);
            int ne = 0;
            for (int base = 0; base < na; base += 32) {
                const int i = base + lane;
                bool keep = i < na;
                if (keep)
                    for (int j = 0; j < nk; ++j) keep = keep && key_id(S.k[j]) != key_id(S.b[i]);
                const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                if (keep) S.a[ne + __popc(bal & lanes_below(lane))] = S.b[i];
                ne += __popc(bal);
            }
            __syncwarp();
            warp_sort(S.a, ne, lane);
            if (ne > cap) ne = cap;
            const int need = (int)Rr - nk;
            if (ne > 0) {
                // all = kept + extra by (distance, id)
                const int nall = nk + ne;
                for (int i = lane; i < nall; i += 32) S.b[i] = i < nk ? S.k[i] : S.a[i - nk];
                __syncwarp();
                warp_sort(S.b, nall, lane);
                // each extra candidate's largest cosine to a nearer candidate
                for (int e = 0; e < ne; ++e) {
                    const u64 ce = S.a[e];
                    const float de = key_d(ce), se = __fsqrt_rn(de);
                    const float *xe = data + (size_t)key_id(ce) * d;
                    float best = -2.0f;
                    for (int j = 0; j < nall && S.b[j] < ce; ++j) {
                        const float dw = key_d(S.b[j]);
                        const float dwc = wdist(data + (size_t)key_id(S.b[j]) * d, xe, nch, lane);
                        const float den = __fmul_rn(__fmul_rn(2.0f, __fsqrt_rn(dw)), se);
                        const float cs = den > 0.0f ? __fdiv_rn(__fsub_rn(__fadd_rn(dw, de), dwc), den) : 1.0f;
                        if (best < cs) best = cs;
                    }
                    if (lane == 0) S.s[e] = best;
                }
                __syncwarp();
                // the threshold: the take-th smallest score
                const int take = need < ne ? need : ne;
                for (int i = lane; i < ne; i += 32) {
                    const uint32_t bits = __float_as_uint(S.s[i]);
                    const uint32_t ord = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
                    S.b[i] = ((u64)ord << 32) | (uint32_t)i;
                }
                __syncwarp();
                warp_sort(S.b, ne, lane);
                const float thr = S.s[(uint32_t)S.b[take - 1]];
                // the nearest `take` candidates scoring at most the threshold
                int added = 0;
                for (int base = 0; base < ne && added < take; base += 32) {
                    const int i = base + lane;
                    const bool sel = i < ne && S.s[i] <= thr;
                    const uint32_t bal = __ballot_sync(0xffffffffu, sel);
                    const int pos = added + __popc(bal & lanes_below(lane));
                    if (sel && pos < take) S.k[nk + pos] = S.a[i];
                    added += __popc(bal);
                }
                __syncwarp();
                nk += added < take ? added : take;
                warp_sort(S.k, nk, lane);
            }
        }
        for (int i = lane; i < nk; i += 32) k2[u * Rr + i] = S.k[i];
        if (lane == 0) {
            n2[u] = (uint32_t)nk;
            flag[u] = fl;
        }
        __syncwarp();
    }
}

struct DevBufs {
    std::vector<void *> ptrs;
    ~DevBufs() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    bool alloc(T **p, size_t count) {
        void *q = nullptr;
        if (cudaMalloc(&q, sizeof(T) * (count ? count : 1)) != cudaSuccess) return false;
        ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return true;
    }
};

inline uint64_t pack_host(const sqg_graph::Cand &c) {
    uint32_t bits;
    std::memcpy(&bits, &c.d, 4);
    return ((uint64_t)bits << 32) | c.id;
}
inline sqg_graph::Cand unpack_host(uint64_t k) {
    sqg_graph::Cand c;
    const uint32_t bits = (uint32_t)(k >> 32);
    std::memcpy(&c.d, &bits, 4);
    c.id = (uint32_t)k;
    return c;
}

}  // namespace

extern "C" int sqg_build_graph_ex(const float *data, uint64_t n, uint32_t d, const uint32_t *cand, uint32_t L,
                                  uint32_t R, uint32_t entry, uint64_t seed, uint32_t flags, uint32_t *out_adj,
                                  uint64_t *out_stats, int threads, int device) {
    if ((flags & ~SQG_GRAPH_IRREGULAR) != 0) return SQG_ERR_INVALID_ARG;
    const bool regular = !(flags & SQG_GRAPH_IRREGULAR);
    if (device < 0) {
        if (out_stats) out_stats[4] = n;  // every vertex refined on the host
        return sqg_graph::build_graph_host(data, n, d, cand, L, R, entry, seed, regular, out_adj, out_stats, threads);
    }
    if (!data || !cand || !out_adj || n < 2 || d == 0 || d % 32 != 0 || R == 0 || R % 32 != 0 || L == 0 ||
        entry >= n || n > 0xFFFFFFF0ull)
        return SQG_ERR_INVALID_ARG;
    const uint32_t Rr = (uint32_t)std::min<uint64_t>(R, n - 1);
    if (L > (uint32_t)kCap || Rr > (uint32_t)kMaxR) return SQG_ERR_UNSUPPORTED;
    std::atomic<uint64_t> bad{0};
    sqg_graph::parallel_for(n, threads, [&](uint64_t v) {
        for (uint32_t i = 0; i < d; ++i)
            if (!std::isfinite(data[v * d + i])) { bad++; break; }
    }, 4096);
    if (bad.load()) return SQG_ERR_INVALID_ARG;  // the packed keys order finite distances only
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SQG_ERR_INVALID_ARG;
    }
    int rc = SQG_OK;
    {
        DevBufs B;
        float *d_data;
        uint32_t *d_cand, *c_cnt, *n1, *n2, *flag;
        u64 *c_own, *k1, *k2, *d_rev;
        uint64_t *d_roff;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        const long long want = ((long long)n + kWarps - 1) / kWarps;
        const int grid = (int)std::max(1LL, std::min<long long>(want, (long long)std::max(sms, 1) * 8));
        std::vector<u64> h_k1((size_t)n * Rr);
        std::vector<uint32_t> h_n1(n);
        std::vector<uint64_t> roff;
        std::vector<sqg_graph::Cand> rev;
        bool ok = B.alloc(&d_data, (size_t)n * d) && B.alloc(&d_cand, (size_t)n * L) && B.alloc(&c_own, (size_t)n * L) &&
                  B.alloc(&c_cnt, n) && B.alloc(&k1, (size_t)n * Rr) && B.alloc(&n1, n) &&
                  B.alloc(&k2, (size_t)n * Rr) && B.alloc(&n2, n) && B.alloc(&flag, n) && B.alloc(&d_roff, n + 1);
        if (!ok) rc = SQG_ERR_OOM;
        if (rc == SQG_OK &&
            (cudaMemcpy(d_data, data, sizeof(float) * n * d, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(d_cand, cand, sizeof(uint32_t) * n * L, cudaMemcpyHostToDevice) != cudaSuccess))
            rc = SQG_ERR_CUDA;
        if (rc == SQG_OK) {  // (1)
            adjust_prune_kernel<<<grid, kWarps * 32>>>(d_data, n, d, d_cand, L, Rr, c_own, c_cnt, k1, n1);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpy(h_k1.data(), k1, sizeof(u64) * h_k1.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(h_n1.data(), n1, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = SQG_ERR_CUDA;
        }
        std::vector<sqg_graph::Cand> k1c;
        if (rc == SQG_OK) {  // (2) reverse candidates on the host
            k1c.resize(h_k1.size());
            sqg_graph::parallel_for(n, threads, [&](uint64_t u) {
                for (uint32_t j = 0; j < h_n1[u]; ++j) k1c[u * Rr + j] = unpack_host(h_k1[u * Rr + j]);
            }, 4096);
            sqg_graph::reverse_edges(n, k1c.data(), h_n1.data(), Rr, roff, rev);
            std::vector<u64> rk(rev.size());
            for (size_t i = 0; i < rev.size(); ++i) rk[i] = pack_host(rev[i]);
            if (!B.alloc(&d_rev, rk.size())) rc = SQG_ERR_OOM;
            else if (cudaMemcpy(d_rev, rk.data(), sizeof(u64) * rk.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                     cudaMemcpy(d_roff, roff.data(), sizeof(uint64_t) * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess)
                rc = SQG_ERR_CUDA;
        }
        std::vector<u64> h_k2;
        std::vector<uint32_t> h_n2(n), h_flag(n);
        if (rc == SQG_OK) {  // (3) re-prune and angle rule
            adjust_refine_kernel<<<grid, kWarps * 32>>>(d_data, n, d, L, Rr, c_own, c_cnt, k1, n1, d_rev, d_roff,
                                                        regular ? 1 : 0, k2, n2, flag);
            h_k2.resize((size_t)n * Rr);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpy(h_k2.data(), k2, sizeof(u64) * h_k2.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(h_n2.data(), n2, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(h_flag.data(), flag, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = SQG_ERR_CUDA;
        }
        if (rc == SQG_OK) {  // (4) host refine of the marked vertices, random fill, rows; (5) reachability
            std::atomic<uint64_t> deg_sum{0}, n_supp{0}, n_fill{0}, n_host{0};
            sqg_graph::parallel_for(n, threads, [&](uint64_t u) {
                std::vector<sqg_graph::Cand> l2;
                deg_sum += h_n1[u];
                if (h_flag[u] & kFlagHost) {
                    n_host++;
                    if (sqg_graph::refine_vertex(data, n, d, cand, L, Rr, u, k1c.data() + u * Rr, h_n1[u],
                                                 rev.data() + roff[u], roff[u + 1] - roff[u], regular, l2))
                        n_supp++;
                } else {
                    for (uint32_t j = 0; j < h_n2[u]; ++j) l2.push_back(unpack_host(h_k2[u * Rr + j]));
                    if (h_flag[u] & kFlagAngle) n_supp++;
                }
                if (sqg_graph::fill_and_write(data, n, d, R, Rr, seed, u, regular, l2, out_adj)) n_fill++;
            });
            const uint64_t repairs = sqg_graph::repair_reachability(n, cand, L, R, entry, out_adj);
            if (out_stats) {
                out_stats[0] = deg_sum.load() * 1000 / n;
                out_stats[1] = n_supp.load();
                out_stats[2] = n_fill.load();
                out_stats[3] = repairs;
                out_stats[4] = n_host.load();
            }
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}
