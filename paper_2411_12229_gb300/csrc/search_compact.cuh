// search_compact.cuh -- the compact search kernel: one warp per query for
// d <= 1024, out-degree 32 or 64, k <= 32 and ef <= 128 (for d <= 256 also
// k <= 128 and ef <= 256), with multiple estimates (instantiated in
// search_compact.cu for d <= 256, search_compact_wide.cu for 256 < d <=
// 1024, search_compact_stop.cu with the learned stop and
// search_compact_big.cu for d <= 256 past k 32 or ef 128).
//
// It runs the same Algorithm 1 (Querying, Sec. 3.1.3) with multiple
// estimated distances and implicit re-ranking (Sec. 3.1.2) as
// search_kernel, takes every decision in the same precision and order, and
// returns the same ids, distances, hop counts and status bits; what differs
// is the bookkeeping, cut to a few warp instructions per step:
//
//   * a beam entry is one 64-bit word, (order-preserving key bits << 32) |
//     (id << 1) | visited, so the (key, id) order of reading R4 is one
//     unsigned compare and a duplicate (key, id) is one xor;
//   * the beam (at most 32 NB entries: NB = 2 for ef <= 64, 4 for ef <=
//     128, 8 for ef <= 256) sits in shared memory, sorted, and lane l also keeps entries
//     l + 32 s (s < NB) in registers for the select and the visited marks;
//     all 32 NB slots are always written, the empty entry (greater than
//     every entry, visited bit set) from the beam's length on, so the
//     binary search, the select and the marks need no bound on the length;
//   * the admitted candidates' beam positions come from a branch-free
//     binary search; the merged beam is gathered into the other of two
//     beam buffers, each output slot finding its source from a 32 NB-bit
//     mask of the candidates' final positions (no shifting loop);
//   * the k <= 32 RK results live in registers, lane l holding results
//     l + 32 s (s < RK);
//   * with out-degree 64 (NR = 2) lane l estimates neighbours l and l + 32
//     and the step's candidates are staged 64 wide.
//
// The next vertex -- the smaller of the best admitted candidate and the
// first unvisited beam entry -- is known as soon as the estimates are, so
// its block copy (1-D bulk copy into shared memory, Sec. 3.1.4's
// prefetch) is issued before the merge, which then runs while the copy is
// in flight, together with the marks of the vertex's copies in the beam
// and its visited-set insert (one warp-wide probe of 32 slots).
#pragma once
#include "search.cuh"

namespace sqg {

namespace compact {

constexpr uint64_t kNone = ~0ull;  // an empty beam or result slot (greater than every entry)

// The learned stop's state carried from hop to hop (12 bytes of the warp's
// shared memory after its mbarrier).
struct StopCarry {
    int last_improve;
    float ema_improve, ema_insert;
};

// Order-preserving map of a float key (never NaN) to uint32: a < b as floats
// iff map(a) < map(b) as unsigned integers; -0 and +0 map to one value, as
// they compare equal as floats.
__device__ __forceinline__ uint32_t key_bits(float f) {
    const uint32_t b = __float_as_uint(__fadd_rn(f, 0.0f));  // -0 + 0 = +0
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ uint64_t pack_entry(uint32_t kb, uint32_t id) {
    return ((uint64_t)kb << 32) | ((uint64_t)id << 1);
}
__device__ __forceinline__ uint32_t entry_id(uint64_t e) { return (uint32_t)(e >> 1) & kIdMask; }
__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    const uint32_t lo = __shfl_sync(kFull, (uint32_t)v, src), hi = __shfl_sync(kFull, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t shfl64_up(uint64_t v, int d) {
    const uint32_t lo = __shfl_up_sync(kFull, (uint32_t)v, d), hi = __shfl_up_sync(kFull, (uint32_t)(v >> 32), d);
    return ((uint64_t)hi << 32) | lo;
}

// Insert an id that is not in the table (an unvisited vertex) with the
// whole warp: lane l reads probe slot s + l, and the first empty slot of the
// window is the one a slot-by-slot linear probe would take.
__device__ __forceinline__ void hash_insert_warp(uint32_t *H, uint32_t bits, uint32_t id, int lane) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t s = hslot(id, bits);
    for (;;) {
        const uint32_t slot = (s + lane) & mask;
        const uint32_t emp = __ballot_sync(kFull, H[slot] == kEmpty);
        if (emp) {
            if (lane == __ffs(emp) - 1) H[slot] = id;
            __syncwarp();
            return;
        }
        s += 32;
    }
}

// S = sum_i b_i qbar_i (Sec. 3.1.1) of neighbours lane + 32 t (t < NR):
// AND + popc of their code words against the 4 bit-planes, out-degree R =
// 32 NR (word w of neighbour j at w * R + j); nw <= 4 * CH words, the
// plane word loaded once for the NR neighbours.
template <int CH, int NR>
__device__ __forceinline__ void estimate_SN(const unsigned char *codes_b, const uint32_t *planes, uint32_t nw,
                                            int lane, int (&S)[NR]) {
    constexpr uint32_t R = 32 * NR;
    const uint32_t *codes = reinterpret_cast<const uint32_t *>(codes_b) + lane;
    const uint4 *pl = reinterpret_cast<const uint4 *>(planes);
    int s0[NR], s1[NR], s2[NR], s3[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t) s0[t] = s1[t] = s2[t] = s3[t] = 0;
    auto word = [&](uint32_t w) {
        const uint4 p = pl[w];
#pragma unroll
        for (int t = 0; t < NR; ++t) {
            const uint32_t c = codes[w * R + 32 * t];
            s0[t] += __popc(c & p.x);
            s1[t] += __popc(c & p.y);
            s2[t] += __popc(c & p.z);
            s3[t] += __popc(c & p.w);
        }
    };
    if constexpr (CH <= 2) {
#pragma unroll
        for (uint32_t w = 0; w < 4 * CH; ++w)
            if (w < nw) word(w);
    } else {
#pragma unroll 4
        for (uint32_t w = 0; w < nw; ++w) word(w);
    }
#pragma unroll
    for (int t = 0; t < NR; ++t) S[t] = s0[t] + 2 * s1[t] + 4 * s2[t] + 8 * s3[t];
}

// The key of neighbour j from its S (the estimator of Sec. 3.1.1 and the
// bound-shifted key of reading R7), out-degree R: the same operations in
// the same order as estimate_from_S.
template <int R>
__device__ __forceinline__ float keyR(const float *fac, const QuerySide &qs, uint32_t d, int j, int S, float dist_c,
                                      float sqrt_dc, float eps0) {
    const float f_add = fac[j], f_rescale = fac[R + j];
    const int pc = (int)reinterpret_cast<const uint32_t *>(fac)[3 * R + j];
    const float A = (float)(2 * S - qs.sq);
    const float B = __fmul_rn(qs.vl, (float)(2 * pc - (int)d));
    const float ip = __fmul_rn(__fmaf_rn(qs.delta, A, B), qs.inv_sqrt_d);
    const float est = __fmaf_rn(f_rescale, ip, __fadd_rn(f_add, dist_c));
    if (eps0 == 0.0f) return est;
    const float bound = __fmul_rn(fac[2 * R + j], sqrt_dc);
    return __fsub_rn(est, __fmul_rn(eps0, bound));
}

// The key a packed entry holds (the inverse of key_bits; -0 comes back as +0).
__device__ __forceinline__ float entry_key(uint64_t e) {
    const uint32_t kb = (uint32_t)(e >> 32);
    return __uint_as_float((kb & 0x80000000u) ? (kb & 0x7FFFFFFFu) : ~kb);
}

// Entry s of a lane's NB beam registers, s warp-uniform (an unrolled
// select: no local-memory array).
template <int NB>
__device__ __forceinline__ uint64_t pick(const uint64_t (&b)[NB], int s) {
    uint64_t v = b[0];
#pragma unroll
    for (int t = 1; t < NB; ++t)
        if (s == t) v = b[t];
    return v;
}

}  // namespace compact

// CH: float4 chunks of the raw vector per lane (d <= 128 CH).  NR:
// neighbours per lane (out-degree 32 NR).  NB: beam slots per lane (2: ef <=
// 64, 4: ef <= 128, 8: ef <= 256).  MINB: resident blocks of 4 warps per SM
// the build is made for (d <= 256 with NR 1: NB 2: 8 for up to 64 registers
// or 9 for 56; NB 4: 7 for up to 72 or 8 for 64).  STOP: the build with the
// learned early stop fused (the same features, network and decision points
// as search_kernel's, so the same hops, results and status bits).  RK:
// result slots per lane (1: k <= 32, 4: k <= 128), lane l holding results
// l + 32 s.
template <int CH, int NR, int NB, int MINB, bool STOP = false, int RK = 1>
__global__ void __launch_bounds__(128, MINB) search_compact_kernel(const SearchArgs a) {
    using namespace compact;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t d = a.d, nch = d / 4;
    unsigned char *ws = smem + (size_t)warp * a.warp_bytes;
    unsigned char *const buf = ws + a.o_buf0;
    uint64_t *const bar = reinterpret_cast<uint64_t *>(ws + a.o_bar);
    uint64_t *beam_a = reinterpret_cast<uint64_t *>(ws + a.o_beam);  // two buffers of 32 NB entries
    uint64_t *beam_b = beam_a + 32 * NB;
    uint64_t *const stage = reinterpret_cast<uint64_t *>(ws + a.o_spos);  // this step's candidates by rank
    uint32_t *const planes = reinterpret_cast<uint32_t *>(ws + a.o_planes);
    const uint32_t gwarp = blockIdx.x * (blockDim.x >> 5) + warp;
    uint32_t *const Hs = reinterpret_cast<uint32_t *>(ws + a.o_hash);
    uint32_t *const Hg = a.ghash ? a.ghash + ((size_t)gwarp << a.hash_bits) : nullptr;
    const Team<32> tm(lane);

    if (lane == 0) mbar_init(&bar[0], 1);
    fence_mbar_init();
    __syncwarp();
    uint32_t phase = 0;
    bool healthy = true;

    while (healthy) {
        int qi = 0;
        if (lane == 0) qi = (int)atomicAdd(a.queue_head, 1u);
        qi = __shfl_sync(kFull, qi, 0);
        if (qi >= a.nq) break;
        const int k = a.k[qi], ef = a.ef[qi];
        const long long off = a.uniform_k ? (long long)qi * a.uniform_k : a.offsets[qi];
        uint32_t status = 0;
        if (!(k >= 1 && k <= a.max_k && ef >= k && ef <= a.max_ef && (!a.uniform_k || k == a.uniform_k))) {
            const int kk = a.uniform_k ? a.uniform_k : (k < 0 ? 0 : (k > SQG_MAX_K ? SQG_MAX_K : k));
            for (int t = lane; t < kk; t += 32) {
                a.out_ids[off + t] = SQG_NO_ID;
                a.out_dists[off + t] = __int_as_float(0x7f800000);
            }
            if (lane == 0) {
                if (a.stats) a.stats[qi] = sqg_query_stats{0u, SQG_STATUS_BAD_PARAM};
                atomicOr(a.status_word, SQG_STATUS_BAD_PARAM);
            }
            continue;
        }
        const int hop_cap = a.hop_cap > 0 ? a.hop_cap : 4 * ef + 64;

        // ---- query setup: raw query in registers, quantized rotated query planes
        float4 qv[CH];
        const float4 *q4 = reinterpret_cast<const float4 *>(a.queries + (size_t)qi * d);
#pragma unroll
        for (int t = 0; t < CH; ++t) {
            const uint32_t c = lane + 32 * t;
            qv[t] = c < nch ? q4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        QuerySide qs;
        if (a.qplanes) {
            const uint4 *src = reinterpret_cast<const uint4 *>(a.qplanes + (size_t)qi * 4 * (d / 32));
            if (lane < (int)(d / 32)) reinterpret_cast<uint4 *>(planes)[lane] = src[lane];
            const float4 sc = a.qscal[qi];
            qs.vl = sc.x;
            qs.delta = sc.y;
            qs.sq = (int)sc.z;
            qs.inv_sqrt_d = sc.w;
        } else {
            qs = quantize_team<32>(a.qrot + (size_t)qi * d, d, planes, tm);
        }
        uint32_t *H = Hs;
        uint32_t hbits = a.shash_bits;
        for (uint32_t i = lane; i < (1u << hbits); i += 32) H[i] = kEmpty;

        // ---- Algorithm 1, line 1: the beam holds the entry, which is expanded
        // first (its key, its exact distance, is set at that expansion)
        int m = 1;
        uint64_t b[NB];  // b[s] = beam[lane + 32 s]
#pragma unroll
        for (int s = 0; s < NB; ++s) {
            b[s] = s == 0 && lane == 0 ? pack_entry(0u, a.entry) | 1ull : kNone;
            beam_a[lane + 32 * s] = b[s];  // all 32 NB slots, kNone from m on: no bound on m below
        }
        uint64_t res[RK];  // res[s] = result[lane + 32 s], for lane + 32 s < k
#pragma unroll
        for (int s = 0; s < RK; ++s) res[s] = kNone;
        uint64_t rworst = kNone;  // result[k - 1]: the entry a new result must beat
        uint64_t bworst = kNone;  // beam[ef - 1] once the beam holds ef entries (the early cut)
        uint32_t p = a.entry;
        __syncwarp();
        hash_insert_warp(H, hbits, p, lane);
        if (lane == 0) {
            fence_proxy_async();
            bulk_fetch(buf, a.blocks + (size_t)p * a.block_bytes, a.block_bytes, &bar[0]);
        }
        int hops = 1;
        // learned-stop state (STOP builds): the last hop whose vertex entered
        // the result and the moving averages of entering and of the inserted
        // share, kept by lane 0 in shared memory beside the barrier (no
        // registers held across the loop)
        StopCarry *const sst = reinterpret_cast<StopCarry *>(ws + a.o_bar + 8);
        if (STOP && lane == 0)
            *sst = StopCarry{0, 0.0f, 0.0f};

        for (;;) {
            if (!mbar_wait_bounded(&bar[0], phase & 1u)) {
                status |= SQG_STATUS_TIMEOUT;
                healthy = false;
                break;
            }
            phase ^= 1u;
            const unsigned char *blk = buf;

            // ---- line 4: exact distance (implicit re-ranking); the neighbours'
            // integer sums S while the distance's butterfly is in flight
            float dacc[1];
            exact_partial<CH, 32>(reinterpret_cast<const float4(&)[1][CH]>(qv),
                                  reinterpret_cast<const float *>(blk), nch, tm, dacc);
            uint32_t cid[NR];
            int S[NR];
#pragma unroll
            for (int t = 0; t < NR; ++t) cid[t] = reinterpret_cast<const uint32_t *>(blk + a.off_ids)[lane + 32 * t];
            estimate_SN<CH, NR>(blk + a.off_codes, planes, d / 32, lane, S);
            const float dist_c = exact_reduce<32>(dacc, tm);
            if (hops == 1) {  // reading R8: the entry's key is its exact distance
                if (lane == 0) {
                    b[0] = pack_entry(key_bits(dist_c), p) | 1ull;
                    beam_a[0] = b[0];
                }
                __syncwarp();
                if (ef == 1) bworst = shfl64(b[0], 0);
            }
            bool improved = false;
            {  // result top-k in registers: (dist bits << 32) | id, dist >= 0
                const uint64_t r = ((uint64_t)__float_as_uint(dist_c) << 32) | p;
                if (r < rworst) {
                    improved = true;
                    int pos = 0;
#pragma unroll
                    for (int s = 0; s < RK; ++s) pos += __popc(__ballot_sync(kFull, lane + 32 * s < k && res[s] < r));
                    // entries pos .. k - 2 move up one slot: slot j takes old j - 1
                    // (lane 0 of row s from lane 31 of row s - 1)
                    uint64_t up[RK];
#pragma unroll
                    for (int s = 0; s < RK; ++s) {
                        const uint64_t u = shfl64_up(res[s], 1);
                        const uint64_t c = s > 0 ? shfl64(res[s > 0 ? s - 1 : 0], 31) : kNone;
                        up[s] = lane == 0 ? c : u;
                    }
#pragma unroll
                    for (int s = 0; s < RK; ++s) {
                        const int j = lane + 32 * s;
                        if (j == pos) res[s] = r;
                        else if (j > pos && j < k) res[s] = up[s];
                    }
                    rworst = shfl64(pick<RK>(res, (k - 1) >> 5), (k - 1) & 31);
                }
            }

            // ---- line 5: the estimate and key of every neighbour from the same block
            const float sqrt_dc = a.eps0 == 0.0f ? 0.0f : __fsqrt_rn(dist_c);
            uint64_t cand[NR];
            bool adm[NR];
            uint32_t am[NR], anyam = 0;
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                const float key = keyR<32 * NR>(reinterpret_cast<const float *>(blk + a.off_factors), qs, d,
                                                lane + 32 * t, S[t], dist_c, sqrt_dc, a.eps0);
                cand[t] = pack_entry(key_bits(key), cid[t]);
                // ---- line 6: unvisited neighbours enter the beam; an entry the
                // cut to ef would drop at once is skipped early
                adm[t] = cid[t] != kEmpty && cand[t] < bworst;
                if (adm[t]) adm[t] = !hash_contains(H, hbits, cid[t]);
                am[t] = __ballot_sync(kFull, adm[t]);
                anyam |= am[t];
            }

            // ---- lines 2-3 of the next step, taken now (Sec. 3.1.4: the next
            // block is fetched while this step's merge runs): the next vertex
            // is the smaller of the best admitted candidate and the first
            // unvisited beam entry.  A candidate equal in (key, id) to a beam
            // entry (dropped below as a duplicate) names that entry's vertex,
            // which is unvisited, so it may stand in for it here.
            uint64_t nxt;
            {  // the smallest of the lane's admitted candidates and unvisited
               // entries, then the warp's smallest (high word, then low word)
                uint64_t v = kNone;
#pragma unroll
                for (int t = 0; t < NR; ++t) v = adm[t] && cand[t] < v ? cand[t] : v;
#pragma unroll
                for (int s = 0; s < NB; ++s) v = !(b[s] & 1ull) && b[s] < v ? b[s] : v;  // kNone: visited
                const uint32_t chi = __reduce_min_sync(kFull, (uint32_t)(v >> 32));
                const uint32_t clo = __reduce_min_sync(kFull, (uint32_t)(v >> 32) == chi ? (uint32_t)v : 0xFFFFFFFFu);
                nxt = ((uint64_t)chi << 32) | clo;
            }
            if constexpr (!STOP) {  // (with the stop these two ends follow its decision)
                if (nxt == kNone) break;  // no unvisited entry: the search ends (line 2)
                if (hops >= hop_cap) {    // reading R6
                    status |= SQG_STATUS_CAPACITY;
                    break;
                }
            }
            const bool go = !STOP || (nxt != kNone && hops < hop_cap);  // a next expansion follows
            const uint32_t pn = entry_id(nxt);
            __syncwarp();  // every lane's reads of the current block are done
            if (go && lane == 0) {
                fence_proxy_async();
                bulk_fetch(buf, a.blocks + (size_t)pn * a.block_bytes, a.block_bytes, &bar[0]);
            }
            int inserted = 0;  // this step's candidates kept by the cut (the stop's features)

            // ---- line 6: merge the admitted candidates, cut the beam to ef
            const uint64_t *B = beam_a;
            int pos[NR];
            if (anyam) {
                anyam = 0;
#pragma unroll
                for (int t = 0; t < NR; ++t) {
                    // beam position (lower bound) by a branch-free binary search;
                    // an identical (key, id) already in the beam is dropped
                    pos[t] = 0;
#pragma unroll
                    for (int step = 16 * NB; step >= 1; step >>= 1) {
                        const int u = pos[t] + step;
                        if (B[u - 1] < cand[t]) pos[t] = u;  // kNone from m on: pos <= m
                    }
                    if (adm[t] && ((B[pos[t]] ^ cand[t]) >> 1) == 0) adm[t] = false;
                    am[t] = __ballot_sync(kFull, adm[t]);
                    anyam |= am[t];
                }
            }
            if (anyam) {
                // rank among the admitted candidates (their ids are distinct):
                // the candidates are compacted into the stage, and every lane
                // counts the smaller ones with broadcast reads
                int nadm = 0;
#pragma unroll
                for (int t = 0; t < NR; ++t) {
                    if (adm[t]) stage[nadm + __popc(am[t] & ((1u << lane) - 1u))] = cand[t];
                    nadm += __popc(am[t]);
                }
                __syncwarp();
                int rank[NR];
#pragma unroll
                for (int t = 0; t < NR; ++t) rank[t] = 0;
                int j = 0;
#pragma unroll 2
                for (; j + 2 <= nadm; j += 2) {  // two staged candidates per 16-byte read
                    const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(stage + j);
#pragma unroll
                    for (int t = 0; t < NR; ++t) rank[t] += (v.x < cand[t] ? 1 : 0) + (v.y < cand[t] ? 1 : 0);
                }
                if (j < nadm) {
                    const uint64_t v = stage[j];
#pragma unroll
                    for (int t = 0; t < NR; ++t) rank[t] += v < cand[t] ? 1 : 0;
                }
                __syncwarp();
                int fp[NR];  // final positions in the merged beam
#pragma unroll
                for (int t = 0; t < NR; ++t) {
                    fp[t] = pos[t] + rank[t];
                    if (adm[t]) stage[rank[t]] = cand[t];
                    if constexpr (STOP) inserted += __popc(__ballot_sync(kFull, adm[t] && fp[t] < ef));
                }
                uint32_t mk[NB];  // bit l of mk[s]: a candidate lands in slot 32 s + l
#pragma unroll
                for (int s = 0; s < NB; ++s) {
                    uint32_t bits = 0;
#pragma unroll
                    for (int t = 0; t < NR; ++t) bits |= adm[t] && (fp[t] >> 5) == s ? 1u << (fp[t] & 31) : 0u;
                    mk[s] = __reduce_or_sync(kFull, bits);
                }
                const int m2 = min(ef, m + nadm);
                uint64_t *Bn = beam_b;
                __syncwarp();
                // output slot o: a candidate if bit o of the mask is set (the one
                // of rank = candidates placed before o), else old entry o - that count
                int cbase = 0;
#pragma unroll
                for (int s = 0; s < NB; ++s) {
                    const int o = lane + 32 * s;
                    const int c = cbase + __popc(mk[s] & ((1u << lane) - 1u));
                    const uint64_t v = o < m2 ? (((mk[s] >> lane) & 1u) ? stage[c] : B[o - c]) : kNone;
                    Bn[o] = v;
                    b[s] = v;
                    cbase += __popc(mk[s]);
                }
                beam_b = beam_a;
                beam_a = Bn;
                m = m2;
                // (a visited mark set below does not matter to the early cut: no
                // candidate shares an id with a visited entry)
                bworst = m == ef ? shfl64(pick<NB>(b, (ef - 1) >> 5), (ef - 1) & 31) : kNone;
            }

            // ---- learned early stop (not in the paper): after the merge, on
            // the merged beam, before the next vertex is marked -- the point
            // where search_kernel takes it
            if constexpr (STOP) {
                constexpr float inv_R = 1.0f / (32 * NR);  // a power of 2: exact, the division's value
                if (lane == 0) {
                    if (improved) sst->last_improve = hops;
                    sst->ema_improve =
                        __fadd_rn(__fmul_rn(0.75f, sst->ema_improve), __fmul_rn(0.25f, improved ? 1.0f : 0.0f));
                    sst->ema_insert =
                        __fadd_rn(__fmul_rn(0.75f, sst->ema_insert), __fmul_rn(0.25f, __fmul_rn((float)inserted, inv_R)));
                }
                // hops mod the period by a multiply-high with the host's
                // 2^64 / period + 1, exact for every hops < 2^32
                const uint64_t hq = __umul64hi((uint64_t)hops, a.stop_magic);
                const bool eval_now = a.stop_every == 1 || (uint64_t)hops == hq * (uint64_t)a.stop_every;
                if (a.stop_every > 0 && eval_now && rworst != kNone) {
                    // lane 0's stop state is visible to every lane after this, and
                    // the gather's reads of both beam buffers and the stage are done
                    __syncwarp();
                    const float rk = __uint_as_float((uint32_t)(rworst >> 32));
                    const float rk2 = __fmul_rn(1.25f, rk);
                    int u = 0, near1 = 0, near2 = 0;  // unvisited; of them with key <= rk, <= 1.25 rk
#pragma unroll
                    for (int s = 0; s < NB; ++s) {
                        const bool un = !(b[s] & 1ull);  // kNone reads as visited
                        const float kk = un ? entry_key(b[s]) : 0.0f;
                        u += __popc(__ballot_sync(kFull, un));
                        near1 += __popc(__ballot_sync(kFull, un && kk <= rk));
                        near2 += __popc(__ballot_sync(kFull, un && kk <= rk2));
                    }
                    const float den = rk > 1e-20f ? rk : 1e-20f;
                    const float since = (float)(hops - sst->last_improve);
                    const float inv_ef = __fdiv_rn(1.0f, (float)ef), inv_den = __fdiv_rn(1.0f, den);
                    const float inv_k = __fdiv_rn(1.0f, (float)k);
                    const float inv_h1 = __fdiv_rn(1.0f, __fadd_rn((float)hops, 1.0f));
                    const float r0 = __uint_as_float((uint32_t)(shfl64(res[0], 0) >> 32));
                    // d <= 256 (builds at their register limit): the features go to
                    // the beam buffer the next merge writes (idle until then), each
                    // as soon as it is known, so that few registers hold them;
                    // larger d: registers.  The stage holds the hidden layer.
                    constexpr bool kFeatSmem = CH <= 2;
                    float *const fs = reinterpret_cast<float *>(beam_b);
                    float f[SQG_MLP_IN];
                    auto put = [&](int i, float v) {
                        if constexpr (kFeatSmem) {
                            if (lane == 0) fs[i] = clamp8(v);
                        } else {
                            f[i] = clamp8(v);
                        }
                    };
                    put(0, __fmul_rn((float)hops, inv_ef));
                    put(1, __fmul_rn(since, inv_ef));
                    put(2, __fmul_rn((float)u, inv_ef));
                    put(3, __fmul_rn((float)m, inv_ef));
                    put(4, __fmul_rn(r0, inv_den));
                    put(5, u > 0 ? __fmul_rn(entry_key(nxt), inv_den) : 0.0f);  // nxt: the first unvisited entry
                    put(6, __fmul_rn(dist_c, inv_den));
                    put(7, __fmul_rn((float)inserted, inv_R));
                    put(8, __fmul_rn((float)k, inv_ef));
                    put(9, sst->ema_improve);
                    put(10, sst->ema_insert);
                    put(11, __fmul_rn((float)near1, inv_k));
                    put(12, __fmul_rn((float)near2, inv_k));
                    put(13, __fmul_rn(since, inv_h1));
                    put(14, dist_c <= rk ? 1.0f : 0.0f);
                    put(15, __fmul_rn((float)k, 0.01f));
                    __syncwarp();
                    float logit;
                    if constexpr (kFeatSmem)
                        logit = mlp_logit_warp(a.mlp, static_cast<const float *>(fs), lane, reinterpret_cast<float *>(stage));
                    else
                        logit = mlp_logit_warp(a.mlp, f, lane, reinterpret_cast<float *>(stage));
                    if (logit > a.stop_logit) {
                        status |= SQG_STATUS_LEARNED_STOP;
                        if (go) {  // the copy issued for the next vertex completes unused
                            if (mbar_wait_bounded(&bar[0], phase & 1u)) {
                                phase ^= 1u;
                            } else {
                                status |= SQG_STATUS_TIMEOUT;
                                healthy = false;
                            }
                        }
                        break;
                    }
                }
                if (nxt == kNone) break;  // no unvisited entry: the search ends (line 2)
                if (hops >= hop_cap) {    // reading R6
                    status |= SQG_STATUS_CAPACITY;
                    break;
                }
            }

            // ---- line 3: the next vertex is visited; every copy of it in the
            // beam is marked (reading R5: the copies keep their slots)
            p = pn;
#pragma unroll
            for (int s = 0; s < NB; ++s)
                if ((uint32_t)b[s] == p << 1) {  // id p, not yet visited (ids < 2^31)
                    b[s] |= 1ull;
                    beam_a[lane + 32 * s] = b[s];
                }
            hash_insert_warp(H, hbits, p, lane);  // its closing __syncwarp also orders the marks above
            ++hops;
            if (Hg && H == Hs && (uint32_t)hops >= (1u << hbits) / 2) {
                hash_migrate<32>(Hs, hbits, Hg, a.hash_bits, tm);
                H = Hg;
                hbits = a.hash_bits;
            }
        }
        // ---- line 8: the k nearest expanded vertices by exact distance
        const bool ok = !(status & SQG_STATUS_TIMEOUT);
#pragma unroll
        for (int s = 0; s < RK; ++s) {
            const int j = lane + 32 * s;
            if (j < k) {
                const bool have = ok && res[s] != kNone;
                a.out_ids[off + j] = have ? (uint32_t)res[s] : SQG_NO_ID;
                a.out_dists[off + j] = have ? __uint_as_float((uint32_t)(res[s] >> 32)) : __int_as_float(0x7f800000);
            }
        }
        if (lane == 0) {
            if (a.stats) a.stats[qi] = sqg_query_stats{(uint32_t)hops, status};
            if (status) atomicOr(a.status_word, status);
        }
        __syncwarp();
    }
}

template <int CH, int NR, int NB, int MINB, bool STOP = false, int RK = 1>
static cudaError_t compact_launch_one(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const SearchArgs &a) {
    auto fn = search_compact_kernel<CH, NR, NB, MINB, STOP, RK>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int CH, int NR, int NB, int MINB, bool STOP = false, int RK = 1>
static cudaError_t compact_occ_one(int block, size_t smem, int *nb) {
    auto fn = search_compact_kernel<CH, NR, NB, MINB, STOP, RK>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, fn, block, smem);
}

}  // namespace sqg
