// shard_merge.cu -- the merge step of a search sharded over several graphs.
//
// When an index is split into S shards, each with its own graph (built by
// Algorithm 2 on the shard's vectors alone), every query is searched in
// every shard and the S per-shard top-k lists -- each sorted by (distance,
// id) as Algorithm 1's output is (reading R4) -- are merged into one global
// top-k.  Shard s's local ids are offset by offsets[s] into the global id
// space.  One warp per query runs a k-step S-way merge: lane s holds the
// head of list s, and each step takes the smallest (distance, global id)
// head by two warp reductions and advances that list.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sqg.h"

namespace {

constexpr int kMergeWarps = 4;
constexpr uint32_t kFullMask = 0xFFFFFFFFu;

struct MergeArgs {
    const uint32_t *ids;
    const float *dists;
    int S, nq, k;
    uint32_t offsets[SQG_MAX_SHARDS];
    uint32_t *out_ids;
    float *out_dists;
};

// (distance bits, global id) of list entry t of shard s for query qi; the
// distances are >= 0 (squared distances) or +inf padding, so their bits
// order as unsigned integers; padding (SQG_NO_ID) sorts last.
__device__ __forceinline__ void head(const MergeArgs &a, int s, int qi, int t, uint32_t &db, uint32_t &gid) {
    if (s >= a.S || t >= a.k) {
        db = 0xFFFFFFFFu;
        gid = 0xFFFFFFFFu;
        return;
    }
    const size_t i = ((size_t)s * a.nq + qi) * a.k + t;
    const uint32_t id = a.ids[i];
    if (id == SQG_NO_ID) {
        db = 0x7F800000u;  // +inf
        gid = 0xFFFFFFFFu;
        return;
    }
    db = __float_as_uint(a.dists[i]);
    gid = id + a.offsets[s];
}

__global__ void __launch_bounds__(kMergeWarps * 32) merge_topk_kernel(const MergeArgs a) {
    const int lane = threadIdx.x & 31;
    const int qi = blockIdx.x * kMergeWarps + (threadIdx.x >> 5);
    if (qi >= a.nq) return;  // uniform over the warp
    int pos = 0;             // list `lane`'s next entry
    uint32_t db, gid;
    head(a, lane, qi, 0, db, gid);
    for (int t = 0; t < a.k; ++t) {
        const uint32_t dmin = __reduce_min_sync(kFullMask, db);
        const uint32_t imin = __reduce_min_sync(kFullMask, db == dmin ? gid : 0xFFFFFFFFu);
        const size_t o = (size_t)qi * a.k + t;
        if (lane == 0) {
            const bool pad = imin == 0xFFFFFFFFu;
            a.out_ids[o] = pad ? SQG_NO_ID : imin;
            a.out_dists[o] = pad ? __uint_as_float(0x7F800000u) : __uint_as_float(dmin);
        }
        // the list that held the head advances (global ids are distinct
        // across shards, so exactly one lane matches unless all are padding)
        if (db == dmin && gid == imin && imin != 0xFFFFFFFFu) {
            ++pos;
            head(a, lane, qi, pos, db, gid);
        }
    }
}

}  // namespace

extern "C" int sqg_merge_topk(const uint32_t *ids, const float *dists, int shards, int nq, int k,
                              const uint32_t *offsets, uint32_t *out_ids, float *out_dists, sqg_stream_t stream) {
    if (shards < 1 || shards > SQG_MAX_SHARDS || nq < 0 || k < 1 || k > SQG_MAX_K) return SQG_ERR_INVALID_ARG;
    if (nq == 0) return SQG_OK;
    if (!ids || !dists || !offsets || !out_ids || !out_dists) return SQG_ERR_INVALID_ARG;
    MergeArgs a;
    a.ids = ids;
    a.dists = dists;
    a.S = shards;
    a.nq = nq;
    a.k = k;
    for (int s = 0; s < SQG_MAX_SHARDS; ++s) a.offsets[s] = s < shards ? offsets[s] : 0u;
    a.out_ids = out_ids;
    a.out_dists = out_dists;
    const int blocks = (nq + kMergeWarps - 1) / kMergeWarps;
    merge_topk_kernel<<<blocks, kMergeWarps * 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? SQG_OK : SQG_ERR_CUDA;
}
