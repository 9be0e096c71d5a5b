/*
 * sqg.h -- C ABI of the GB300 SymphonyQG query-phase library (libsqg.so).
 *
 * SymphonyQG (arXiv 2411.12229) answers an approximate k-nearest-neighbour
 * query by a beam search over a graph in which every vertex owns one
 * contiguous block: its raw fp32 vector, the RaBitQ 1-bit codes and
 * correction factors of its out-neighbours (normalized about the vertex
 * itself), and the neighbour ids (Sec. 3.1.3, "dedicated data layout").
 * Expanding a vertex reads that block once: its exact distance updates the
 * result set (implicit re-ranking, Sec. 3.1.2) and the neighbours' distances
 * are estimated in one batch (Sec. 3.1.1, Eq. (5)-(6)); every unvisited
 * neighbour enters the beam with its estimate, even when already there
 * (multiple estimated distances, Sec. 3.1.2); Algorithm 1 gives the loop.
 *
 * Conventions for every entry point:
 *   - Return 0 (SQG_OK) or a negative SQG_ERR_* code; nothing is thrown and
 *     nothing is printed.  sqg_error_string() names a code.
 *   - Pointers are DEVICE pointers unless the comment says host.  The caller
 *     owns every buffer it passes; the library owns the index's device copy.
 *   - Work is enqueued on the caller's stream and returns before it runs,
 *     unless the comment says the call synchronizes.
 *   - Floats are IEEE fp32; ids are uint32; SQG_NO_ID marks padding.
 *   - Queries must be finite; d is the index's dimension.
 *   - An index is read-only after loading: searches on different streams
 *     may run concurrently.
 */
#ifndef SQG_H
#define SQG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sqg_stream_t; /* a cudaStream_t; NULL = legacy default stream */

/* ---- error codes (return values) ---- */
#define SQG_OK 0
#define SQG_ERR_INVALID_ARG (-1) /* null pointer, nq < 0, k < 1, ef < k, k > SQG_MAX_K, ... */
#define SQG_ERR_IO (-2)          /* index file cannot be opened or read / written */
#define SQG_ERR_FORMAT (-3)      /* bad magic, version, sizes or hash in the index file */
#define SQG_ERR_OOM (-4)         /* host or device allocation failed */
#define SQG_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define SQG_ERR_TIMEOUT (-6)     /* a bounded device wait expired (see SQG_STATUS_TIMEOUT) */
#define SQG_ERR_CAPACITY (-7)    /* workspace or shared memory too small for the request */
#define SQG_ERR_UNSUPPORTED (-8) /* shape the kernels are not built for (see sqg_index_load) */

/* ---- per-query status bits (sqg_query_stats.status, device status word) ---- */
#define SQG_STATUS_CAPACITY 1u     /* the hop cap ended the search (results still valid) */
#define SQG_STATUS_LEARNED_STOP 2u /* the learned early stop ended the search */
#define SQG_STATUS_BAD_PARAM 4u    /* this query's k or ef was invalid: output is padding */
#define SQG_STATUS_TIMEOUT 8u      /* a bounded wait on a block copy expired: output is padding */

#define SQG_MAX_K 256
#define SQG_MAX_EF 2048
#define SQG_MAX_SHARDS 32 /* shards one sqg_merge_topk call merges */
#define SQG_NO_ID 0xFFFFFFFFu

/* Learned early stop: a 16 -> 64 -> 64 -> 1 fp32 MLP (ReLU hidden units)
 * over 16 search-state features; parameters flat in the order
 * W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3. Not in the paper. */
#define SQG_MLP_IN 16
#define SQG_MLP_HIDDEN 64
#define SQG_MLP_NPARAM 5313

typedef struct sqg_index sqg_index; /* opaque; owns the device-resident blocks */

typedef struct {
    uint64_t n;            /* vertices */
    uint32_t d;            /* dimension (a multiple of 32) */
    uint32_t degree;       /* out-degree R of every vertex (a multiple of 32) */
    uint32_t block_bytes;  /* bytes per vertex block, a multiple of 128 */
    uint32_t entry;        /* entry point of Algorithm 1 */
    uint32_t off_codes, off_factors, off_ids; /* byte offsets inside a block */
    int32_t device;        /* CUDA device holding the index */
    uint64_t device_bytes; /* device memory held by the index */
    uint32_t metric;       /* 0 squared Euclidean; 1 cosine (see sqg_index_load) */
    uint32_t version;      /* file format version: 1 dense rotation, 2 fast JLT */
} sqg_info;

typedef struct {
    float eps0;              /* admission key = estimate - eps0 * bound; 0 = Algorithm 1 */
    int32_t multi_estimate;  /* 1: every unvisited neighbour enters the beam (Sec. 3.1.2);
                                0: ablation "w/o ME", the first estimate only (Sec. 5.4) */
    int32_t hop_cap;         /* expansions per query; 0 = 4*ef + 64 */
    int32_t max_k, max_ef;   /* bounds of the batch's k[] and ef[]; 0 = read them from the
                                device (sqg_search then synchronizes the stream once) */
    const float *stop_mlp;   /* device, SQG_MLP_NPARAM floats, or NULL: learned stop off */
    float stop_logit;        /* stop when the MLP's logit exceeds this */
    int32_t stop_every;      /* evaluate the stop every this many expansions (>= 1) */
    int32_t team;            /* lanes per query: 32 (default, 0), 16 or 8 -- a warp then
                                runs 2 or 4 queries side by side; 16 and 8 need d <= 256
                                and no stop_mlp / trace (else SQG_ERR_UNSUPPORTED) */
    int32_t warps_per_block; /* 1, 2 or 4; 0 = the one with the most resident warps per SM */
    void *timing_events[2];  /* optional cudaEvent_t pair recorded on the stream right before
                                and right after the search kernel; NULL = none */
    int32_t visited_smem_log2; /* log2 of the visited set's shared-memory slots (5..12;
                                  0 = 9); a search past half of them continues in a
                                  full-size table in the workspace */
    int32_t prefetch;        /* 1 (default, 0): the next block is copied into shared
                                memory during the merge; 2: also L2-prefetch the
                                runner-up candidate's block */
    int32_t lean;            /* d <= 256 only.  General kernel: 0 or 1 = the build capped at
                                64 registers (more resident warps, a few spills; the
                                default), 2 = the 96-register build (and never the
                                compact kernel).  Compact kernel: 0 = the build for 8
                                resident blocks of 4 warps per SM (64 registers) up to
                                ef 64 and for 7 (72) up to ef 128 with k <= 32; 1 = one
                                block more (56 / 64 registers); ignored past ef 128 or
                                k 32 */
    int32_t rotation;        /* q' = P^-1 q: 1 = the canonical fp32 order (see
                                sqg_prepare_queries) on the CUDA cores; 2 = tcgen05 tensor
                                cores (3xTF32) followed by an exact pass that recomputes in
                                the canonical order every coordinate whose 4-bit code or
                                min/max role the tensor-core error could change, so the
                                quantized query is identical to 1; 0 = 2 for d >= 512,
                                else 1.  Ignored for a fast-JLT index (format version 2),
                                whose queries always take the fast transform */
    int32_t kernel;          /* 0 (default) = the compact search kernel wherever it applies
                                (one warp per query, d <= 1024, degree 32 or 64, every k[i] <= 32
                                and ef[i] <= 128 by max_k / max_ef -- for d <= 256 k[i] <= 128
                                and ef[i] <= 256 --, multiple estimates, no trace, prefetch 1;
                                with or without the learned stop), else the general one;
                                1 = always the general kernel; 2 = the compact kernel or
                                SQG_ERR_UNSUPPORTED.  Both return identical results. */
    int32_t uniform_k;       /* 0 (default): k[] may differ per query, outputs ragged at the
                                exclusive prefix sum of k[] (a planning kernel computes it);
                                > 0: every k[i] is this value, query i's outputs start at
                                i * uniform_k and no planning kernel runs; a query whose k[i]
                                differs gets padding and SQG_STATUS_BAD_PARAM */
} sqg_search_params;

typedef struct {
    uint32_t hops;   /* vertices expanded */
    uint32_t status; /* SQG_STATUS_* bits */
} sqg_query_stats;

/* Self-test of the bounded device waits (failure detection without a GPU
 * fault): one thread waits, through the search kernel's bounded wait, on an
 * mbarrier phase that nothing completes; the wait gives up after its 1 s
 * limit.  Writes (HOST) *status = SQG_STATUS_TIMEOUT (0 had the wait
 * completed) and *waited_ns = how long it waited.  Synchronous; the
 * context stays usable. */
int sqg_wait_selftest(int device, uint32_t *status, uint64_t *waited_ns);

/* Name of an error code (static string). */
const char *sqg_error_string(int code);

/* Load an index file (format below) from the HOST path `path` onto CUDA
 * device `device` and return a handle in *out.  Validates magic, version,
 * sizes and both FNV-1a hashes; SQG_ERR_FORMAT on any mismatch, SQG_ERR_IO
 * if unreadable, SQG_ERR_UNSUPPORTED if d or degree is outside the built
 * kernels (d in {32,...,2048} multiple of 32, degree in {32, 64}).
 * Synchronous.  Layout of the file and of each vertex block: Sec. 3.1.3
 * (raw vector, then the FastScan data, then the neighbour ids); space
 * n(32D + 32R + DR) bits plus factors (Sec. 3.3).
 *
 * File v1, little-endian: 256-byte header
 *   0 "SQG1" | 4 version u32 (1: dense rotation; 2: the fast JLT, see
 *   sqg_write_index2) | 8 n u64 | 16 d u32 | 20 R u32 |
 *   24 block_bytes u32 | 28 entry u32 | 32 metric u32 (see below) |
 *   36 off_codes | 40 off_factors | 44 off_ids (u32) | 48 rot_offset u64 |
 *   56 blocks_offset u64 | 64 file_bytes u64 | 72 seed_rotation u64 |
 *   80 seed_graph u64 | 88 payload_hash u64 | 96 header_hash u64
 * header_hash = FNV-1a-64 over u64 words of bytes [0,96); payload_hash over
 * u64 words of [rot_offset, file_bytes).  At rot_offset: P^-1 as d*d fp32
 * row-major.  At blocks_offset: n blocks; block of vertex v:
 *   raw[d] fp32 | codes: u32 word w of neighbour j at index w*R + j, bit
 *   (i mod 32) of word i/32 = code bit of dimension i | f_add[R],
 *   f_rescale[R], f_err[R] fp32, popcount[R] u32 | ids[R] u32 | zero pad
 *   to a multiple of 128 bytes.  A neighbour id is < n, not the vertex
 *   itself and distinct within the block, or SQG_NO_ID: an empty slot of a
 *   degree-unaligned graph (zero code bits and factors), which the search
 *   skips.
 * Metric (Sec. 3: the method serves Euclidean distance and cosine
 * similarity): 0 = squared Euclidean; 1 = cosine, served as Euclidean
 * search between unit vectors -- the raw vectors are unit-norm (or zero),
 * and every search, sqg_prepare_queries(_tc) and sqg_estimate_block first
 * scales each query to unit norm: s = ||q||^2 as 32 partial fmaf sums over
 * float4 chunks l, l+32, ... then pairwise sums of partials l and l^16, ^8,
 * ^4, ^2, ^1, and q_i / fl(sqrt(s)) per coordinate (a query with s = 0 or s
 * not finite is used as it is).  Distances returned are then
 * ||q/||q|| - x||^2 = 2 - 2 cos(q, x). */
int sqg_index_load(const char *path, int device, sqg_index **out);

/* Free an index and its device memory (synchronizes the device). NULL is a no-op. */
void sqg_index_free(sqg_index *ix);

/* Shape of a loaded index into *out (host). */
int sqg_index_info(const sqg_index *ix, sqg_info *out);

/* Device workspace bytes sqg_search_ex needs for nq queries with the given
 * bounds (host call, no device work). */
size_t sqg_workspace_size(const sqg_index *ix, int nq, int max_k, int max_ef);

/* Search nq queries (Algorithm 1 per query, with multiple estimated
 * distances and implicit re-ranking, Sec. 3.1).
 *   queries  nq x d fp32 row-major, 16-byte aligned (else SQG_ERR_INVALID_ARG,
 *            nothing launched; every CUDA allocation is)
 *   k, ef    nq int32 each: results wanted and beam size n_b per query
 *            (1 <= k <= SQG_MAX_K, k <= ef <= SQG_MAX_EF)
 *   out_ids, out_dists: ragged, query i at offset sum_{j<i} k[j]; k[i]
 *            (id, exact squared distance) pairs sorted by (dist, id),
 *            padded with (SQG_NO_ID, +inf) when fewer vertices were reached.
 *            A query with invalid k or ef contributes max(0, min(k,
 *            SQG_MAX_K)) slots, all padding, and sets SQG_STATUS_BAD_PARAM.
 * Scratch is taken from the stream-ordered allocator on `stream`.  The
 * call synchronizes the stream once to read the batch's largest k and ef.
 * SQG_ERR_INVALID_ARG for null pointers or nq < 0 (nq = 0 is a no-op). */
int sqg_search(const sqg_index *ix, const float *queries, int nq, const int32_t *k, const int32_t *ef,
               uint32_t *out_ids, float *out_dists, sqg_stream_t stream);

/* sqg_search with explicit parameters (NULL = defaults), a caller-owned
 * workspace (NULL = stream-ordered allocation; else 256-byte aligned) of ws_bytes >=
 * sqg_workspace_size(), and optional per-query stats (nq entries, device).
 * With params->max_k and max_ef given and a workspace, the call is
 * asynchronous and allocates nothing.  With params->uniform_k > 0 the
 * outputs are nq rows of uniform_k slots (the caller sizes them nq *
 * uniform_k), max_k must be 0 or uniform_k (else SQG_ERR_INVALID_ARG), and
 * no planning kernel runs.  SQG_ERR_CAPACITY when the workspace
 * is too small or the bounds need more shared memory than a block has. */
int sqg_search_ex(const sqg_index *ix, const float *queries, int nq, const int32_t *k, const int32_t *ef,
                  uint32_t *out_ids, float *out_dists, const sqg_search_params *params, void *workspace,
                  size_t ws_bytes, sqg_query_stats *stats, sqg_stream_t stream);

/* Device workspace bytes sqg_search_ex needs for nq queries with the given
 * bounds and these parameters (NULL = defaults; their max_k/max_ef fields are
 * ignored).  The tuning fields (warps_per_block, visited_smem_log2, lean) set
 * how many warps run at once and so how much room the spilled visited sets
 * take; 0 on invalid arguments.  Host call, no device work. */
size_t sqg_workspace_size_ex(const sqg_index *ix, int nq, int max_k, int max_ef, const sqg_search_params *params);

/* Query preparation alone (the first kernels of sqg_search), for tests:
 *   out_qrot   nq x d fp32: q' = P^-1 q (Eq. (4)) in the canonical order:
 *              per 32-column chunk c an fmaf chain over j = 32c..32c+31 from
 *              0, the chunk sums added in order c = 0, 1, ... to a total from 0
 *   out_planes nq x 4 x d/32 u32: bit (i mod 32) of word [b][i/32] = bit b
 *              of the 4-bit code qbar_i
 *   out_scal   nq x 4: (v_l, delta, Sq as float, 1/sqrt(d)) with
 *              delta = (v_r - v_l)/15 and qbar_i = min(15,
 *              trunc((q'_i - v_l) * 15/(v_r - v_l) + 0.5))
 * queries and the three outputs 16-byte aligned, else SQG_ERR_INVALID_ARG. */
int sqg_prepare_queries(const sqg_index *ix, const float *queries, int nq, float *out_qrot,
                        uint32_t *out_planes, float *out_scal, sqg_stream_t stream);

/* Query preparation through the tensor-core path (rotation = 2), for tests:
 *   out_qrot   nq x d fp32: q' from tcgen05.mma kind::tf32 with the 3xTF32
 *              split (differs from the canonical order by at most c(d) ||q||)
 *   out_planes nq x 4 x d/32 u32 and out_scal nq x 4 as sqg_prepare_queries
 *              gives them -- identical by construction
 *   recomputed (1 u32, device, added to): coordinates the exact pass redid */
int sqg_prepare_queries_tc(const sqg_index *ix, const float *queries, int nq, float *out_qrot, uint32_t *out_planes,
                           float *out_scal, uint32_t *recomputed, sqg_stream_t stream);

/* Estimates for all R neighbours of one vertex per query, for tests
 * (Sec. 3.1.1): for query i and vertex v[i] writes, at [i*R + j],
 *   S      = sum_d b_d qbar_d (int32, exact)
 *   est    = f_add + dist_c + f_rescale * ip,
 *            ip = fmaf(delta, 2S - Sq, v_l (2 popcount - d)) / sqrt(d)
 *   key    = est - eps0 * f_err * sqrt(dist_c)
 * and dist_c[i] = exact squared distance of query i to v[i]; queries
 * 16-byte aligned. */
int sqg_estimate_block(const sqg_index *ix, const float *queries, int nq, const uint32_t *v, float eps0,
                       int32_t *out_S, float *out_est, float *out_key, float *out_dist_c, sqg_stream_t stream);

/* sqg_search_ex that also records what the search did.
 * Learned-stop training data (not in the paper; trace_feat may be NULL): at
 * every stop_every-th expansion once the result holds k entries, query i
 * appends the 16 search-state features (fp32) to
 * trace_feat[(i*trace_cap + t)*16 ...] and, when gt is given (nq x gt_k
 * ground-truth ids, gt_k >= every k[i]), the number of the first k[i] gt ids
 * present in its current result to trace_hit[i*trace_cap + t]; trace_n[i]
 * receives the number of rows written (at most trace_cap).
 * Expansion order (path may be NULL): path[i*path_cap + h] = id of the h-th
 * vertex query i expanded (Algorithm 1, line 3), for h < min(hops,
 * path_cap); the rest is left untouched.  Used by the index builder
 * (search-path candidates) and by parity tests.  At least one of trace_feat
 * and path must be given.  Scratch comes from the stream-ordered allocator. */
int sqg_search_trace(const sqg_index *ix, const float *queries, int nq, const int32_t *k, const int32_t *ef,
                     uint32_t *out_ids, float *out_dists, const sqg_search_params *params, sqg_query_stats *stats,
                     const uint32_t *gt, int gt_k, float *trace_feat, int32_t *trace_hit, int32_t *trace_n,
                     int trace_cap, uint32_t *path, int path_cap, sqg_stream_t stream);

/* sqg_search for callers that cannot allocate device memory while they
 * search -- e.g. an application that reserved all GPU memory for its own
 * pool at start-up, or a latency-critical thread that must not enter the
 * allocator or meet an out-of-memory error mid-request.  The paper has no
 * counterpart: this is a packaging of the same search.
 *   Same arguments as sqg_search, with the batch's bounds given explicitly
 *   (max_k, max_ef: every valid k[i] <= max_k, ef[i] <= max_ef), so nothing
 *   is read back from the device either.
 *   Scratch: one file-scope device array of sqg_noalloc_scratch_bytes()
 *   (32 MiB) that a GPU holds until the process exits once the entry point
 *   has run on it.  A batch whose sqg_workspace_size(ix, nq, max_k, max_ef)
 *   exceeds it is rejected with SQG_ERR_CAPACITY (for d = 128: about 60,000
 *   queries with max_ef <= 112; larger ef also needs the visited tables).
 *   The call performs no cudaMalloc, cudaFree or stream-ordered allocation.
 *   Set-up: the first call on a device loads the array's module there,
 *   which commits the 32 MiB, and looks the array's address up
 *   (cudaGetSymbolAddress) and caches it.  Make that first call -- a call
 *   with nq = 0 does only the set-up -- before reserving the rest of the
 *   GPU's memory and before any stream capture.  The cached address is not
 *   valid after a cudaDeviceReset of that device.  All calls share the
 *   array and it keeps the last call's contents (the search resets what
 *   must start at zero); calls whose work overlaps on one GPU race on it
 *   and must be serialized by the caller. */
int sqg_search_noalloc(const sqg_index *ix, const float *queries, int nq, const int32_t *k, const int32_t *ef,
                       int max_k, int max_ef, uint32_t *out_ids, float *out_dists, sqg_stream_t stream);

/* Size in bytes of the fixed scratch array used by sqg_search_noalloc. */
size_t sqg_noalloc_scratch_bytes(void);

/* ---- sharded search (an index split over several graphs) ---- */

/* Merge per-shard results into one top-k per query.  An index too large
 * for one GPU is split into `shards` shards, each with its own graph
 * (Algorithm 2, Sec. 3.2, on the shard's vectors alone); every query is
 * searched in every shard (Algorithm 1, Sec. 3.1.3, whose output is the k
 * nearest expanded vertices sorted by (distance, id)), and this call merges
 * the shards' lists by (distance, global id).  The paper has no sharded
 * form; its scalability study (Sec. 5) keeps one graph per index.
 *   ids, dists: DEVICE, [shards][nq][k] -- shard s's result list of query i
 *   at ((s * nq) + i) * k, local ids (SQG_NO_ID = padding, distance +inf),
 *   each list sorted by (distance, id).
 *   offsets: HOST, shards values; global id = local id + offsets[s] (the
 *   shards' id ranges must not overlap).
 *   out_ids, out_dists: DEVICE, [nq][k], the k smallest (distance, global
 *   id) of the shards' lists, padded with (SQG_NO_ID, +inf).
 * 1 <= shards <= SQG_MAX_SHARDS, 1 <= k <= SQG_MAX_K; stream-ordered on
 * `stream`, no allocation. */
int sqg_merge_topk(const uint32_t *ids, const float *dists, int shards, int nq, int k, const uint32_t *offsets,
                   uint32_t *out_ids, float *out_dists, sqg_stream_t stream);

/* ---- learned early stop: training kernels (not in the paper) ---- */

/* Gradient of the weighted binary cross-entropy of the stop MLP:
 *   loss = sum_b w_b [softplus(z_b) - y_b z_b] / sum_b w_b,
 *   z_b = MLP(x_b) (16 -> 64 -> 64 -> 1, ReLU; parameter order as above).
 * params SQG_MLP_NPARAM; x n x 16; y, w n floats (labels 0/1, weights > 0);
 * grad (out) SQG_MLP_NPARAM; loss (out, optional) 1 float; scratch: 4
 * bytes of caller memory for sum(w).  Overwrites grad and loss. */
int sqg_mlp_grad(const float *params, const float *x, const float *y, const float *w, int n, float *grad,
                 float *loss, float *scratch, sqg_stream_t stream);

/* One Adam step (Kingma & Ba) on all SQG_MLP_NPARAM parameters, in place:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr (m/(1-b1^step)) / (sqrt(v/(1-b2^step)) + eps).  step >= 1. */
int sqg_mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr, float beta1,
                 float beta2, float eps, sqg_stream_t stream);

/* Logits of the stop MLP for n feature rows (x n x 16 -> logits n). */
int sqg_mlp_forward(const float *params, const float *x, int n, float *logits, sqg_stream_t stream);

/* OR of the status bits every search on this index has raised since the
 * last call, then cleared.  Synchronizes `stream`. */
int sqg_get_status(const sqg_index *ix, sqg_stream_t stream, uint32_t *status);

/* ---- host-side index construction (Algorithm 2, Sec. 3.2) ---- */

/* Exact k nearest neighbours of every base vector among the base vectors
 * (itself excluded), multithreaded on the host, fp32.  data n x d (host),
 * out n x k (host) sorted by (dist, id).  For small n only (O(n^2 d)). */
int sqg_knn_host(const float *data, uint64_t n, uint32_t d, uint32_t k, uint32_t *out, int threads);

/* Build one graph of Algorithm 2 from candidate lists (host):
 *   data n x d fp32; cand n x L uint32 candidates per vertex (any order,
 *   SQG_NO_ID = none; the vertex itself and repeats are ignored);
 *   out_adj n x R: for each vertex, NSG's pruning rule keeps at most R
 *   candidates (Sec. 3.2.1), reverse edges are offered to their targets and
 *   re-pruned, and the adaptive angle rule supplements pruned candidates
 *   until exactly R edges remain (Sec. 3.2.2); random vertices fill any
 *   remaining gap (Sec. 3.2.2, footnote).  Every vertex is then made
 *   reachable from `entry` by replacing the edge of a reachable vertex
 *   whose target has the most in-edges.  Distances are the search's exact
 *   distance in its canonical fp32 order, candidates ordered by (distance,
 *   id).  out_stats (host, 4): [avg degree after NSG pruning x 1000,
 *   vertices needing supplement, vertices randomly filled, repairs]. */
int sqg_build_graph(const float *data, uint64_t n, uint32_t d, const uint32_t *cand, uint32_t L, uint32_t R,
                    uint32_t entry, uint64_t seed, uint32_t *out_adj, uint64_t *out_stats, int threads);

/* Flag of sqg_build_graph_ex: the degree-unaligned graph of the "w/o GR"
 * ablation (Sec. 5): NSG pruning and reverse edges only, no angle-rule
 * supplement and no random fill; a row's unused slots are SQG_NO_ID. */
#define SQG_GRAPH_IRREGULAR 1u

/* sqg_build_graph with flags (0 or SQG_GRAPH_IRREGULAR) and a device.
 * device < 0: on the host threads.  device >= 0: steps (1)-(3) run on that
 * CUDA device, one warp per vertex pruning its own candidates, then
 * re-pruning them with its reverse candidates and (regular graphs)
 * supplementing by the angle rule (Sec. 3.2.1-3.2.2), with the same
 * distance order and the same (distance, id) order as the host, so the rows
 * are the host's bit for bit; the reverse lists, a vertex whose lists
 * exceed a warp's 512-entry lists, the random fill and the reachability
 * repair run on the host.  data and cand are HOST arrays (copied to the
 * device; synchronous); every value of data must be finite; on a device
 * L <= 512 and min(R, n-1) <= 64, else SQG_ERR_UNSUPPORTED.  out_stats (5
 * u64, optional): as sqg_build_graph's four, then the vertices refined on
 * the host. */
int sqg_build_graph_ex(const float *data, uint64_t n, uint32_t d, const uint32_t *cand, uint32_t L, uint32_t R,
                       uint32_t entry, uint64_t seed, uint32_t flags, uint32_t *out_adj, uint64_t *out_stats,
                       int threads, int device);

/* Vertex nearest to the mean of the data (host), the entry point used by
 * the builder. */
uint32_t sqg_medoid(const float *data, uint64_t n, uint32_t d, int threads);

/* Quantize every edge and write an index file (host; "prepare data for
 * FastScan", Algorithm 2):  rot = P^-1 (d x d fp32, row-major, orthogonal);
 * for the edge c -> o, v = P^-1 (o - c)/||o - c||, code bit b_i = [v_i >= 0],
 * alpha = sum|v_i|/sqrt(d), xc = <x_bar, P^-1 c>,
 * f_add = ||o-c||^2 + 2||o-c|| xc/alpha, f_rescale = -2||o-c||/alpha,
 * f_err = 2||o-c|| sqrt((1-alpha^2)/alpha^2)/sqrt(d-1); o = c gives zero
 * bits and factors; adj entries SQG_NO_ID are empty slots (zero bits and
 * factors).  Writes `path` (host) in the format of sqg_index_load. */
int sqg_write_index(const char *path, const float *data, uint64_t n, uint32_t d, const uint32_t *adj,
                    uint32_t R, const float *rot, uint32_t entry, uint64_t seed_rotation, uint64_t seed_graph,
                    int threads);

/* sqg_write_index with the rotation's kind and the metric.  rotation_kind
 * 0 = the dense P^-1 (version 1);
 * 1 = the fast JLT of Sec. 3.1.4 (version 2, d a power of 2): three rounds
 * of a sign flip s_r and the Walsh-Hadamard transform scaled by 1/sqrt(d),
 * s_r[i] = -1 when bit 63 of splitmix64(seed_rotation ^ (r << 32 | i)) is
 * set.  `rot` must then hold that transform as a dense matrix (the edges'
 * codes are built with it); queries are rotated by the fast transform.
 * metric 0 = squared Euclidean; 1 = cosine: every vector of `data` must have
 * ||x||^2 within 1e-4 of 1 (or be zero), else SQG_ERR_INVALID_ARG. */
int sqg_write_index2(const char *path, const float *data, uint64_t n, uint32_t d, const uint32_t *adj,
                     uint32_t R, const float *rot, uint32_t entry, uint64_t seed_rotation, uint64_t seed_graph,
                     int threads, uint32_t rotation_kind, uint32_t metric);

#ifdef __cplusplus
}
#endif
#endif /* SQG_H */
