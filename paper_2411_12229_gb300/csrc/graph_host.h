// graph_host.h -- the host half of Algorithm 2's adjust step (Sec. 3.2),
// shared by the host builder (builder.cpp) and the GPU one (graph.cu), so
// that a vertex refined on either side gets the same list.
//
// Steps, per vertex u (readings R11):
//   (1) NSG-prune u's own candidates to at most R' = min(R, n-1) edges;
//   (2) offer every kept edge u -> v to v as a reverse candidate and
//       NSG-prune v's kept edges plus its reverse candidates again;
//   (3) supplement a list still short of R' by the adaptive angle rule;
//   (4) fill a list that is still short with random vertices;
//   (5) connect every vertex the entry point cannot reach.
// A degree-unaligned graph (the "w/o GR" ablation of Sec. 5) stops after
// step (2): a row keeps its re-pruned edges and marks the rest of its R
// slots SQG_NO_ID.
// Distances are the search's exact distance in its canonical fp32 order;
// candidates are ordered by (distance, id).
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/sqg.h"

namespace sqg_graph {

inline int resolve_threads(int t) {
    if (t > 0) return t;
    unsigned h = std::thread::hardware_concurrency();
    return h ? (int)h : 1;
}

template <class F>
void parallel_for(uint64_t n, int threads, F f, uint64_t chunk = 64) {
    threads = resolve_threads(threads);
    std::atomic<uint64_t> next{0};
    auto work = [&]() {
        for (;;) {
            uint64_t a = next.fetch_add(chunk);
            if (a >= n) break;
            uint64_t b = std::min(n, a + chunk);
            for (uint64_t i = a; i < b; ++i) f(i);
        }
    };
    std::vector<std::thread> ts;
    for (int t = 1; t < threads; ++t) ts.emplace_back(work);
    work();
    for (auto &t : ts) t.join();
}

// Squared L2 distance in the search's exact-distance order: 32 partial
// sums, partial l over the float4 chunks l, l+32, ... with fma(x, x, acc)
// on their four coordinates in order, then pairwise sums of partials l and
// l+16, l and l+8, ..., l and l+1.  Symmetric in a and b.
inline float l2c(const float *a, const float *b, uint32_t d) {
    float p[32];
    const uint32_t nch = d / 4;
    for (uint32_t l = 0; l < 32; ++l) {
        float acc = 0.0f;
        for (uint32_t c = l; c < nch; c += 32)
            for (uint32_t t = 0; t < 4; ++t) {
                const float x = a[4 * c + t] - b[4 * c + t];
                acc = std::fma(x, x, acc);
            }
        p[l] = acc;
    }
    for (uint32_t o = 16; o >= 1; o >>= 1)
        for (uint32_t l = 0; l < o; ++l) p[l] = p[l] + p[l + o];
    return p[0];
}

struct Cand {
    float d;
    uint32_t id;
    bool operator<(const Cand &o) const { return d < o.d || (d == o.d && id < o.id); }
};

inline void unique_ids(std::vector<Cand> &c) {  // one of each id (their distances are equal)
    std::sort(c.begin(), c.end(), [](const Cand &a, const Cand &b) { return a.id < b.id; });
    c.erase(std::unique(c.begin(), c.end(), [](const Cand &a, const Cand &b) { return a.id == b.id; }), c.end());
}

inline uint64_t splitmix64_next(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// NSG's pruning rule (Sec. 3.2.1, after NSG): walk the candidates nearest
// first and keep c unless a kept w is closer to c than the vertex is
// (d(w,c) < d(u,c)), which keeps every pair of out-edges at least 60
// degrees apart.
inline void nsg_prune(const float *data, uint32_t d, const std::vector<Cand> &cands, uint32_t R,
                      std::vector<Cand> &kept) {
    kept.clear();
    for (const Cand &c : cands) {
        if (kept.size() >= R) break;
        const float *xc = data + (uint64_t)c.id * d;
        bool ok = true;
        for (const Cand &w : kept)
            if (l2c(data + (uint64_t)w.id * d, xc, d) < c.d) { ok = false; break; }
        if (ok) kept.push_back(c);
    }
}

// Adaptive angle rule (Sec. 3.2.2): a pruned candidate c is dropped at
// threshold theta if a candidate closer to u makes an angle < theta with it.
// The count of survivors falls monotonically as theta grows; the largest
// theta that still leaves `need` survivors is the need-th smallest of the
// candidates' largest cosines to a closer candidate, which is what a binary
// search over theta converges to.  Returns the chosen candidates.
inline void angle_supplement(const float *data, uint32_t d, const std::vector<Cand> &kept,
                             const std::vector<Cand> &extra, uint32_t need, std::vector<Cand> &out) {
    out.clear();
    if (need == 0 || extra.empty()) return;
    std::vector<Cand> all(kept);
    all.insert(all.end(), extra.begin(), extra.end());
    std::sort(all.begin(), all.end());
    std::vector<std::pair<float, Cand>> score;  // (max cosine to a closer candidate, c)
    score.reserve(extra.size());
    for (const Cand &c : extra) {
        const float *xc = data + (uint64_t)c.id * d;
        float best = -2.0f;
        for (const Cand &w : all) {
            if (!(w < c)) break;
            float dwc = l2c(data + (uint64_t)w.id * d, xc, d);
            float den = 2.0f * std::sqrt(w.d) * std::sqrt(c.d);
            float cs = den > 0.0f ? (w.d + c.d - dwc) / den : 1.0f;
            best = std::max(best, cs);
        }
        score.push_back({best, c});
    }
    std::vector<float> cs;
    for (auto &s : score) cs.push_back(s.first);
    uint32_t take = std::min<uint32_t>(need, (uint32_t)cs.size());
    std::nth_element(cs.begin(), cs.begin() + (take - 1), cs.end());
    float thr = cs[take - 1];
    for (auto &s : score)
        if (s.first <= thr) out.push_back(s.second);
    std::sort(out.begin(), out.end());
    if (out.size() > take) out.resize(take);
}

// u's own candidates: valid ids from its list (not u, each once) with their
// distances, sorted by (distance, id).
inline void own_cands(const float *data, uint64_t n, uint32_t d, const uint32_t *cand, uint32_t L, uint64_t u,
                      std::vector<Cand> &c) {
    c.clear();
    const float *xu = data + u * d;
    for (uint32_t t = 0; t < L; ++t) {
        uint32_t v = cand[u * L + t];
        if (v == SQG_NO_ID || v >= n || v == u) continue;
        c.push_back({l2c(xu, data + (uint64_t)v * d, d), v});
    }
    unique_ids(c);
    std::sort(c.begin(), c.end());
}

// (2) the reverse candidates: every kept edge u -> v, as (d, u) at v, in a
// CSR (rev[off[v] .. off[v+1])).  k1: n lists of stride `stride`, counts n1.
inline void reverse_edges(uint64_t n, const Cand *k1, const uint32_t *n1, uint32_t stride, std::vector<uint64_t> &off,
                          std::vector<Cand> &rev) {
    off.assign(n + 1, 0);
    for (uint64_t u = 0; u < n; ++u)
        for (uint32_t j = 0; j < n1[u]; ++j) off[k1[u * stride + j].id + 1]++;
    for (uint64_t v = 0; v < n; ++v) off[v + 1] += off[v];
    rev.resize(off[n]);
    std::vector<uint64_t> fill(off.begin(), off.end() - 1);
    for (uint64_t u = 0; u < n; ++u)
        for (uint32_t j = 0; j < n1[u]; ++j) {
            const Cand &c = k1[u * stride + j];
            rev[fill[c.id]++] = {c.d, (uint32_t)u};
        }
}

// (2)-(3) for vertex u: re-prune its kept edges with its reverse candidates,
// then (regular graphs) supplement by the angle rule from its own and
// reverse candidates not kept, the nearest 2R' (d >= 512) or 3R' of them.
// Returns whether the angle rule ran.
inline bool refine_vertex(const float *data, uint64_t n, uint32_t d, const uint32_t *cand, uint32_t L, uint32_t Rr,
                          uint64_t u, const Cand *k1u, uint32_t n1u, const Cand *rev, uint64_t nrev, bool regular,
                          std::vector<Cand> &k2) {
    std::vector<Cand> pool(k1u, k1u + n1u);
    pool.insert(pool.end(), rev, rev + nrev);
    unique_ids(pool);
    std::sort(pool.begin(), pool.end());
    nsg_prune(data, d, pool, Rr, k2);
    if (!regular || k2.size() >= Rr) return false;
    std::vector<Cand> all;
    own_cands(data, n, d, cand, L, u, all);
    all.insert(all.end(), rev, rev + nrev);
    unique_ids(all);
    std::vector<uint32_t> have;
    for (auto &c : k2) have.push_back(c.id);
    std::sort(have.begin(), have.end());
    std::vector<Cand> extra;
    for (auto &c : all)
        if (!std::binary_search(have.begin(), have.end(), c.id)) extra.push_back(c);
    std::sort(extra.begin(), extra.end());
    const uint32_t cap = d >= 512 ? 2 * Rr : 3 * Rr;
    if (extra.size() > cap) extra.resize(cap);
    std::vector<Cand> sup;
    angle_supplement(data, d, k2, extra, Rr - (uint32_t)k2.size(), sup);
    k2.insert(k2.end(), sup.begin(), sup.end());
    std::sort(k2.begin(), k2.end());
    return true;
}

// (4) a list still short of R' gets random distinct vertices (footnote of
// Sec. 3.2.2); then the n x R rows (tiny graphs with R' < R repeat entries).
// A degree-unaligned row instead ends in SQG_NO_ID slots.  Returns whether
// vertex u needed the fill.
inline bool fill_and_write(const float *data, uint64_t n, uint32_t d, uint32_t R, uint32_t Rr, uint64_t seed, uint64_t u,
                           bool regular, std::vector<Cand> &k2, uint32_t *out_adj) {
    if (!regular) {
        for (uint32_t t = 0; t < R; ++t) out_adj[u * R + t] = t < k2.size() ? k2[t].id : SQG_NO_ID;
        return false;
    }
    bool filled = false;
    if (k2.size() < Rr) {
        filled = true;
        const float *xu = data + u * d;
        uint64_t st = seed ^ (u * 0x9E3779B97F4A7C15ull);
        std::vector<uint32_t> have;
        for (auto &c : k2) have.push_back(c.id);
        while (k2.size() < Rr) {
            uint32_t v = (uint32_t)(splitmix64_next(st) % n);
            if (v == u || std::find(have.begin(), have.end(), v) != have.end()) continue;
            have.push_back(v);
            k2.push_back({l2c(xu, data + (uint64_t)v * d, d), v});
        }
        std::sort(k2.begin(), k2.end());
    }
    for (uint32_t t = 0; t < R; ++t) out_adj[u * R + t] = t < k2.size() ? k2[t].id : k2[t % k2.size()].id;
    return filled;
}

// (5) reachability from the entry point: connect each unreachable vertex
// from a nearby reachable vertex, replacing that vertex's edge whose target
// has the most other in-edges.  Returns the number of edges replaced.
inline uint64_t repair_reachability(uint64_t n, const uint32_t *cand, uint32_t L, uint32_t R, uint32_t entry,
                                    uint32_t *out_adj) {
    std::vector<uint32_t> in(n, 0);
    for (uint64_t i = 0; i < n * R; ++i)
        if (out_adj[i] != SQG_NO_ID) in[out_adj[i]]++;
    uint64_t repairs = 0;
    for (int round = 0; round < 16; ++round) {
        std::vector<uint8_t> seen(n, 0);
        std::vector<uint32_t> stack{entry};
        seen[entry] = 1;
        auto flood = [&]() {
            while (!stack.empty()) {
                uint32_t u = stack.back();
                stack.pop_back();
                for (uint32_t t = 0; t < R; ++t) {
                    uint32_t v = out_adj[(uint64_t)u * R + t];
                    if (v != SQG_NO_ID && !seen[v]) { seen[v] = 1; stack.push_back(v); }
                }
            }
        };
        flood();
        uint64_t fixed = 0;
        for (uint64_t v = 0; v < n; ++v) {
            if (seen[v]) continue;
            uint32_t r = entry;
            for (uint32_t t = 0; t < L; ++t) {
                uint32_t c = cand[v * L + t];
                if (c != SQG_NO_ID && c < n && c != v && seen[c]) { r = c; break; }
            }
            uint32_t *row = out_adj + (uint64_t)r * R;
            bool dup = false;
            for (uint32_t t = 0; t < R; ++t) dup |= row[t] == v;
            if (dup) continue;
            // an empty slot if the row has one, else replace the edge whose
            // target has the most in-edges (farthest on ties)
            int slot = -1;
            for (uint32_t t = 0; t < R && slot < 0; ++t)
                if (row[t] == SQG_NO_ID) slot = (int)t;
            if (slot < 0) {
                slot = (int)R - 1;
                for (int t = (int)R - 2; t >= 0; --t)
                    if (in[row[t]] > in[row[slot]]) slot = t;
                in[row[slot]]--;
            }
            row[slot] = (uint32_t)v;
            in[v]++;
            ++fixed;
            seen[v] = 1;
            stack.push_back((uint32_t)v);
            flood();
        }
        repairs += fixed;
        if (fixed == 0) break;
    }
    return repairs;
}

// Steps (1)-(5) on the host threads (builder.cpp); regular = false builds
// the degree-unaligned graph.
int build_graph_host(const float *data, uint64_t n, uint32_t d, const uint32_t *cand, uint32_t L, uint32_t R,
                     uint32_t entry, uint64_t seed, bool regular, uint32_t *out_adj, uint64_t *out_stats, int threads);

}  // namespace sqg_graph
