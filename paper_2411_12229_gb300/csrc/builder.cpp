// builder.cpp -- host-side index construction for the GB300 SymphonyQG library.
//
// Algorithm 2 (Indexing, Sec. 3.2) in pieces the Python driver strings
// together: candidate lists come from a brute-force kNN (sqg_knn_host) or
// from the GPU search on the previous iteration's graph; sqg_build_graph
// prunes them with NSG's rule and refines the graph so that every vertex has
// exactly R edges (Sec. 3.2.2); sqg_write_index prepares the FastScan data
// (RaBitQ codes and factors of every edge, normalized about the source
// vertex, Sec. 3.1.1) and writes the file the search loads.
//
// Host code only: nothing here runs on the search path.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "../../include/sqg.h"
#include "index_format.h"

namespace {

int resolve_threads(int t) {
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

// Squared L2 distance, fp32, eight independent partial sums (d % 32 == 0).
inline float l2(const float *a, const float *b, uint32_t d) {
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t i = 0; i < d; i += 8)
        for (int t = 0; t < 8; ++t) {
            float x = a[i + t] - b[i + t];
            s[t] += x * x;
        }
    return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

// Squared L2 distance in the search's exact-distance order, which the
// pruning and the angle rule use so that their decisions are those of the
// GPU graph kernels: 32 partial sums, partial l over the float4 chunks l,
// l+32, ... with fma(x, x, acc) on their four coordinates in order, then
// pairwise sums of partials l and l+16, l and l+8, ..., l and l+1.
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

uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// NSG's pruning rule (Sec. 3.2.1, after NSG): walk the candidates nearest
// first and keep c unless a kept w is closer to c than the vertex is
// (d(w,c) < d(u,c)), which keeps every pair of out-edges at least 60
// degrees apart.
void nsg_prune(const float *data, uint32_t d, const std::vector<Cand> &cands, uint32_t R,
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
void angle_supplement(const float *data, uint32_t d, const float *xu, const std::vector<Cand> &kept,
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

}  // namespace

extern "C" int sqg_knn_host(const float *data, uint64_t n, uint32_t d, uint32_t k, uint32_t *out, int threads) {
    if (!data || !out || n == 0 || d == 0 || d % 32 != 0 || k == 0) return SQG_ERR_INVALID_ARG;
    parallel_for(n, threads, [&](uint64_t i) {
        std::vector<Cand> c;
        c.reserve(n);
        const float *xi = data + i * d;
        for (uint64_t j = 0; j < n; ++j)
            if (j != i) c.push_back({l2(xi, data + j * d, d), (uint32_t)j});
        uint64_t kk = std::min<uint64_t>(k, c.size());
        std::partial_sort(c.begin(), c.begin() + kk, c.end());
        for (uint64_t t = 0; t < k; ++t) out[i * k + t] = t < kk ? c[t].id : SQG_NO_ID;
    }, 16);
    return SQG_OK;
}

extern "C" uint32_t sqg_medoid(const float *data, uint64_t n, uint32_t d, int threads) {
    if (!data || n == 0) return 0;
    std::vector<double> mean(d, 0.0);
    for (uint64_t i = 0; i < n; ++i)
        for (uint32_t t = 0; t < d; ++t) mean[t] += data[i * d + t];
    std::vector<float> m(d);
    for (uint32_t t = 0; t < d; ++t) m[t] = (float)(mean[t] / (double)n);
    std::vector<float> dist(n);
    parallel_for(n, threads, [&](uint64_t i) { dist[i] = l2(data + i * d, m.data(), d); }, 4096);
    uint64_t best = 0;
    for (uint64_t i = 1; i < n; ++i)
        if (dist[i] < dist[best]) best = i;
    return (uint32_t)best;
}

extern "C" int sqg_build_graph(const float *data, uint64_t n, uint32_t d, const uint32_t *cand, uint32_t L,
                               uint32_t R, uint32_t entry, uint64_t seed, uint32_t *out_adj, uint64_t *out_stats,
                               int threads) {
    if (!data || !cand || !out_adj || n < 2 || d == 0 || d % 32 != 0 || R == 0 || R % 32 != 0 || L == 0 ||
        entry >= n || n > 0xFFFFFFF0ull)
        return SQG_ERR_INVALID_ARG;
    const uint32_t Rr = (uint32_t)std::min<uint64_t>(R, n - 1);  // tiny graphs: R distinct targets may not exist
    std::vector<std::vector<Cand>> kept(n);
    std::atomic<uint64_t> deg_sum{0};

    auto own_cands = [&](uint64_t u, std::vector<Cand> &c) {
        c.clear();
        const float *xu = data + u * d;
        for (uint32_t t = 0; t < L; ++t) {
            uint32_t v = cand[u * L + t];
            if (v == SQG_NO_ID || v >= n || v == u) continue;
            c.push_back({l2c(xu, data + (uint64_t)v * d, d), v});
        }
        std::sort(c.begin(), c.end(), [](const Cand &a, const Cand &b) { return a.id < b.id; });
        c.erase(std::unique(c.begin(), c.end(), [](const Cand &a, const Cand &b) { return a.id == b.id; }),
                c.end());
        std::sort(c.begin(), c.end());
    };

    // 1. prune every vertex's candidates (NSG rule)
    parallel_for(n, threads, [&](uint64_t u) {
        std::vector<Cand> c;
        own_cands(u, c);
        nsg_prune(data, d, c, Rr, kept[u]);
        deg_sum += kept[u].size();
    });

    // 2. offer every kept edge u -> v back to v as a candidate (reverse edges)
    std::vector<uint32_t> indeg(n + 1, 0);
    for (uint64_t u = 0; u < n; ++u)
        for (const Cand &c : kept[u]) indeg[c.id + 1]++;
    std::vector<uint64_t> roff(n + 1, 0);
    for (uint64_t v = 0; v < n; ++v) roff[v + 1] = roff[v] + indeg[v + 1];
    std::vector<Cand> rev(roff[n]);
    {
        std::vector<uint64_t> fill(roff.begin(), roff.end() - 1);
        for (uint64_t u = 0; u < n; ++u)
            for (const Cand &c : kept[u]) rev[fill[c.id]++] = {c.d, (uint32_t)u};
    }

    std::atomic<uint64_t> n_supp{0}, n_fill{0};
    parallel_for(n, threads, [&](uint64_t u) {
        const float *xu = data + u * d;
        std::vector<Cand> pool(kept[u]);
        for (uint64_t t = roff[u]; t < roff[u + 1]; ++t) pool.push_back(rev[t]);
        std::sort(pool.begin(), pool.end(), [](const Cand &a, const Cand &b) { return a.id < b.id; });
        pool.erase(std::unique(pool.begin(), pool.end(), [](const Cand &a, const Cand &b) { return a.id == b.id; }),
                   pool.end());
        std::sort(pool.begin(), pool.end());
        std::vector<Cand> k2;
        nsg_prune(data, d, pool, Rr, k2);
        // 3. supplement to exactly R with the adaptive angle rule
        if (k2.size() < Rr) {
            n_supp++;
            std::vector<Cand> all;
            own_cands(u, all);
            for (uint64_t t = roff[u]; t < roff[u + 1]; ++t) all.push_back(rev[t]);
            std::sort(all.begin(), all.end(), [](const Cand &a, const Cand &b) { return a.id < b.id; });
            all.erase(std::unique(all.begin(), all.end(), [](const Cand &a, const Cand &b) { return a.id == b.id; }),
                      all.end());
            std::vector<uint32_t> have;
            for (auto &c : k2) have.push_back(c.id);
            std::sort(have.begin(), have.end());
            std::vector<Cand> extra;
            for (auto &c : all)
                if (!std::binary_search(have.begin(), have.end(), c.id)) extra.push_back(c);
            std::sort(extra.begin(), extra.end());
            uint32_t cap = d >= 512 ? 2 * Rr : 3 * Rr;
            if (extra.size() > cap) extra.resize(cap);
            std::vector<Cand> sup;
            angle_supplement(data, d, xu, k2, extra, Rr - (uint32_t)k2.size(), sup);
            k2.insert(k2.end(), sup.begin(), sup.end());
            std::sort(k2.begin(), k2.end());
        }
        // 4. random fill when the candidates run out (footnote of Sec. 3.2.2)
        if (k2.size() < Rr) {
            n_fill++;
            uint64_t st = seed ^ (u * 0x9E3779B97F4A7C15ull);
            std::vector<uint32_t> have;
            for (auto &c : k2) have.push_back(c.id);
            while (k2.size() < Rr) {
                uint32_t v = (uint32_t)(splitmix64(st) % n);
                if (v == u || std::find(have.begin(), have.end(), v) != have.end()) continue;
                have.push_back(v);
                k2.push_back({l2c(xu, data + (uint64_t)v * d, d), v});
            }
            std::sort(k2.begin(), k2.end());
        }
        for (uint32_t t = 0; t < R; ++t) out_adj[u * R + t] = t < k2.size() ? k2[t].id : k2[t % k2.size()].id;
    });

    // 5. reachability from the entry point: connect each unreachable vertex
    //    from a nearby reachable vertex, replacing that vertex's edge whose
    //    target has the most other in-edges.
    std::vector<uint32_t> in(n, 0);
    for (uint64_t i = 0; i < n * R; ++i) in[out_adj[i]]++;
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
                    if (!seen[v]) { seen[v] = 1; stack.push_back(v); }
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
            // replace the edge whose target has the most in-edges (farthest on ties)
            int slot = (int)R - 1;
            for (int t = (int)R - 2; t >= 0; --t)
                if (in[row[t]] > in[row[slot]]) slot = t;
            in[row[slot]]--;
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
    if (out_stats) {
        out_stats[0] = deg_sum.load() * 1000 / n;
        out_stats[1] = n_supp.load();
        out_stats[2] = n_fill.load();
        out_stats[3] = repairs;
    }
    return SQG_OK;
}

extern "C" int sqg_write_index2(const char *path, const float *data, uint64_t n, uint32_t d, const uint32_t *adj,
                                uint32_t R, const float *rot, uint32_t entry, uint64_t seed_rotation,
                                uint64_t seed_graph, int threads, uint32_t rotation_kind, uint32_t metric) {
    if (!path || !data || !adj || !rot || n == 0 || d == 0 || d % 32 != 0 || R == 0 || R % 32 != 0 || entry >= n ||
        rotation_kind > 1 || (rotation_kind == 1 && (d & (d - 1)) != 0) || metric > sqg_fmt::kMetricCosine)
        return SQG_ERR_INVALID_ARG;
    for (uint64_t i = 0; i < n * R; ++i)
        if (adj[i] >= n) return SQG_ERR_INVALID_ARG;
    if (metric == sqg_fmt::kMetricCosine) {  // a cosine index holds unit vectors (or zero vectors)
        std::atomic<uint64_t> bad{0};
        parallel_for(n, threads, [&](uint64_t v) {
            double s = 0.0;
            for (uint32_t i = 0; i < d; ++i) s += (double)data[v * d + i] * data[v * d + i];
            if (s != 0.0 && std::fabs(s - 1.0) > 1e-4) bad++;
        }, 4096);
        if (bad.load()) return SQG_ERR_INVALID_ARG;
    }
    sqg_fmt::Layout lay = sqg_fmt::layout(n, d, R);

    // P^-1 x for every vertex, fp64 (the rotation is linear, so the rotated
    // edge P^-1(o - c) is the difference of rotated endpoints).
    std::vector<double> rv;
    try {
        rv.resize(n * d);
    } catch (...) {
        return SQG_ERR_OOM;
    }
    parallel_for(n, threads, [&](uint64_t v) {
        const float *x = data + v * d;
        double *y = rv.data() + v * d;
        for (uint32_t i = 0; i < d; ++i) {
            const float *r = rot + (uint64_t)i * d;
            double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
            for (uint32_t j = 0; j < d; j += 4) {
                s0 += (double)r[j] * x[j];
                s1 += (double)r[j + 1] * x[j + 1];
                s2 += (double)r[j + 2] * x[j + 2];
                s3 += (double)r[j + 3] * x[j + 3];
            }
            y[i] = (s0 + s1) + (s2 + s3);
        }
    }, 256);

    FILE *f = std::fopen(path, "wb");
    if (!f) return SQG_ERR_IO;
    std::vector<unsigned char> header(sqg_fmt::kHeaderBytes, 0);
    uint64_t h = sqg_fmt::kFnvBasis;
    auto put = [&](const void *p, size_t nbytes) -> bool {
        h = sqg_fmt::fnv_words(h, (const unsigned char *)p, nbytes);
        return std::fwrite(p, 1, nbytes, f) == nbytes;
    };
    bool ok = std::fwrite(header.data(), 1, header.size(), f) == header.size();
    ok = ok && put(rot, sizeof(float) * (uint64_t)d * d);
    std::vector<unsigned char> pad(lay.blocks_offset - lay.rot_offset - sizeof(float) * (uint64_t)d * d, 0);
    ok = ok && put(pad.data(), pad.size());

    const double sd = std::sqrt((double)d), sd1 = std::sqrt((double)d - 1.0);
    const uint64_t chunk = 8192;
    std::vector<unsigned char> buf;
    for (uint64_t c0 = 0; ok && c0 < n; c0 += chunk) {
        uint64_t c1 = std::min(n, c0 + chunk);
        buf.assign((c1 - c0) * lay.block_bytes, 0);
        parallel_for(c1 - c0, threads, [&](uint64_t t) {
            uint64_t c = c0 + t;
            unsigned char *b = buf.data() + t * lay.block_bytes;
            std::memcpy(b, data + c * d, sizeof(float) * d);
            uint32_t *codes = (uint32_t *)(b + lay.off_codes);
            float *fa = (float *)(b + lay.off_factors), *fr = fa + R, *fe = fa + 2 * R;
            uint32_t *pc = (uint32_t *)(fa + 3 * R);
            uint32_t *ids = (uint32_t *)(b + lay.off_ids);
            const double *cr = rv.data() + c * d;
            for (uint32_t j = 0; j < R; ++j) {
                uint32_t o = adj[c * R + j];
                ids[j] = o;
                double n2 = 0.0;
                for (uint32_t i = 0; i < d; ++i) {
                    double u = (double)data[(uint64_t)o * d + i] - (double)data[c * d + i];
                    n2 += u * u;
                }
                double n_o = std::sqrt(n2);
                if (n_o == 0.0) {  // neighbour equal to its centre: estimate = exact distance
                    for (uint32_t w = 0; w < d / 32; ++w) codes[w * R + j] = 0u;
                    fa[j] = fr[j] = fe[j] = 0.0f;
                    pc[j] = 0;
                    continue;
                }
                const double *orr = rv.data() + (uint64_t)o * d;
                double alpha = 0.0, xc = 0.0;
                uint32_t cnt = 0;
                for (uint32_t w = 0; w < d / 32; ++w) {
                    uint32_t word = 0;
                    for (uint32_t bit = 0; bit < 32; ++bit) {
                        uint32_t i = w * 32 + bit;
                        double v = (orr[i] - cr[i]) / n_o;
                        bool pos = v >= 0.0;
                        word |= (uint32_t)pos << bit;
                        alpha += std::fabs(v);
                        xc += pos ? cr[i] : -cr[i];
                        cnt += pos;
                    }
                    codes[w * R + j] = word;
                }
                alpha /= sd;
                xc /= sd;
                fa[j] = (float)(n_o * n_o + 2.0 * n_o * xc / alpha);
                fr[j] = (float)(-2.0 * n_o / alpha);
                double a2 = alpha * alpha;
                fe[j] = (float)(2.0 * n_o * std::sqrt(std::max(0.0, (1.0 - a2) / a2)) / sd1);
                pc[j] = cnt;
            }
        }, 64);
        ok = put(buf.data(), buf.size());
    }
    sqg_fmt::fill_header(header.data(), lay, entry, seed_rotation, seed_graph, h,
                         rotation_kind == 1 ? sqg_fmt::kVersionFjlt : sqg_fmt::kVersion, metric);
    ok = ok && std::fseek(f, 0, SEEK_SET) == 0 && std::fwrite(header.data(), 1, header.size(), f) == header.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SQG_OK : SQG_ERR_IO;
}

extern "C" int sqg_write_index(const char *path, const float *data, uint64_t n, uint32_t d, const uint32_t *adj,
                               uint32_t R, const float *rot, uint32_t entry, uint64_t seed_rotation,
                               uint64_t seed_graph, int threads) {
    return sqg_write_index2(path, data, n, d, adj, R, rot, entry, seed_rotation, seed_graph, threads, 0,
                            sqg_fmt::kMetricL2);
}
