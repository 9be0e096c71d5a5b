// builder.cpp -- host-side index construction for the GB300 SymphonyQG library.
//
// Algorithm 2 (Indexing, Sec. 3.2) in pieces the Python driver strings
// together: candidate lists come from a brute-force kNN (sqg_knn_host) or
// from the GPU search on the previous iteration's graph; sqg_build_graph
// prunes them with NSG's rule and refines the graph so that every vertex has
// exactly R edges (Sec. 3.2.2; the steps are in graph_host.h, and graph.cu
// runs them on the GPU); sqg_write_index prepares the FastScan data
// (RaBitQ codes and factors of every edge, normalized about the source
// vertex, Sec. 3.1.1) and writes the file the search loads.
//
// Host code only: nothing here runs on the search path.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/sqg.h"
#include "graph_host.h"
#include "index_format.h"

namespace {

using sqg_graph::Cand;
using sqg_graph::parallel_for;

// Squared L2 distance, fp32, eight independent partial sums (d % 32 == 0):
// the brute-force kNN and the medoid, whose order decides nothing the
// search or the oracle must reproduce.
inline float l2(const float *a, const float *b, uint32_t d) {
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t i = 0; i < d; i += 8)
        for (int t = 0; t < 8; ++t) {
            float x = a[i + t] - b[i + t];
            s[t] += x * x;
        }
    return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
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

int sqg_graph::build_graph_host(const float *data, uint64_t n, uint32_t d, const uint32_t *cand, uint32_t L,
                                uint32_t R, uint32_t entry, uint64_t seed, bool regular, uint32_t *out_adj,
                                uint64_t *out_stats, int threads) {
    if (!data || !cand || !out_adj || n < 2 || d == 0 || d % 32 != 0 || R == 0 || R % 32 != 0 || L == 0 ||
        entry >= n || n > 0xFFFFFFF0ull)
        return SQG_ERR_INVALID_ARG;
    const uint32_t Rr = (uint32_t)std::min<uint64_t>(R, n - 1);  // tiny graphs: R distinct targets may not exist
    // 1. prune every vertex's own candidates (NSG rule)
    std::vector<Cand> k1((size_t)n * Rr);
    std::vector<uint32_t> n1(n, 0);
    std::atomic<uint64_t> deg_sum{0};
    parallel_for(n, threads, [&](uint64_t u) {
        std::vector<Cand> c, kept;
        sqg_graph::own_cands(data, n, d, cand, L, u, c);
        sqg_graph::nsg_prune(data, d, c, Rr, kept);
        std::copy(kept.begin(), kept.end(), k1.begin() + (size_t)u * Rr);
        n1[u] = (uint32_t)kept.size();
        deg_sum += kept.size();
    });
    // 2. reverse edges, re-prune; 3. angle rule; 4. random fill and rows
    std::vector<uint64_t> roff;
    std::vector<Cand> rev;
    sqg_graph::reverse_edges(n, k1.data(), n1.data(), Rr, roff, rev);
    std::atomic<uint64_t> n_supp{0}, n_fill{0};
    parallel_for(n, threads, [&](uint64_t u) {
        std::vector<Cand> k2;
        if (sqg_graph::refine_vertex(data, n, d, cand, L, Rr, u, k1.data() + (size_t)u * Rr, n1[u],
                                     rev.data() + roff[u], roff[u + 1] - roff[u], regular, k2))
            n_supp++;
        if (sqg_graph::fill_and_write(data, n, d, R, Rr, seed, u, regular, k2, out_adj)) n_fill++;
    });
    // 5. reachability from the entry point
    const uint64_t repairs = sqg_graph::repair_reachability(n, cand, L, R, entry, out_adj);
    if (out_stats) {
        out_stats[0] = deg_sum.load() * 1000 / n;
        out_stats[1] = n_supp.load();
        out_stats[2] = n_fill.load();
        out_stats[3] = repairs;
    }
    return SQG_OK;
}

extern "C" int sqg_build_graph(const float *data, uint64_t n, uint32_t d, const uint32_t *cand, uint32_t L,
                               uint32_t R, uint32_t entry, uint64_t seed, uint32_t *out_adj, uint64_t *out_stats,
                               int threads) {
    return sqg_graph::build_graph_host(data, n, d, cand, L, R, entry, seed, true, out_adj, out_stats, threads);
}

extern "C" int sqg_write_index2(const char *path, const float *data, uint64_t n, uint32_t d, const uint32_t *adj,
                                uint32_t R, const float *rot, uint32_t entry, uint64_t seed_rotation,
                                uint64_t seed_graph, int threads, uint32_t rotation_kind, uint32_t metric) {
    if (!path || !data || !adj || !rot || n == 0 || d == 0 || d % 32 != 0 || R == 0 || R % 32 != 0 || entry >= n ||
        rotation_kind > 1 || (rotation_kind == 1 && (d & (d - 1)) != 0) || metric > sqg_fmt::kMetricCosine)
        return SQG_ERR_INVALID_ARG;
    for (uint64_t i = 0; i < n * R; ++i)
        if (adj[i] >= n && adj[i] != SQG_NO_ID) return SQG_ERR_INVALID_ARG;  // an empty slot is SQG_NO_ID
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
                if (o == SQG_NO_ID) {  // an empty slot of a degree-unaligned row: zero codes and factors
                    for (uint32_t w = 0; w < d / 32; ++w) codes[w * R + j] = 0u;
                    fa[j] = fr[j] = fe[j] = 0.0f;
                    pc[j] = 0;
                    continue;
                }
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
