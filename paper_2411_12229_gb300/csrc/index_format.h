// index_format.h -- layout of the index file and of one vertex block
// (Sec. 3.1.3: the raw vector, then the FastScan data -- codes and factors
// of the out-neighbours -- then the neighbour ids, in one sequential block).
// Library-internal; the format itself is documented in include/sqg.h.
#pragma once
#include <cstdint>
#include <cstring>

namespace sqg_fmt {

constexpr uint32_t kVersion = 1;      // the rotation is the stored dense P^-1
constexpr uint32_t kVersionFjlt = 2;  // the query side applies the fast JLT (d a power of 2)
constexpr uint64_t kHeaderBytes = 256;
constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ull;
constexpr uint64_t kFnvPrime = 0x100000001b3ull;

struct Layout {
    uint64_t n;
    uint32_t d, R;
    uint32_t off_codes, off_factors, off_ids, block_bytes;
    uint64_t rot_offset, blocks_offset, file_bytes;
};

inline uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

inline Layout layout(uint64_t n, uint32_t d, uint32_t R) {
    Layout l{};
    l.n = n;
    l.d = d;
    l.R = R;
    l.off_codes = 4u * d;                     // raw vector: d fp32
    l.off_factors = l.off_codes + d * R / 8;  // codes: d bits per neighbour
    l.off_ids = l.off_factors + 16u * R;      // f_add, f_rescale, f_err, popcount
    l.block_bytes = (uint32_t)round_up(l.off_ids + 4ull * R, 128);
    l.rot_offset = kHeaderBytes;
    l.blocks_offset = round_up(kHeaderBytes + 4ull * d * d, 4096);
    l.file_bytes = l.blocks_offset + n * l.block_bytes;
    return l;
}

inline uint64_t load_u64(const unsigned char *p) {
    uint64_t v = 0;
    for (int i = 7; i >= 0; --i) v = (v << 8) | p[i];
    return v;
}
inline uint32_t load_u32(const unsigned char *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
inline void store_u64(unsigned char *p, uint64_t v) {
    for (int i = 0; i < 8; ++i) p[i] = (unsigned char)(v >> (8 * i));
}
inline void store_u32(unsigned char *p, uint32_t v) {
    for (int i = 0; i < 4; ++i) p[i] = (unsigned char)(v >> (8 * i));
}

// FNV-1a 64 over little-endian u64 words; nbytes must be a multiple of 8.
inline uint64_t fnv_words(uint64_t h, const unsigned char *p, uint64_t nbytes) {
    for (uint64_t i = 0; i + 8 <= nbytes; i += 8) {
        h ^= load_u64(p + i);
        h *= kFnvPrime;
    }
    return h;
}

// Metric of an index: squared Euclidean, or cosine similarity served as
// Euclidean search between unit vectors (the file holds unit-norm vectors,
// the search normalizes every query first).
constexpr uint32_t kMetricL2 = 0, kMetricCosine = 1;

inline void fill_header(unsigned char *h, const Layout &l, uint32_t entry, uint64_t seed_rot, uint64_t seed_graph,
                        uint64_t payload_hash, uint32_t version = kVersion, uint32_t metric = kMetricL2) {
    std::memset(h, 0, kHeaderBytes);
    std::memcpy(h, "SQG1", 4);
    store_u32(h + 4, version);
    store_u64(h + 8, l.n);
    store_u32(h + 16, l.d);
    store_u32(h + 20, l.R);
    store_u32(h + 24, l.block_bytes);
    store_u32(h + 28, entry);
    store_u32(h + 32, metric);
    store_u32(h + 36, l.off_codes);
    store_u32(h + 40, l.off_factors);
    store_u32(h + 44, l.off_ids);
    store_u64(h + 48, l.rot_offset);
    store_u64(h + 56, l.blocks_offset);
    store_u64(h + 64, l.file_bytes);
    store_u64(h + 72, seed_rot);
    store_u64(h + 80, seed_graph);
    store_u64(h + 88, payload_hash);
    store_u64(h + 96, fnv_words(kFnvBasis, h, 96));
}

struct Header {
    Layout l;
    uint32_t entry, metric, version;
    uint64_t payload_hash, seed_rot;
};

// splitmix64 (Steele, Lea, Flood 2014): the generator's output for state x.
inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The fast JLT's sign of round r (0..2) at coordinate i: -1 when bit 63 of
// splitmix64(seed ^ (r << 32 | i)) is set.
inline float fjlt_sign(uint64_t seed, uint32_t r, uint32_t i) {
    return (splitmix64(seed ^ (((uint64_t)r << 32) | i)) >> 63) ? -1.0f : 1.0f;
}

// Parse and check a header against the layout it implies and the file size.
inline bool parse_header(const unsigned char *h, uint64_t file_size, Header &out) {
    const uint32_t version = load_u32(h + 4);
    if (std::memcmp(h, "SQG1", 4) != 0 || (version != kVersion && version != kVersionFjlt)) return false;
    if (fnv_words(kFnvBasis, h, 96) != load_u64(h + 96)) return false;
    uint64_t n = load_u64(h + 8);
    uint32_t d = load_u32(h + 16), R = load_u32(h + 20);
    if (n == 0 || n > 0xFFFFFFF0ull || d == 0 || d % 32 || R == 0 || R % 32 || d > 65536 || R > 4096) return false;
    Layout l = layout(n, d, R);
    if (load_u32(h + 24) != l.block_bytes || load_u32(h + 36) != l.off_codes ||
        load_u32(h + 40) != l.off_factors || load_u32(h + 44) != l.off_ids || load_u64(h + 48) != l.rot_offset ||
        load_u64(h + 56) != l.blocks_offset || load_u64(h + 64) != l.file_bytes || l.file_bytes != file_size)
        return false;
    if (version == kVersionFjlt && (d & (d - 1)) != 0) return false;
    out.l = l;
    out.entry = load_u32(h + 28);
    out.metric = load_u32(h + 32);
    out.version = version;
    out.payload_hash = load_u64(h + 88);
    out.seed_rot = load_u64(h + 72);
    return out.entry < n && out.metric <= kMetricCosine;
}

}  // namespace sqg_fmt
