/*
 * sqg_oracle.c -- plain, slow, single-threaded CPU oracle for SymphonyQG's
 * query phase (arXiv 2411.12229).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and
 * the benchmark's CPU-baseline leg may load this file.  The library never
 * links, imports or calls it, and it shares no code with the library: it
 * has its own index-file reader, its own estimator and its own search.
 *
 * What each function follows:
 *   - Eq. (1)-(2), "normalization": ||o_r-q_r||^2 = ||o_r-c||^2 + ||q_r-c||^2
 *     - 2 ||o_r-c|| ||q_r-c|| <o,q>                   (Sec. 2.2)
 *   - Eq. (3), the codebook C_rand = { P x : x[i] in {+-1/sqrt(D)} } and the
 *     estimator <o_bar,q>/<o_bar,o> of <o,q>           (Sec. 2.2)
 *   - Eq. (4), rotation equivalence <o_bar,q> = <x_bar, P^-1 q>  (Sec. 2.2)
 *   - Eq. (5)-(6), centre-independent form
 *     <x_bar,P^-1 q> = (<x_bar,P^-1 q_r> - <x_bar,P^-1 c>)/||q_r-c||
 *                                                       (Sec. 3.1.1)
 *   - Algorithm 1 (Querying) with multiple estimated distances and implicit
 *     re-ranking                                        (Sec. 3.1.2-3.1.3)
 *   - Algorithm 2's "adjust G": NSG's occlusion rule and the adaptive
 *     angle supplement                                   (Sec. 3.2.1-3.2.2)
 *
 * Readings taken where the paper is silent (each also stated at its use):
 *   R1 the query is quantized to 4 bits per coordinate, uniform on
 *      [min q', max q'], rounding half up (the paper gives no query bits);
 *   R2 a rotated coordinate exactly 0 gets code bit 1;
 *   R3 a neighbour identical to its centre (||o-c|| = 0) gets all-zero code
 *      bits and zero factors, so its estimate is the centre's exact distance;
 *   R4 the beam is totally ordered by (key, id); the result by (dist, id);
 *   R5 visited copies stay in the beam and hold their slots until evicted;
 *      an identical (key, id) pair is stored once;
 *   R6 a hop cap stops a search after hop_cap expansions with a status flag;
 *   R7 admission key = estimate - eps0 * bound, bound = f_err*||q_r-c||
 *      (RaBitQ's bound form); eps0 = 0 is Algorithm 1 exactly;
 *   R8 the initial beam entry carries the entry point's exact distance;
 *   R16 cosine similarity (Sec. 3: RaBitQ serves Euclidean distance and
 *      cosine similarity) is served as Euclidean search between unit
 *      vectors: an index of metric 1 stores unit-norm vectors, and every
 *      query is scaled to unit norm before anything else (orc_normalize_f32);
 *      the distances returned are ||q/|q| - x||^2 = 2 - 2 cos(q, x);
 *   R17 a degree-unaligned graph (the "w/o GR" ablation of Sec. 5, no
 *      degree alignment by the angle rule) keeps R slots per vertex and
 *      marks the empty ones with id ORC_NO_ID, zero code bits and zero
 *      factors; the search skips an empty slot.
 *
 * Floating point.  Fp64 functions give the plain definitions (used by the
 * pins).  The search takes its decisions (which vertex to expand, what
 * enters the beam, when to stop) in fp32, in the same precision and order
 * as the device code, because a float decides an integer there:
 *   - rotation: q'_i = sum over chunks c = 0, 1, ... (in order, from 0) of
 *     s_c = fmaf-chain over j = 32c..32c+31 of P^-1[i][j]*q_j from 0;
 *   - exact distance: 32 partial sums, partial l runs over float4 chunks
 *     l, l+32, ... (x, y, z, w in order, fmaf(d,d,acc)), then a pairwise
 *     tree that adds partials l and l^16, then ^8, ^4, ^2, ^1;
 *   - estimate: ip = fmaf(delta, 2S-Sq, v_l*(2pc-D)) * (1/sqrt(D)),
 *     est = fmaf(f_rescale, ip, f_add + dist_c), key = est - eps0*bound.
 * Build with -ffp-contract=off so that no other product is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_IO (-2)
#define ORC_ERR_FORMAT (-3)
#define ORC_ERR_OOM (-4)

#define ORC_STATUS_CAPACITY 1u
#define ORC_STATUS_LEARNED_STOP 2u

#define ORC_NO_ID 0xFFFFFFFFu

/* ------------------------------------------------------------------ */
/* Index file (version 1).  Little-endian.                             */
/*   header, 256 bytes:                                                */
/*     0 magic "SQG1" | 4 version u32 | 8 n u64 | 16 d u32 | 20 R u32   */
/*     24 block_bytes u32 | 28 entry u32 | 32 metric u32 (0 squared    */
/*     Euclidean, 1 cosine: unit-norm vectors, queries normalized, R16) */
/*     36 off_codes u32 | 40 off_factors u32 | 44 off_ids u32           */
/*     48 rot_offset u64 | 56 blocks_offset u64 | 64 file_bytes u64     */
/*     72 seed_rotation u64 | 80 seed_graph u64 | 88 payload_hash u64   */
/*     96 header_hash u64 (over bytes 0..95) | rest zero                */
/*   rotation P^-1: d*d float32 row-major at rot_offset                 */
/*   version 2: the rotation is the fast JLT of Sec. 3.1.4 (d a power   */
/*     of 2): three rounds of a sign flip s_r followed by the Walsh-    */
/*     Hadamard transform scaled by 1/sqrt(d); s_r[i] = -1 when bit 63  */
/*     of splitmix64(seed_rotation ^ (r << 32 | i)) is set, else +1.    */
/*     The d*d region then holds the same transform as a dense matrix   */
/*     (what the index's codes were built with).                        */
/*   n vertex blocks of block_bytes each at blocks_offset; a block is   */
/*     raw vector  d float32                          @ 0               */
/*     codes       d*R bits: u32 word w of neighbour j at index w*R+j;  */
/*                 bit (i mod 32) of word i/32 is dimension i           */
/*                                                   @ off_codes        */
/*     factors     f_add[R], f_rescale[R], f_err[R] float32,            */
/*                 popcount[R] u32                    @ off_factors     */
/*     neighbour ids R u32                            @ off_ids         */
/*   hashes: FNV-1a 64 over little-endian u64 words.                    */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t n;
    uint32_t d, R, block_bytes, entry, metric;
    uint32_t off_codes, off_factors, off_ids;
    uint64_t rot_offset, blocks_offset, file_bytes;
    unsigned char *file; /* whole file */
    const float *rot;    /* d*d */
    const unsigned char *blocks;
    int fjlt;            /* version 2: the query side uses the fast JLT */
    float *signs;        /* 3*d, +1 / -1 (version 2) */
} orc_index;

static uint32_t rd32(const unsigned char *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static uint64_t rd64(const unsigned char *p) { return (uint64_t)rd32(p) | ((uint64_t)rd32(p + 4) << 32); }

static uint64_t fnv_words(const unsigned char *p, uint64_t nbytes) {
    uint64_t h = 0xcbf29ce484222325ull;
    for (uint64_t i = 0; i + 8 <= nbytes; i += 8) {
        h ^= rd64(p + i);
        h *= 0x100000001b3ull;
    }
    return h;
}

void orc_index_free(orc_index *ix) {
    if (!ix) return;
    free(ix->file);
    free(ix->signs);
    free(ix);
}

/* splitmix64 (Steele, Lea, Flood 2014): the output for state x, i.e. the
 * first value the generator returns after being seeded with x. */
uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The fast JLT's three sign vectors (3*d values, +1 / -1). */
void orc_fjlt_signs(uint64_t seed, uint32_t d, float *signs) {
    for (uint32_t r = 0; r < 3; ++r)
        for (uint32_t i = 0; i < d; ++i)
            signs[r * d + i] = (orc_splitmix64(seed ^ (((uint64_t)r << 32) | i)) >> 63) ? -1.0f : 1.0f;
}

int orc_index_load(const char *path, orc_index **out) {
    if (!path || !out) return ORC_ERR_ARG;
    *out = NULL;
    FILE *f = fopen(path, "rb");
    if (!f) return ORC_ERR_IO;
    if (fseek(f, 0, SEEK_END) != 0) { fclose(f); return ORC_ERR_IO; }
    long long sz = ftell(f);
    if (sz < 256) { fclose(f); return ORC_ERR_FORMAT; }
    rewind(f);
    unsigned char *buf = (unsigned char *)malloc((size_t)sz);
    if (!buf) { fclose(f); return ORC_ERR_OOM; }
    if (fread(buf, 1, (size_t)sz, f) != (size_t)sz) { free(buf); fclose(f); return ORC_ERR_IO; }
    fclose(f);
    const uint32_t version = rd32(buf + 4);
    if (memcmp(buf, "SQG1", 4) != 0 || (version != 1u && version != 2u)) { free(buf); return ORC_ERR_FORMAT; }
    if (fnv_words(buf, 96) != rd64(buf + 96)) { free(buf); return ORC_ERR_FORMAT; }
    orc_index *ix = (orc_index *)calloc(1, sizeof(orc_index));
    if (!ix) { free(buf); return ORC_ERR_OOM; }
    ix->n = rd64(buf + 8);
    ix->d = rd32(buf + 16);
    ix->R = rd32(buf + 20);
    ix->block_bytes = rd32(buf + 24);
    ix->entry = rd32(buf + 28);
    ix->metric = rd32(buf + 32);
    if (ix->metric > 1u) { free(buf); free(ix); return ORC_ERR_FORMAT; }
    ix->off_codes = rd32(buf + 36);
    ix->off_factors = rd32(buf + 40);
    ix->off_ids = rd32(buf + 44);
    ix->rot_offset = rd64(buf + 48);
    ix->blocks_offset = rd64(buf + 56);
    ix->file_bytes = rd64(buf + 64);
    ix->file = buf;
    uint64_t d = ix->d, R = ix->R;
    int ok = ix->n > 0 && d > 0 && d % 32 == 0 && R > 0 && R % 32 == 0 &&
             ix->off_codes == 4 * d && ix->off_factors == ix->off_codes + d * R / 8 &&
             ix->off_ids == ix->off_factors + 16 * R && ix->block_bytes >= ix->off_ids + 4 * R &&
             ix->entry < ix->n && ix->file_bytes == (uint64_t)sz &&
             ix->rot_offset + 4 * d * d <= ix->blocks_offset &&
             ix->blocks_offset + ix->n * ix->block_bytes == ix->file_bytes;
    if (!ok || fnv_words(buf + ix->rot_offset, ix->file_bytes - ix->rot_offset) != rd64(buf + 88)) {
        orc_index_free(ix);
        return ORC_ERR_FORMAT;
    }
    ix->rot = (const float *)(buf + ix->rot_offset);
    ix->blocks = buf + ix->blocks_offset;
    if (version == 2u) {
        if (d & (d - 1)) { orc_index_free(ix); return ORC_ERR_FORMAT; }  /* a power of 2 */
        ix->fjlt = 1;
        ix->signs = (float *)malloc(sizeof(float) * 3 * d);
        if (!ix->signs) { orc_index_free(ix); return ORC_ERR_OOM; }
        orc_fjlt_signs(rd64(buf + 72), (uint32_t)d, ix->signs);
    }
    *out = ix;
    return ORC_OK;
}

void orc_index_shape(const orc_index *ix, uint64_t *n, uint32_t *d, uint32_t *R, uint32_t *entry,
                     uint32_t *block_bytes) {
    *n = ix->n; *d = ix->d; *R = ix->R; *entry = ix->entry; *block_bytes = ix->block_bytes;
}

const float *orc_rotation(const orc_index *ix) { return ix->rot; }
uint32_t orc_metric(const orc_index *ix) { return ix->metric; }

/* The fast JLT's signs (3*d) of a version-2 index, else NULL. */
const float *orc_fjlt_index_signs(const orc_index *ix) { return ix->fjlt ? ix->signs : NULL; }

static const unsigned char *blk(const orc_index *ix, uint32_t v) {
    return ix->blocks + (uint64_t)v * ix->block_bytes;
}
const float *orc_raw(const orc_index *ix, uint32_t v) { return (const float *)blk(ix, v); }
static uint32_t code_word(const orc_index *ix, uint32_t v, uint32_t w, uint32_t j) {
    return rd32(blk(ix, v) + ix->off_codes + 4u * (w * ix->R + j));
}
static float fac(const orc_index *ix, uint32_t v, uint32_t which, uint32_t j) {
    float x;
    memcpy(&x, blk(ix, v) + ix->off_factors + 4u * (which * ix->R + j), 4);
    return x;
}
static uint32_t popc_stored(const orc_index *ix, uint32_t v, uint32_t j) {
    return rd32(blk(ix, v) + ix->off_factors + 4u * (3u * ix->R + j));
}
static uint32_t nbr(const orc_index *ix, uint32_t v, uint32_t j) {
    return rd32(blk(ix, v) + ix->off_ids + 4u * j);
}
/* code bit of dimension i for neighbour j of vertex v */
static int code_bit(const orc_index *ix, uint32_t v, uint32_t j, uint32_t i) {
    return (int)((code_word(ix, v, i / 32u, j) >> (i % 32u)) & 1u);
}

/* Export a vertex's neighbours, code bits (one byte per dimension) and
 * factors, for the tests. */
void orc_vertex(const orc_index *ix, uint32_t v, uint32_t *ids, unsigned char *bits, float *f_add,
                float *f_rescale, float *f_err, uint32_t *pc) {
    for (uint32_t j = 0; j < ix->R; ++j) {
        ids[j] = nbr(ix, v, j);
        f_add[j] = fac(ix, v, 0, j);
        f_rescale[j] = fac(ix, v, 1, j);
        f_err[j] = fac(ix, v, 2, j);
        pc[j] = popc_stored(ix, v, j);
        for (uint32_t i = 0; i < ix->d; ++i) bits[(uint64_t)j * ix->d + i] = (unsigned char)code_bit(ix, v, j, i);
    }
}

/* ------------------------------------------------------------------ */
/* Plain fp64 definitions                                              */
/* ------------------------------------------------------------------ */

/* y = P^-1 x in fp64 (Eq. (4): the rotation moves onto the query). */
void orc_rotate_f64(const float *rot, uint32_t d, const float *x, double *y) {
    for (uint32_t i = 0; i < d; ++i) {
        double s = 0.0;
        for (uint32_t j = 0; j < d; ++j) s += (double)rot[(uint64_t)i * d + j] * (double)x[j];
        y[i] = s;
    }
}

/* y = P^-1 x for the fast JLT in fp64 (Sec. 3.1.4): for r = 0, 1, 2 the
 * signs s_r, the Walsh-Hadamard transform H (entries +1/-1, H_ij =
 * (-1)^popcount(i & j)) and the scale 1/sqrt(d).  d a power of 2. */
void orc_fjlt_f64(const float *signs, uint32_t d, const float *x, double *y) {
    const double c = 1.0 / sqrt((double)d);
    for (uint32_t i = 0; i < d; ++i) y[i] = (double)x[i];
    for (uint32_t r = 0; r < 3; ++r) {
        for (uint32_t i = 0; i < d; ++i) y[i] *= (double)signs[r * d + i];
        for (uint32_t h = 1; h < d; h <<= 1)
            for (uint32_t i = 0; i < d; i += 2 * h)
                for (uint32_t j = i; j < i + h; ++j) {
                    const double a = y[j], b = y[j + h];
                    y[j] = a + b;
                    y[j + h] = a - b;
                }
        for (uint32_t i = 0; i < d; ++i) y[i] *= c;
    }
}

double orc_sqdist_f64(const float *a, const float *b, uint32_t d) {
    double s = 0.0;
    for (uint32_t i = 0; i < d; ++i) {
        double t = (double)a[i] - (double)b[i];
        s += t * t;
    }
    return s;
}

/*
 * RaBitQ quantization of neighbour o about centre c (Sec. 2.2 with the
 * vertex as centre, Sec. 3.1.1):
 *   o = (o_r - c)/||o_r - c||, v = P^-1 o; the nearest codeword P x_bar has
 *   x_bar[i] = sign(v[i])/sqrt(D) (Eq. (3)); bit b_i = 1 iff v[i] >= 0 (R2);
 *   alpha = <o_bar, o> = <x_bar, v> = sum|v_i|/sqrt(D);
 *   xc = <x_bar, P^-1 c>.
 * Substituting Eq. (6) into Eq. (2), ||q_r - c|| cancels:
 *   est = n_o^2 + dist_c - 2 n_o (<x_bar,q'> - xc)/alpha
 *       = f_add + dist_c + f_rescale * <x_bar, q'>
 * with f_add = n_o^2 + 2 n_o xc/alpha, f_rescale = -2 n_o/alpha, q' = P^-1 q_r.
 * Error factor (R7): f_err = 2 n_o sqrt((1-alpha^2)/alpha^2)/sqrt(D-1).
 * out[0..6] = n_o, alpha, xc, f_add, f_rescale, f_err, popcount.
 */
void orc_quantize_edge(const float *rot, uint32_t d, const float *c, const float *o, unsigned char *bits,
                       double *out) {
    double *u = (double *)malloc(sizeof(double) * d);
    double n2 = 0.0;
    for (uint32_t i = 0; i < d; ++i) {
        u[i] = (double)o[i] - (double)c[i];
        n2 += u[i] * u[i];
    }
    double n_o = sqrt(n2);
    double sd = sqrt((double)d);
    if (n_o == 0.0) { /* R3 */
        memset(bits, 0, d);
        out[0] = 0.0; out[1] = 1.0; out[2] = 0.0; out[3] = 0.0; out[4] = 0.0; out[5] = 0.0; out[6] = 0.0;
        free(u);
        return;
    }
    double alpha = 0.0, xc = 0.0, pc = 0.0;
    for (uint32_t i = 0; i < d; ++i) {
        double v = 0.0, cr = 0.0;
        for (uint32_t j = 0; j < d; ++j) {
            v += (double)rot[(uint64_t)i * d + j] * u[j];
            cr += (double)rot[(uint64_t)i * d + j] * (double)c[j];
        }
        v /= n_o;
        bits[i] = (unsigned char)(v >= 0.0);
        double xb = (v >= 0.0 ? 1.0 : -1.0) / sd;
        alpha += xb * v;
        xc += xb * cr;
        pc += bits[i];
    }
    out[0] = n_o;
    out[1] = alpha;
    out[2] = xc;
    out[3] = n_o * n_o + 2.0 * n_o * xc / alpha;
    out[4] = -2.0 * n_o / alpha;
    out[5] = 2.0 * n_o * sqrt((1.0 - alpha * alpha) / (alpha * alpha)) / sqrt((double)d - 1.0);
    out[6] = pc;
    free(u);
}

/* The unquantized estimate (fp64) of ||q_r - o_r||^2 from the definitions of
 * Eq. (2)-(4): dist_c + n_o^2 - 2 n_o ||q_r-c|| <o_bar,q>/<o_bar,o>, with q
 * the query normalized about c.  Used by the unbiasedness pins.  out[0] =
 * estimate, out[1] = the bound f_err*||q_r-c|| (R7), out[2] = exact. */
void orc_estimate_unquantized_f64(const float *rot, uint32_t d, const float *c, const float *o, const float *q,
                                  double *out) {
    unsigned char *bits = (unsigned char *)malloc(d);
    double f[7];
    orc_quantize_edge(rot, d, c, o, bits, f);
    double n_o = f[0], alpha = f[1];
    double dist_c = orc_sqdist_f64(q, c, d);
    double nq = sqrt(dist_c);
    double sd = sqrt((double)d);
    double ip = 0.0; /* <x_bar, P^-1 q> with q = (q_r - c)/||q_r - c|| */
    if (nq > 0.0 && n_o > 0.0) {
        for (uint32_t i = 0; i < d; ++i) {
            double s = 0.0;
            for (uint32_t j = 0; j < d; ++j)
                s += (double)rot[(uint64_t)i * d + j] * (((double)q[j] - (double)c[j]) / nq);
            ip += (bits[i] ? 1.0 : -1.0) / sd * s;
        }
    }
    out[0] = (n_o > 0.0) ? dist_c + n_o * n_o - 2.0 * n_o * nq * ip / alpha : dist_c;
    out[1] = f[5] * nq;
    out[2] = orc_sqdist_f64(q, o, d);
    free(bits);
}

/* Exact kNN by brute force in fp64, ties by id (R4).  data: n x d. */
void orc_bruteforce(const float *data, uint64_t n, uint32_t d, const float *q, uint32_t k, uint32_t *ids,
                    double *dists) {
    for (uint32_t t = 0; t < k; ++t) { ids[t] = ORC_NO_ID; dists[t] = INFINITY; }
    for (uint64_t v = 0; v < n; ++v) {
        double x = orc_sqdist_f64(q, data + v * d, d);
        /* insertion into the sorted k-list */
        if (!(x < dists[k - 1] || (x == dists[k - 1] && (uint32_t)v < ids[k - 1]))) continue;
        int32_t p = (int32_t)k - 1;
        while (p > 0 && (x < dists[p - 1] || (x == dists[p - 1] && (uint32_t)v < ids[p - 1]))) {
            dists[p] = dists[p - 1];
            ids[p] = ids[p - 1];
            --p;
        }
        dists[p] = x;
        ids[p] = (uint32_t)v;
    }
}

/* ------------------------------------------------------------------ */
/* Fp32 query side, in the device's precision and order                */
/* ------------------------------------------------------------------ */

/* q'_i = P^-1 q (Eq. (4)) in fp32: per chunk of 32 columns an fmaf chain
 * started from 0, the chunk sums added to a total (from 0) in column order. */
void orc_rotate_f32(const float *rot, uint32_t d, const float *q, float *y) {
    for (uint32_t i = 0; i < d; ++i) {
        const float *row = rot + (uint64_t)i * d;
        float total = 0.0f;
        for (uint32_t c = 0; c < d; c += 32) {
            float s = 0.0f;
            for (uint32_t j = c; j < c + 32 && j < d; ++j) s = fmaf(row[j], q[j], s);
            total = total + s;
        }
        y[i] = total;
    }
}

/* The fast JLT in fp32, the order both sides take: per round the sign
 * flip (exact), the transform's stages h = 1, 2, 4, ... each replacing
 * (y_j, y_j+h) by (y_j + y_j+h, y_j - y_j+h), then y_i * fl(1/sqrt(d)). */
void orc_fjlt_f32(const float *signs, uint32_t d, const float *x, float *y) {
    const float c = 1.0f / sqrtf((float)d);
    for (uint32_t i = 0; i < d; ++i) y[i] = x[i];
    for (uint32_t r = 0; r < 3; ++r) {
        for (uint32_t i = 0; i < d; ++i) y[i] = y[i] * signs[r * d + i];
        for (uint32_t h = 1; h < d; h <<= 1)
            for (uint32_t i = 0; i < d; i += 2 * h)
                for (uint32_t j = i; j < i + h; ++j) {
                    const float a = y[j], b = y[j + h];
                    y[j] = a + b;
                    y[j + h] = a - b;
                }
        for (uint32_t i = 0; i < d; ++i) y[i] = y[i] * c;
    }
}

/* q' of the query side: the fast JLT for a version-2 index, else P^-1 q. */
static void rotate_query(const orc_index *ix, const float *q, float *qrot) {
    if (ix->fjlt) orc_fjlt_f32(ix->signs, ix->d, q, qrot);
    else orc_rotate_f32(ix->rot, ix->d, q, qrot);
}

/* R1: v_l = min q', v_r = max q', delta = (v_r - v_l)/15,
 * qbar_i = min(15, trunc((q'_i - v_l) * (15/(v_r - v_l)) + 0.5)).  */
void orc_quantize_query(const float *qr, uint32_t d, unsigned char *qbar, float *vl_out, float *delta_out,
                        int32_t *sq_out) {
    float vl = qr[0], vr = qr[0];
    for (uint32_t i = 1; i < d; ++i) {
        if (qr[i] < vl) vl = qr[i];
        if (qr[i] > vr) vr = qr[i];
    }
    float range = vr - vl;
    float delta = 0.0f, inv = 0.0f;
    if (range > 0.0f) {
        delta = range / 15.0f;
        inv = 15.0f / range;
    }
    int32_t sq = 0;
    for (uint32_t i = 0; i < d; ++i) {
        int32_t t = 0;
        if (range > 0.0f) {
            float x = qr[i] - vl;
            x = x * inv;
            x = x + 0.5f;
            t = (int32_t)x;
            if (t > 15) t = 15;
        }
        qbar[i] = (unsigned char)t;
        sq += t;
    }
    *vl_out = vl;
    *delta_out = delta;
    *sq_out = sq;
}

float orc_exact_dist_f32(const float *q, const float *x, uint32_t d) {
    float part[32];
    uint32_t chunks = d / 4u;
    for (uint32_t l = 0; l < 32; ++l) {
        float acc = 0.0f;
        for (uint32_t c = l; c < chunks; c += 32) {
            for (uint32_t t = 0; t < 4; ++t) {
                float df = q[4 * c + t] - x[4 * c + t];
                acc = fmaf(df, df, acc);
            }
        }
        part[l] = acc;
    }
    for (uint32_t off = 16; off >= 1; off >>= 1) {
        float nxt[32];
        for (uint32_t l = 0; l < 32; ++l) nxt[l] = part[l] + part[l ^ off];
        memcpy(part, nxt, sizeof(part));
    }
    return part[0];
}

/* R16: q / ||q|| in fp32.  s = ||q||^2 in the exact distance's order (32
 * partial sums over float4 chunks l, l+32, ..., fmaf(x, x, acc), then the
 * pairwise tree over partials l and l^16, ^8, ^4, ^2, ^1); each coordinate is
 * then divided by fl(sqrt(s)).  A query with s = 0 (or s not finite) is
 * left as it is. */
void orc_normalize_f32(const float *q, uint32_t d, float *out) {
    float part[32];
    uint32_t chunks = d / 4u;
    for (uint32_t l = 0; l < 32; ++l) {
        float acc = 0.0f;
        for (uint32_t c = l; c < chunks; c += 32)
            for (uint32_t t = 0; t < 4; ++t) acc = fmaf(q[4 * c + t], q[4 * c + t], acc);
        part[l] = acc;
    }
    for (uint32_t off = 16; off >= 1; off >>= 1) {
        float nxt[32];
        for (uint32_t l = 0; l < 32; ++l) nxt[l] = part[l] + part[l ^ off];
        memcpy(part, nxt, sizeof(part));
    }
    const float s = part[0];
    if (s > 0.0f && s <= 3.40282347e38f) {
        const float r = sqrtf(s);
        for (uint32_t i = 0; i < d; ++i) out[i] = q[i] / r;
    } else {
        for (uint32_t i = 0; i < d; ++i) out[i] = q[i];
    }
}

/* The query every search step sees: normalized on a cosine index (R16),
 * else the caller's vector.  Returns a buffer to free, or NULL. */
static float *query_for(const orc_index *ix, const float **q) {
    if (ix->metric != 1u) return NULL;
    float *qn = (float *)malloc(sizeof(float) * ix->d);
    orc_normalize_f32(*q, ix->d, qn);
    *q = qn;
    return qn;
}

typedef struct {
    const float *q;        /* raw query, d */
    unsigned char *qbar;   /* quantized rotated query, d */
    float vl, delta, inv_sqrt_d;
    int32_t sq;
} orc_query;

/* The estimate for neighbour j of centre v (Sec. 3.1.1 with R1).
 * S = sum_i b_i qbar_i (brute force over the dimensions),
 * ip = <x_bar, v_l + delta*qbar> = (delta (2S - Sq) + v_l (2pc - D))/sqrt(D). */
static void estimate(const orc_index *ix, const orc_query *qq, uint32_t v, uint32_t j, float dist_c, float eps0,
                     int32_t *S_out, float *est_out, float *key_out) {
    int32_t S = 0;
    for (uint32_t i = 0; i < ix->d; ++i) S += code_bit(ix, v, j, i) * (int32_t)qq->qbar[i];
    int32_t pc = (int32_t)popc_stored(ix, v, j);
    float a = (float)(2 * S - qq->sq);
    float b = qq->vl * (float)(2 * pc - (int32_t)ix->d);
    float ip = fmaf(qq->delta, a, b) * qq->inv_sqrt_d;
    float est = fmaf(fac(ix, v, 1, j), ip, fac(ix, v, 0, j) + dist_c);
    float bound = fac(ix, v, 2, j) * sqrtf(dist_c);
    *S_out = S;
    *est_out = est;
    *key_out = est - eps0 * bound;
}

static void prepare_query(const orc_index *ix, const float *q, orc_query *qq, float *qrot) {
    rotate_query(ix, q, qrot);
    qq->q = q;
    orc_quantize_query(qrot, ix->d, qq->qbar, &qq->vl, &qq->delta, &qq->sq);
    qq->inv_sqrt_d = 1.0f / sqrtf((float)ix->d);
}

/* Test hook: the estimate (S, est, key) for every neighbour of vertex v. */
int orc_estimate_block(const orc_index *ix, const float *q, uint32_t v, float eps0, int32_t *S, float *est,
                       float *key, float *dist_c_out) {
    if (v >= ix->n) return ORC_ERR_ARG;
    float *qn = query_for(ix, &q);
    orc_query qq;
    float *qrot = (float *)malloc(sizeof(float) * ix->d);
    qq.qbar = (unsigned char *)malloc(ix->d);
    prepare_query(ix, q, &qq, qrot);
    float dist_c = orc_exact_dist_f32(q, orc_raw(ix, v), ix->d);
    for (uint32_t j = 0; j < ix->R; ++j) estimate(ix, &qq, v, j, dist_c, eps0, &S[j], &est[j], &key[j]);
    *dist_c_out = dist_c;
    free(qrot);
    free(qq.qbar);
    free(qn);
    return ORC_OK;
}

/* Test hook: the prepared query (q', qbar, v_l, delta, Sq). */
void orc_prepare_query(const orc_index *ix, const float *q, float *qrot, unsigned char *qbar, float *vl,
                       float *delta, int32_t *sq) {
    float *qn = query_for(ix, &q);
    rotate_query(ix, q, qrot);
    orc_quantize_query(qrot, ix->d, qbar, vl, delta, sq);
    free(qn);
}

/* ------------------------------------------------------------------ */
/* Learned early stop: 16 search-state features -> MLP 16-64-64-1      */
/* (not in the paper).  Parameters, flat fp32: W1[64][16] b1[64]        */
/* W2[64][64] b2[64] W3[64] b3.                                         */
/* ------------------------------------------------------------------ */

#define MLP_IN 16
#define MLP_H 64
#define MLP_NPARAM (MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)

/* fp32 forward in the device's order: each hidden neuron is an fmaf chain
 * over its inputs in order starting from its bias; the output sums
 * p_l = fmaf(W3[l+32], h[l+32], W3[l]*h[l]) with the same pairwise tree as
 * the exact distance, then adds b3. */
float orc_mlp_logit_f32(const float *P, const float *x) {
    const float *W1 = P, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const float *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    float h1[MLP_H], h2[MLP_H];
    for (int o = 0; o < MLP_H; ++o) {
        float a = b1[o];
        for (int i = 0; i < MLP_IN; ++i) a = fmaf(W1[o * MLP_IN + i], x[i], a);
        h1[o] = a > 0.0f ? a : 0.0f;
    }
    for (int o = 0; o < MLP_H; ++o) {
        float a = b2[o];
        for (int i = 0; i < MLP_H; ++i) a = fmaf(W2[o * MLP_H + i], h1[i], a);
        h2[o] = a > 0.0f ? a : 0.0f;
    }
    float part[32];
    for (int l = 0; l < 32; ++l) part[l] = fmaf(W3[l + 32], h2[l + 32], W3[l] * h2[l]);
    for (int off = 16; off >= 1; off >>= 1) {
        float nxt[32];
        for (int l = 0; l < 32; ++l) nxt[l] = part[l] + part[l ^ off];
        memcpy(part, nxt, sizeof(part));
    }
    return part[0] + b3[0];
}

/* fp64 forward + binary cross-entropy loss + gradient for a batch.
 * x: nb x 16, y: nb labels in {0,1}, w: nb sample weights.
 * loss = sum_b w_b * BCE(sigmoid(z_b), y_b) / sum_b w_b.  grad: MLP_NPARAM. */
double orc_mlp_loss_grad_f64(const double *P, const float *x, const float *y, const float *w, int nb,
                             double *grad) {
    const double *W1 = P, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const double *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    double *gW1 = grad, *gb1 = gW1 + MLP_H * MLP_IN, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H;
    double *gW3 = gb2 + MLP_H, *gb3 = gW3 + MLP_H;
    memset(grad, 0, sizeof(double) * MLP_NPARAM);
    double wsum = 0.0, loss = 0.0;
    for (int b = 0; b < nb; ++b) wsum += w[b];
    if (wsum <= 0.0) return 0.0;
    for (int b = 0; b < nb; ++b) {
        const float *xb = x + (size_t)b * MLP_IN;
        double a1[MLP_H], h1[MLP_H], a2[MLP_H], h2[MLP_H];
        for (int o = 0; o < MLP_H; ++o) {
            double a = b1[o];
            for (int i = 0; i < MLP_IN; ++i) a += W1[o * MLP_IN + i] * xb[i];
            a1[o] = a;
            h1[o] = a > 0.0 ? a : 0.0;
        }
        for (int o = 0; o < MLP_H; ++o) {
            double a = b2[o];
            for (int i = 0; i < MLP_H; ++i) a += W2[o * MLP_H + i] * h1[i];
            a2[o] = a;
            h2[o] = a > 0.0 ? a : 0.0;
        }
        double z = b3[0];
        for (int i = 0; i < MLP_H; ++i) z += W3[i] * h2[i];
        /* BCE with logits: log(1+e^z) - y z, computed stably */
        double lz = z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
        double wb = w[b] / wsum;
        loss += wb * (lz - y[b] * z);
        double s = 1.0 / (1.0 + exp(-z));
        double dz = wb * (s - y[b]);
        gb3[0] += dz;
        double d2[MLP_H], d1[MLP_H];
        for (int i = 0; i < MLP_H; ++i) {
            gW3[i] += dz * h2[i];
            d2[i] = a2[i] > 0.0 ? dz * W3[i] : 0.0;
        }
        for (int o = 0; o < MLP_H; ++o) {
            gb2[o] += d2[o];
            for (int i = 0; i < MLP_H; ++i) gW2[o * MLP_H + i] += d2[o] * h1[i];
        }
        for (int i = 0; i < MLP_H; ++i) {
            double s1 = 0.0;
            for (int o = 0; o < MLP_H; ++o) s1 += W2[o * MLP_H + i] * d2[o];
            d1[i] = a1[i] > 0.0 ? s1 : 0.0;
        }
        for (int o = 0; o < MLP_H; ++o) {
            gb1[o] += d1[o];
            for (int i = 0; i < MLP_IN; ++i) gW1[o * MLP_IN + i] += d1[o] * xb[i];
        }
    }
    return loss;
}

/* One Adam step (Kingma & Ba 2015) in fp64:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps). */
void orc_adam_step_f64(double *p, double *m, double *v, const double *g, int n, int t, double lr, double b1,
                       double b2, double eps) {
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 (Querying) with multiple estimated distances (Sec.      */
/* 3.1.2) and implicit re-ranking, plus the learned stop.               */
/* ------------------------------------------------------------------ */

typedef struct {
    float key;
    uint32_t id;
    uint32_t fresh; /* merge bookkeeping only: 1 for this hop's candidates */
} orc_entry;

static int entry_less(orc_entry a, orc_entry b) { return a.key < b.key || (a.key == b.key && a.id < b.id); }

static int entry_cmp(const void *pa, const void *pb) {
    orc_entry a = *(const orc_entry *)pa, b = *(const orc_entry *)pb;
    if (entry_less(a, b)) return -1;
    if (entry_less(b, a)) return 1;
    return 0;
}

static float clampf8(float x) { return x < -8.0f ? -8.0f : (x > 8.0f ? 8.0f : x); }

typedef struct {
    /* search state the features read */
    int hops, ef, k, R, last_improve_hop, inserted_last;
    float ema_improve, ema_insert, dist_c;
} orc_stop_state;

/* The 16 features of the learned stop, all fp32 ratios (IEEE +,-,*,/ only,
 * so that both sides compute the same bits). */
static void stop_features(const orc_stop_state *s, const orc_entry *pool, int m, const int *visited_flags,
                          const orc_entry *res, int nres, float *f) {
    float rk = res[nres - 1].key;
    float den = rk > 1e-20f ? rk : 1e-20f;
    float fef = (float)s->ef;
    int u = 0, near1 = 0, near2 = 0; /* unvisited; of them with key <= rk, <= 1.25 rk */
    float fu = 0.0f;
    const float rk2 = 1.25f * rk;
    for (int i = m - 1; i >= 0; --i)
        if (!visited_flags[i]) {
            ++u;
            fu = pool[i].key;
            near1 += pool[i].key <= rk;
            near2 += pool[i].key <= rk2;
        }
    float since = (float)(s->hops - s->last_improve_hop);
    /* ratios as products with four reciprocals */
    const float inv_ef = 1.0f / fef, inv_den = 1.0f / den, inv_k = 1.0f / (float)s->k;
    const float inv_h1 = 1.0f / ((float)s->hops + 1.0f);
    f[0] = (float)s->hops * inv_ef;
    f[1] = since * inv_ef;
    f[2] = (float)u * inv_ef;
    f[3] = (float)m * inv_ef;
    f[4] = res[0].key * inv_den;
    f[5] = u > 0 ? fu * inv_den : 0.0f;
    f[6] = s->dist_c * inv_den;
    f[7] = (float)s->inserted_last * (1.0f / (float)s->R);
    f[8] = (float)s->k * inv_ef;
    f[9] = s->ema_improve;
    f[10] = s->ema_insert;
    f[11] = (float)near1 * inv_k;
    f[12] = (float)near2 * inv_k;
    f[13] = since * inv_h1;
    f[14] = s->dist_c <= rk ? 1.0f : 0.0f;
    f[15] = (float)s->k * 0.01f;
    for (int i = 0; i < MLP_IN; ++i) f[i] = clampf8(f[i]);
}

/*
 * Search one query.  ids/dists: k outputs sorted by (dist, id), padded with
 * (ORC_NO_ID, +inf).  stats[0] = hops, stats[1] = status flags.
 * mlp (optional): learned-stop parameters; evaluated after every
 * stop_every-th expansion once the result holds k entries; stop when the
 * logit exceeds stop_logit.
 * trace (optional): at every evaluation point append the 16 features and,
 * if gt (k ids) is given, the number of gt ids in the current result;
 * trace_feat: cap x 16, trace_hit: cap, *trace_n in/out.
 * path (optional): the ids of the first path_cap expanded vertices, in order.
 */
/* Optional record of the beam after every expansion's cut to ef (test
 * export, no effect on the search): for hop h < cap, m[h] entries at
 * ids/keys/visited[h*ef ..], in beam order. */
typedef struct {
    uint32_t cap;
    int32_t *m;
    uint32_t *ids;
    float *keys;
    unsigned char *visited;
} orc_beam_record;

static int search_core(const orc_index *ix, const float *q, uint32_t k, uint32_t ef, float eps0,
                       int multi_estimate, uint32_t hop_cap, const float *mlp, float stop_logit,
                       uint32_t stop_every, uint32_t *ids, float *dists, uint32_t *stats, const uint32_t *gt,
                       float *trace_feat, int32_t *trace_hit, int32_t trace_cap, int32_t *trace_n, uint32_t *path,
                       uint32_t path_cap, const orc_beam_record *rec) {
    if (!ix || !q || k == 0 || ef < k || !ids || !dists || !stats) return ORC_ERR_ARG;
    const uint32_t d = ix->d, R = ix->R;
    float *qn = query_for(ix, &q);
    orc_query qq;
    float *qrot = (float *)malloc(sizeof(float) * d);
    qq.qbar = (unsigned char *)malloc(d);
    prepare_query(ix, q, &qq, qrot);

    unsigned char *visited = (unsigned char *)calloc(ix->n, 1);
    size_t cap = (size_t)ef + R;
    orc_entry *pool = (orc_entry *)malloc(sizeof(orc_entry) * cap);
    int *vflag = (int *)malloc(sizeof(int) * cap);
    orc_entry *res = (orc_entry *)malloc(sizeof(orc_entry) * (k + 1)); /* (dist, id) */
    orc_entry *cand = (orc_entry *)malloc(sizeof(orc_entry) * R);
    int m = 0, nres = 0;
    uint32_t status = 0;
    int32_t tn = 0;

    /* line 1: the beam and NN start from the entry point (R8) */
    pool[0].key = orc_exact_dist_f32(q, orc_raw(ix, ix->entry), d);
    pool[0].id = ix->entry;
    pool[0].fresh = 0;
    m = 1;

    orc_stop_state st;
    memset(&st, 0, sizeof(st));
    st.ef = (int)ef; st.k = (int)k; st.R = (int)R;
    uint32_t hops = 0;
    for (;;) {
        /* line 2-3: the unvisited entry with the smallest key */
        int sel = -1;
        for (int i = 0; i < m; ++i)
            if (!visited[pool[i].id]) { sel = i; break; }
        if (sel < 0) break;
        if (hops >= hop_cap) { status |= ORC_STATUS_CAPACITY; break; } /* R6 */
        uint32_t p = pool[sel].id;
        visited[p] = 1;
        if (path && hops < path_cap) path[hops] = p;
        ++hops;
        /* line 4: exact distance from the raw vector in p's block; update NN
         * (implicit re-ranking, Sec. 3.1.2) */
        float dist_c = orc_exact_dist_f32(q, orc_raw(ix, p), d);
        int improved = 0;
        orc_entry e = {dist_c, p};
        if (nres < (int)k || entry_less(e, res[nres - 1])) {
            int pos = nres < (int)k ? nres : (int)k - 1;
            if (nres < (int)k) ++nres;
            while (pos > 0 && entry_less(e, res[pos - 1])) { res[pos] = res[pos - 1]; --pos; }
            res[pos] = e;
            improved = 1;
        }
        /* line 5: estimates for all neighbours of p from the same block */
        int nc = 0;
        for (uint32_t j = 0; j < R; ++j) {
            uint32_t id = nbr(ix, p, j);
            if (id == ORC_NO_ID) continue; /* an empty slot (R17) */
            if (visited[id]) continue;     /* line 6: unvisited neighbours only */
            int32_t S;
            float est, key;
            estimate(ix, &qq, p, j, dist_c, eps0, &S, &est, &key);
            if (!multi_estimate) { /* ablation w/o ME: keep the first estimate */
                int in = 0;
                for (int i = 0; i < m && !in; ++i) in = pool[i].id == id;
                for (int i = 0; i < nc && !in; ++i) in = cand[i].id == id;
                if (in) continue;
            }
            cand[nc].key = key;
            cand[nc].id = id;
            cand[nc].fresh = 1;
            ++nc;
        }
        /* line 6: append (every copy, Sec. 3.1.2) and cut the beam to ef (R5) */
        for (int i = 0; i < m; ++i) pool[i].fresh = 0;
        for (int i = 0; i < nc; ++i) {
            int dup = 0; /* an identical (key, id) is stored once */
            for (int t = 0; t < m && !dup; ++t) dup = entry_cmp(&pool[t], &cand[i]) == 0;
            if (dup) continue;
            pool[m] = cand[i];
            pool[m].fresh = 1;
            ++m;
        }
        qsort(pool, (size_t)m, sizeof(orc_entry), entry_cmp);
        int w = 0;
        for (int i = 0; i < m; ++i)
            if (w == 0 || entry_cmp(&pool[i], &pool[w - 1]) != 0) pool[w++] = pool[i];
        m = w < (int)ef ? w : (int)ef;
        int inserted = 0; /* this hop's candidates that survive the cut */
        for (int i = 0; i < m; ++i) inserted += (int)pool[i].fresh;
        if (rec && hops - 1 < rec->cap) {
            const size_t h = hops - 1;
            rec->m[h] = m;
            for (int i = 0; i < m; ++i) {
                rec->ids[h * ef + i] = pool[i].id;
                rec->keys[h * ef + i] = pool[i].key;
                rec->visited[h * ef + i] = visited[pool[i].id];
            }
        }

        st.hops = (int)hops;
        st.inserted_last = inserted;
        st.dist_c = dist_c;
        if (improved) st.last_improve_hop = (int)hops;
        st.ema_improve = 0.75f * st.ema_improve + 0.25f * (improved ? 1.0f : 0.0f);
        st.ema_insert = 0.75f * st.ema_insert + 0.25f * ((float)inserted * (1.0f / (float)R));
        if ((mlp || trace_feat) && stop_every > 0 && hops % stop_every == 0 && nres == (int)k) {
            float f[MLP_IN];
            for (int i = 0; i < m; ++i) vflag[i] = visited[pool[i].id];
            stop_features(&st, pool, m, vflag, res, nres, f);
            if (trace_feat && tn < trace_cap) {
                memcpy(trace_feat + (size_t)tn * MLP_IN, f, sizeof(f));
                if (gt && trace_hit) {
                    int hit = 0;
                    for (int a = 0; a < nres; ++a)
                        for (uint32_t b = 0; b < k; ++b) hit += res[a].id == gt[b];
                    trace_hit[tn] = hit;
                }
                ++tn;
            }
            if (mlp && orc_mlp_logit_f32(mlp, f) > stop_logit) { status |= ORC_STATUS_LEARNED_STOP; break; }
        }
    }
    /* line 8: return the NN set, sorted by (dist, id) */
    for (uint32_t t = 0; t < k; ++t) {
        if ((int)t < nres) { ids[t] = res[t].id; dists[t] = res[t].key; }
        else { ids[t] = ORC_NO_ID; dists[t] = INFINITY; }
    }
    stats[0] = hops;
    stats[1] = status;
    if (trace_n) *trace_n = tn;
    free(qrot); free(qq.qbar); free(visited); free(pool); free(vflag); free(res); free(cand);
    free(qn);
    return ORC_OK;
}

int orc_search(const orc_index *ix, const float *q, uint32_t k, uint32_t ef, float eps0, int multi_estimate,
               uint32_t hop_cap, const float *mlp, float stop_logit, uint32_t stop_every, uint32_t *ids,
               float *dists, uint32_t *stats, const uint32_t *gt, float *trace_feat, int32_t *trace_hit,
               int32_t trace_cap, int32_t *trace_n, uint32_t *path, uint32_t path_cap) {
    return search_core(ix, q, k, ef, eps0, multi_estimate, hop_cap, mlp, stop_logit, stop_every, ids, dists, stats,
                       gt, trace_feat, trace_hit, trace_cap, trace_n, path, path_cap, NULL);
}

/* orc_search (eps0 = 0, multiple estimates, no learned stop) that also
 * records the beam after each of the first rec_cap expansions: rec_m[h]
 * entries (ids, keys, visited flags) at offset h*ef of the rec arrays. */
int orc_search_record(const orc_index *ix, const float *q, uint32_t k, uint32_t ef, uint32_t hop_cap,
                      uint32_t *ids, float *dists, uint32_t *stats, uint32_t rec_cap, int32_t *rec_m,
                      uint32_t *rec_ids, float *rec_keys, unsigned char *rec_visited) {
    if (rec_cap > 0 && (!rec_m || !rec_ids || !rec_keys || !rec_visited)) return ORC_ERR_ARG;
    orc_beam_record rec = {rec_cap, rec_m, rec_ids, rec_keys, rec_visited};
    return search_core(ix, q, k, ef, 0.0f, 1, hop_cap, NULL, 0.0f, 1, ids, dists, stats, NULL, NULL, NULL, 0,
                       NULL, NULL, 0, &rec);
}

/* ------------------------------------------------------------------ */
/* Index construction: the "adjust G" step of Algorithm 2 (Sec. 3.2)  */
/* ------------------------------------------------------------------ */

/* An edge candidate of a vertex u: (exact distance to u, id).  Ordered by
 * (dist, id) (R4); distances are orc_exact_dist_f32, symmetric in its two
 * arguments (the differences are negated exactly). */
typedef struct {
    float d;
    uint32_t id;
} orc_cand;

static int cand_less(orc_cand a, orc_cand b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }

static void sort_by_dist(orc_cand *a, int n) { /* insertion sort: plain and stable */
    for (int i = 1; i < n; ++i) {
        orc_cand x = a[i];
        int j = i;
        while (j > 0 && cand_less(x, a[j - 1])) { a[j] = a[j - 1]; --j; }
        a[j] = x;
    }
}

/* Drop repeated ids (their distances are equal), keep one of each. */
static int unique_ids(orc_cand *a, int n) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        int seen = 0;
        for (int j = 0; j < m && !seen; ++j) seen = a[j].id == a[i].id;
        if (!seen) a[m++] = a[i];
    }
    return m;
}

static float vdist(const float *data, uint32_t d, uint32_t a, uint32_t b) {
    return orc_exact_dist_f32(data + (uint64_t)a * d, data + (uint64_t)b * d, d);
}

/* NSG's occlusion rule (Sec. 3.2.1): walk the candidates nearest first and
 * keep c unless an already kept w is nearer to c than u is (dist(w, c) <
 * dist(u, c)); stop at R kept.  `c` sorted by (dist, id). */
static int nsg_prune(const float *data, uint32_t d, const orc_cand *c, int nc, int R, orc_cand *kept) {
    int nk = 0;
    for (int i = 0; i < nc && nk < R; ++i) {
        int occluded = 0;
        for (int j = 0; j < nk && !occluded; ++j) occluded = vdist(data, d, kept[j].id, c[i].id) < c[i].d;
        if (!occluded) kept[nk++] = c[i];
    }
    return nk;
}

/* The adaptive angle rule (Sec. 3.2.2), reading R11.  Every extra candidate
 * c gets the largest cosine, at u, between c and a candidate w before it in
 * (dist, id) order among kept and extra together: cos = (|uw|^2 + |uc|^2 -
 * |wc|^2) / (2 |uw| |uc|) in fp32 (1 when a length is 0; -2 when nothing is
 * before c).  Raising the angle threshold theta drops every c whose score
 * is above cos(theta); the largest theta that leaves `need` candidates
 * keeps exactly those scoring at most the need-th smallest score, and the
 * `need` nearest of them are added.  Returns how many were added to out. */
static int angle_supplement(const float *data, uint32_t d, const orc_cand *kept, int nk, const orc_cand *extra,
                            int ne, int need, orc_cand *out) {
    if (need <= 0 || ne == 0) return 0;
    orc_cand *all = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)(nk + ne));
    float *score = (float *)malloc(sizeof(float) * (size_t)ne);
    float *sorted = (float *)malloc(sizeof(float) * (size_t)ne);
    memcpy(all, kept, sizeof(orc_cand) * (size_t)nk);
    memcpy(all + nk, extra, sizeof(orc_cand) * (size_t)ne);
    sort_by_dist(all, nk + ne);
    for (int e = 0; e < ne; ++e) {
        float best = -2.0f;
        for (int j = 0; j < nk + ne && cand_less(all[j], extra[e]); ++j) {
            float dwc = vdist(data, d, all[j].id, extra[e].id);
            float den = 2.0f * sqrtf(all[j].d) * sqrtf(extra[e].d);
            float cs = den > 0.0f ? (all[j].d + extra[e].d - dwc) / den : 1.0f;
            if (cs > best) best = cs;
        }
        score[e] = best;
        sorted[e] = best;
    }
    int take = need < ne ? need : ne;
    for (int i = 1; i < ne; ++i) { /* ascending scores */
        float x = sorted[i];
        int j = i;
        while (j > 0 && x < sorted[j - 1]) { sorted[j] = sorted[j - 1]; --j; }
        sorted[j] = x;
    }
    float thr = sorted[take - 1];
    int no = 0;
    for (int e = 0; e < ne && no < take; ++e) /* extra is in (dist, id) order */
        if (score[e] <= thr) out[no++] = extra[e];
    free(all); free(score); free(sorted);
    return no;
}

/* The own candidates of u: ids from its candidate list (invalid ids, u
 * itself and repeats dropped) with their distances, sorted by (dist, id). */
static int own_candidates(const float *data, uint64_t n, uint32_t d, const uint32_t *cand, uint32_t L, uint32_t u,
                          orc_cand *c) {
    int m = 0;
    for (uint32_t t = 0; t < L; ++t) {
        uint32_t v = cand[(uint64_t)u * L + t];
        if (v == ORC_NO_ID || v >= n || v == u) continue;
        c[m].id = v;
        c[m].d = vdist(data, d, u, v);
        ++m;
    }
    m = unique_ids(c, m);
    sort_by_dist(c, m);
    return m;
}

/* "Adjust G" of Algorithm 2 for every vertex, readings R11 (with regular =
 * 0, the "w/o GR" ablation, R17: steps (1)-(2) only): (1) NSG-prune
 * the vertex's own candidates to at most R' = min(R, n-1) edges; (2) offer
 * every kept edge u -> v to v as the reverse candidate (u, dist) and prune
 * v's kept edges plus its reverse candidates again; (3) a vertex left with
 * fewer than R' edges is supplemented by the adaptive angle rule from its
 * own and reverse candidates not yet kept, the nearest 2R' (d >= 512) or
 * 3R' of them.  Writes each vertex's list sorted by (dist, id) to
 * out[u*R ...] (ORC_NO_ID after its count) and its count to counts[u].
 * The builder's random fill of a list still short and its reachability
 * repair come after this and are not part of it. */
int orc_adjust_graph(const float *data, uint64_t n, uint32_t d, const uint32_t *cand, uint32_t L, uint32_t R,
                     int regular, uint32_t *out, uint32_t *counts) {
    if (!data || !cand || !out || !counts || n < 2 || R == 0 || L == 0 || d == 0 || d % 4 != 0) return ORC_ERR_ARG;
    const int Rr = (int)(R < n - 1 ? R : n - 1);
    orc_cand *k1 = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)n * (size_t)Rr);
    int *n1 = (int *)calloc(n, sizeof(int));
    int *indeg = (int *)calloc(n, sizeof(int));
    orc_cand *c = (orc_cand *)malloc(sizeof(orc_cand) * L);
    for (uint32_t u = 0; u < n; ++u) { /* (1) */
        int m = own_candidates(data, n, d, cand, L, u, c);
        n1[u] = nsg_prune(data, d, c, m, Rr, k1 + (size_t)u * Rr);
        for (int j = 0; j < n1[u]; ++j) indeg[k1[(size_t)u * Rr + j].id]++;
    }
    uint64_t *roff = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
    for (uint64_t v = 0; v < n; ++v) roff[v + 1] = roff[v] + (uint64_t)indeg[v];
    orc_cand *rev = (orc_cand *)malloc(sizeof(orc_cand) * (roff[n] ? roff[n] : 1));
    uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * n);
    memcpy(fill, roff, sizeof(uint64_t) * n);
    for (uint32_t u = 0; u < n; ++u) /* (2) reverse candidates */
        for (int j = 0; j < n1[u]; ++j) {
            orc_cand e = k1[(size_t)u * Rr + j];
            rev[fill[e.id]].id = u;
            rev[fill[e.id]].d = e.d;
            fill[e.id]++;
        }
    for (uint32_t u = 0; u < n; ++u) {
        const int nr = (int)(roff[u + 1] - roff[u]);
        orc_cand *pool = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)(n1[u] + nr + L));
        memcpy(pool, k1 + (size_t)u * Rr, sizeof(orc_cand) * (size_t)n1[u]);
        memcpy(pool + n1[u], rev + roff[u], sizeof(orc_cand) * (size_t)nr);
        int np = unique_ids(pool, n1[u] + nr);
        sort_by_dist(pool, np);
        orc_cand *k2 = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)Rr);
        int nk = nsg_prune(data, d, pool, np, Rr, k2);
        if (regular && nk < Rr) { /* (3) */
            int m = own_candidates(data, n, d, cand, L, u, pool);
            memcpy(pool + m, rev + roff[u], sizeof(orc_cand) * (size_t)nr);
            int na = unique_ids(pool, m + nr);
            int ne = 0;
            for (int i = 0; i < na; ++i) {
                int have = 0;
                for (int j = 0; j < nk && !have; ++j) have = k2[j].id == pool[i].id;
                if (!have) pool[ne++] = pool[i];
            }
            sort_by_dist(pool, ne);
            int cap = d >= 512 ? 2 * Rr : 3 * Rr;
            if (ne > cap) ne = cap;
            orc_cand *sup = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)(ne ? ne : 1));
            int ns = angle_supplement(data, d, k2, nk, pool, ne, Rr - nk, sup);
            for (int i = 0; i < ns; ++i) k2[nk++] = sup[i];
            sort_by_dist(k2, nk);
            free(sup);
        }
        for (int t = 0; t < (int)R; ++t) out[(uint64_t)u * R + t] = t < nk ? k2[t].id : ORC_NO_ID;
        counts[u] = (uint32_t)nk;
        free(pool);
        free(k2);
    }
    free(k1); free(n1); free(indeg); free(c); free(roff); free(rev); free(fill);
    return ORC_OK;
}
