/*
 * graphgen.c — seeded synthetic directed graphs, delivered as an in-edge CSR
 * (row v lists the sources u of the edges u -> v) plus out-degrees.
 *
 * This file is input tooling only: it holds none of PageRank's arithmetic.
 * Both the CPU oracle and the CUDA library consume what it produces.
 *
 * Graph families (stand-ins for the paper's SuiteSparse web/social/road
 * graphs of Section 2, which are not available here):
 *   - directed Erdos-Renyi with a fixed number of unique non-self edges and a
 *     chosen number of vertices made dangling by deleting their out-edges;
 *   - R-MAT (recursive matrix) with quadrant probabilities a, b, c, d, a random
 *     vertex relabelling, self-loops and duplicates removed;
 *   - directed configuration model with discrete power-law in/out degrees.
 *
 * Randomness: one counter-based generator, the SplitMix64 output function of
 * Steele, Lea and Flood (OOPSLA 2014): value(key, i) = mix64(key + (i+1)*gamma).
 * Every draw is addressed by (seed, stream, counter), so results do not depend
 * on thread count, platform or call order. Only integer arithmetic decides
 * which edge is drawn, so x86-64 and aarch64 builds produce identical graphs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Key of an independent stream derived from (seed, stream). */
static inline uint64_t gg_key(uint64_t seed, uint64_t stream) {
    return gg_mix64(seed * GG_GAMMA + gg_mix64(stream + GG_GAMMA));
}

/* The counter-th output of the SplitMix64 sequence whose state starts at key. */
static inline uint64_t gg_at(uint64_t key, uint64_t counter) {
    return gg_mix64(key + (counter + 1) * GG_GAMMA);
}

/* Uniform integer in [0, n) by the multiply-high method (bias < n / 2^64). */
static inline uint64_t gg_below(uint64_t x, uint64_t n) {
    return (uint64_t)(((unsigned __int128)x * n) >> 64);
}

uint64_t gg_splitmix64(uint64_t state_before, uint64_t steps) {
    /* Exposed for tests: output number `steps` (0-based) of a SplitMix64
     * generator whose state is state_before. */
    return gg_at(state_before, steps);
}

uint64_t gg_draw(uint64_t seed, uint64_t stream, uint64_t counter) {
    return gg_at(gg_key(seed, stream), counter);
}

/* ------------------------------------------------------------------------ */
/* Graph container handed to Python through an opaque pointer.              */

typedef struct gg_graph {
    int32_t n;
    int64_t nnz;
    int32_t *offsets;   /* n + 1 */
    int32_t *sources;   /* nnz, ascending within each row */
    int32_t *outdeg;    /* n */
} gg_graph;

int32_t gg_graph_n(const gg_graph *g) { return g ? g->n : -1; }
int64_t gg_graph_nnz(const gg_graph *g) { return g ? g->nnz : -1; }

void gg_graph_free(gg_graph *g) {
    if (!g) return;
    free(g->offsets);
    free(g->sources);
    free(g->outdeg);
    free(g);
}

int gg_graph_copy(const gg_graph *g, int32_t *offsets, int32_t *sources, int32_t *outdeg) {
    if (!g) return 1;
    if (offsets) memcpy(offsets, g->offsets, sizeof(int32_t) * ((size_t)g->n + 1));
    if (sources && g->nnz) memcpy(sources, g->sources, sizeof(int32_t) * (size_t)g->nnz);
    if (outdeg) memcpy(outdeg, g->outdeg, sizeof(int32_t) * (size_t)g->n);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* LSD radix sort of 64-bit keys (16-bit digits), only over significant bits. */

static int radix_sort_u64(uint64_t *keys, int64_t m, int key_bits) {
    if (m <= 1) return 0;
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m);
    if (!tmp) return 2;
    size_t *count = (size_t *)malloc(sizeof(size_t) * 65536);
    if (!count) { free(tmp); return 2; }
    uint64_t *a = keys, *b = tmp;
    int passes = (key_bits + 15) / 16;
    for (int p = 0; p < passes; p++) {
        int shift = 16 * p;
        memset(count, 0, sizeof(size_t) * 65536);
        for (int64_t i = 0; i < m; i++) count[(a[i] >> shift) & 0xFFFF]++;
        size_t s = 0;
        for (int d = 0; d < 65536; d++) { size_t c = count[d]; count[d] = s; s += c; }
        for (int64_t i = 0; i < m; i++) b[count[(a[i] >> shift) & 0xFFFF]++] = a[i];
        uint64_t *t = a; a = b; b = t;
    }
    if (a != keys) memcpy(keys, a, sizeof(uint64_t) * (size_t)m);
    free(tmp);
    free(count);
    return 0;
}

static int bits_for(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b)) b++;
    return b < 1 ? 1 : b;
}

/* Build the in-edge CSR from keys = (dst << 32) | src. Sorts, drops
 * self-loops and duplicates. Consumes (frees) keys. */
static int csr_from_keys(int32_t n, uint64_t *keys, int64_t m, gg_graph **out) {
    int key_bits = 32 + bits_for((uint64_t)(n > 0 ? n - 1 : 0));
    int rc = radix_sort_u64(keys, m, key_bits);
    if (rc) { free(keys); return rc; }
    int64_t w = 0;
    for (int64_t i = 0; i < m; i++) {
        uint64_t k = keys[i];
        uint32_t s = (uint32_t)(k & 0xFFFFFFFFu), d = (uint32_t)(k >> 32);
        if (s == d) continue;
        if (w > 0 && keys[w - 1] == k) continue;
        keys[w++] = k;
    }
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    if (!g) { free(keys); return 2; }
    g->n = n;
    g->nnz = w;
    g->offsets = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    g->sources = (int32_t *)malloc(sizeof(int32_t) * (size_t)(w > 0 ? w : 1));
    g->outdeg = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    if (!g->offsets || !g->sources || !g->outdeg) { gg_graph_free(g); free(keys); return 2; }
    for (int64_t i = 0; i < w; i++) {
        uint32_t s = (uint32_t)(keys[i] & 0xFFFFFFFFu), d = (uint32_t)(keys[i] >> 32);
        g->sources[i] = (int32_t)s;
        g->offsets[d + 1]++;
        g->outdeg[s]++;
    }
    for (int32_t v = 0; v < n; v++) g->offsets[v + 1] += g->offsets[v];
    free(keys);
    *out = g;
    return 0;
}

/* Build a graph from an explicit edge list (src[i] -> dst[i]); self-loops and
 * duplicates are dropped. Returns 1 on an out-of-range endpoint. */
int gg_from_edges(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, gg_graph **out) {
    if (n < 1 || m < 0 || !out) return 1;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    if (!keys) return 2;
    for (int64_t i = 0; i < m; i++) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) { free(keys); return 1; }
        keys[i] = ((uint64_t)(uint32_t)dst[i] << 32) | (uint32_t)src[i];
    }
    return csr_from_keys(n, keys, m, out);
}

/* ------------------------------------------------------------------------ */
/* Random relabelling: Fisher-Yates shuffle driven by stream `stream`.       */

static int32_t *random_permutation(int32_t n, uint64_t seed, uint64_t stream) {
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!perm) return NULL;
    for (int32_t i = 0; i < n; i++) perm[i] = i;
    uint64_t key = gg_key(seed, stream);
    for (int32_t i = n - 1; i > 0; i--) {
        int32_t j = (int32_t)gg_below(gg_at(key, (uint64_t)i), (uint64_t)i + 1);
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    return perm;
}

/* ------------------------------------------------------------------------ */
/* R-MAT: 2^scale vertices, edge_factor * 2^scale sampled edges. Each edge
 * descends `scale` levels; at each level a 32-bit draw picks quadrant
 * a (src bit 0, dst bit 0), b (0,1), c (1,0) or d (1,1). Two levels share one
 * 64-bit draw (high and low halves). Ids are then relabelled by a random
 * permutation (stream 2); self-loops and duplicate edges are removed. */
int gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c,
            uint64_t seed, int32_t permute, gg_graph **out) {
    if (scale < 1 || scale > 30 || edge_factor < 1 || !out) return 1;
    if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return 1;
    int32_t n = (int32_t)1 << scale;
    int64_t m = (int64_t)edge_factor << scale;
    const double two32 = 4294967296.0;
    uint64_t ta = (uint64_t)(a * two32);
    uint64_t tab = (uint64_t)((a + b) * two32);
    uint64_t tabc = (uint64_t)((a + b + c) * two32);
    uint64_t key = gg_key(seed, 1);
    int pairs = (scale + 1) / 2;
    int32_t *perm = NULL;
    if (permute) {
        perm = random_permutation(n, seed, 2);
        if (!perm) return 2;
    }
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m);
    if (!keys) { free(perm); return 2; }
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        uint32_t s = 0, d = 0;
        for (int p = 0; p < pairs; p++) {
            uint64_t x = gg_at(key, (uint64_t)e * (uint64_t)pairs + (uint64_t)p);
            for (int h = 0; h < 2; h++) {
                int level = 2 * p + h;
                if (level >= scale) break;
                uint64_t u = h == 0 ? (x >> 32) : (x & 0xFFFFFFFFu);
                uint32_t sb, db;
                if (u < ta) { sb = 0; db = 0; }
                else if (u < tab) { sb = 0; db = 1; }
                else if (u < tabc) { sb = 1; db = 0; }
                else { sb = 1; db = 1; }
                s |= sb << level;
                d |= db << level;
            }
        }
        if (perm) { s = (uint32_t)perm[s]; d = (uint32_t)perm[d]; }
        keys[e] = ((uint64_t)d << 32) | s;
    }
    free(perm);
    return csr_from_keys(n, keys, m, out);
}

/* ------------------------------------------------------------------------ */
/* Road-like grid: rows x cols vertices on a lattice, vertex (i, j) = i*cols + j.
 * Each lattice link to the right and downward neighbour exists with
 * probability p_keep (first draw of stream 4 for the link); an existing link
 * is one-way with probability p_oneway (second draw's high half), in the
 * direction given by the second draw's lowest bit, else two-way. Ids are then
 * relabelled by a random permutation (stream 5) when `permute` is set. Mean
 * out-degree 2 p_keep (2 - p_oneway), at most 4; vertices with no outgoing
 * link are dangling. */
int gg_road_grid(int32_t rows, int32_t cols, double p_keep, double p_oneway, uint64_t seed, int32_t permute,
                 gg_graph **out) {
    if (rows < 1 || cols < 1 || !out) return 1;
    if ((int64_t)rows * cols > 2147483647LL) return 1;
    if (!(p_keep >= 0.0 && p_keep <= 1.0 && p_oneway >= 0.0 && p_oneway <= 1.0)) return 1;
    const int32_t n = rows * cols;
    const double two32 = 4294967296.0;
    const uint64_t t_keep = (uint64_t)(p_keep * two32), t_one = (uint64_t)(p_oneway * two32);
    uint64_t key = gg_key(seed, 4);
    int32_t *perm = NULL;
    if (permute) {
        perm = random_permutation(n, seed, 5);
        if (!perm) return 2;
    }
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n * 4 + 8);
    if (!keys) { free(perm); return 2; }
    int64_t m = 0;
    for (int32_t i = 0; i < rows; i++) {
        for (int32_t j = 0; j < cols; j++) {
            const int32_t v = i * cols + j;
            for (int dir = 0; dir < 2; dir++) {
                int32_t w;
                if (dir == 0) { if (j + 1 >= cols) continue; w = v + 1; }
                else { if (i + 1 >= rows) continue; w = v + cols; }
                const uint64_t x = gg_at(key, 4 * (uint64_t)v + 2 * (uint64_t)dir);
                if ((x >> 32) >= t_keep) continue;
                const uint64_t y = gg_at(key, 4 * (uint64_t)v + 2 * (uint64_t)dir + 1);
                uint32_t a = (uint32_t)v, b = (uint32_t)w;
                if (perm) { a = (uint32_t)perm[a]; b = (uint32_t)perm[b]; }
                if ((y >> 32) < t_one) {
                    if (y & 1u) keys[m++] = ((uint64_t)a << 32) | b;   /* b -> a */
                    else keys[m++] = ((uint64_t)b << 32) | a;          /* a -> b */
                } else {
                    keys[m++] = ((uint64_t)b << 32) | a;
                    keys[m++] = ((uint64_t)a << 32) | b;
                }
            }
        }
    }
    free(perm);
    return csr_from_keys(n, keys, m, out);
}

/* ------------------------------------------------------------------------ */
/* Directed Erdos-Renyi: draw (src, dst) uniformly (stream 1, two draws per
 * candidate) and keep the first m_unique distinct non-self-loop edges in draw
 * order; then pick n_dangling distinct vertices (partial Fisher-Yates,
 * stream 3) and delete their out-edges. */

typedef struct { uint64_t *slot; uint64_t mask; } gg_set;

static int set_insert(gg_set *s, uint64_t k) { /* returns 1 if newly inserted; k != ~0 */
    uint64_t h = gg_mix64(k) & s->mask;
    for (;;) {
        if (s->slot[h] == ~0ULL) { s->slot[h] = k; return 1; }
        if (s->slot[h] == k) return 0;
        h = (h + 1) & s->mask;
    }
}

int gg_erdos_renyi(int32_t n, int64_t m_unique, int32_t n_dangling, uint64_t seed, gg_graph **out) {
    if (n < 2 || m_unique < 0 || n_dangling < 0 || n_dangling > n || !out) return 1;
    if ((double)m_unique > (double)n * (double)(n - 1)) return 1;
    uint64_t cap = 1;
    while (cap < (uint64_t)(m_unique * 2 + 16)) cap <<= 1;
    gg_set set;
    set.slot = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    if (!set.slot) return 2;
    memset(set.slot, 0xFF, sizeof(uint64_t) * cap);
    set.mask = cap - 1;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m_unique > 0 ? m_unique : 1));
    if (!keys) { free(set.slot); return 2; }
    uint64_t key = gg_key(seed, 1);
    int64_t got = 0;
    for (uint64_t i = 0; got < m_unique; i++) {
        uint32_t s = (uint32_t)gg_below(gg_at(key, 2 * i), (uint64_t)n);
        uint32_t d = (uint32_t)gg_below(gg_at(key, 2 * i + 1), (uint64_t)n);
        if (s == d) continue;
        uint64_t k = ((uint64_t)d << 32) | s;
        if (set_insert(&set, k)) keys[got++] = k;
    }
    free(set.slot);
    /* choose dangling vertices */
    uint8_t *dang = (uint8_t *)calloc((size_t)n, 1);
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!dang || !ids) { free(dang); free(ids); free(keys); return 2; }
    for (int32_t i = 0; i < n; i++) ids[i] = i;
    uint64_t dkey = gg_key(seed, 3);
    for (int32_t i = 0; i < n_dangling; i++) {
        int32_t j = i + (int32_t)gg_below(gg_at(dkey, (uint64_t)i), (uint64_t)(n - i));
        int32_t t = ids[i]; ids[i] = ids[j]; ids[j] = t;
        dang[ids[i]] = 1;
    }
    int64_t w = 0;
    for (int64_t i = 0; i < got; i++)
        if (!dang[keys[i] & 0xFFFFFFFFu]) keys[w++] = keys[i];
    free(dang);
    free(ids);
    return csr_from_keys(n, keys, w, out);
}

/* ------------------------------------------------------------------------ */
/* Directed configuration model. Out- and in-degrees are drawn independently
 * (streams 4 and 5) from the discrete power law P(k) ~ k^-gamma on
 * [k_min, k_max] by inverse CDF. The larger stub total is trimmed by
 * decrementing the degree of uniformly drawn vertices with positive degree
 * (stream 6) until both totals agree. In-stubs are shuffled (stream 7) and
 * matched to out-stubs in vertex order; self-loops and duplicates are then
 * removed. */
int gg_config_model(int32_t n, double gamma, int32_t k_min, int32_t k_max, uint64_t seed, gg_graph **out) {
    if (n < 2 || k_min < 1 || k_max < k_min || gamma <= 1.0 || !out) return 1;
    int32_t span = k_max - k_min + 1;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)span);
    int32_t *dout = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *din = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!cdf || !dout || !din) { free(cdf); free(dout); free(din); return 2; }
    double acc = 0.0;
    for (int32_t i = 0; i < span; i++) { acc += pow((double)(k_min + i), -gamma); cdf[i] = acc; }
    for (int32_t i = 0; i < span; i++) cdf[i] /= acc;
    cdf[span - 1] = 1.0;
    for (int side = 0; side < 2; side++) {
        int32_t *deg = side == 0 ? dout : din;
        uint64_t key = gg_key(seed, side == 0 ? 4 : 5);
        for (int32_t v = 0; v < n; v++) {
            double u = (double)(gg_at(key, (uint64_t)v) >> 11) * (1.0 / 9007199254740992.0);
            int32_t lo = 0, hi = span - 1;
            while (lo < hi) { int32_t mid = (lo + hi) / 2; if (cdf[mid] > u) hi = mid; else lo = mid + 1; }
            deg[v] = k_min + lo;
        }
    }
    free(cdf);
    int64_t so = 0, si = 0;
    for (int32_t v = 0; v < n; v++) { so += dout[v]; si += din[v]; }
    {
        uint64_t key = gg_key(seed, 6);
        uint64_t ctr = 0;
        while (so != si) {
            int32_t *deg = so > si ? dout : din;
            int32_t v = (int32_t)gg_below(gg_at(key, ctr++), (uint64_t)n);
            if (deg[v] > 0) { deg[v]--; if (so > si) so--; else si--; }
        }
    }
    int64_t m = so;
    int32_t *instub = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    if (!instub || !keys) { free(instub); free(keys); free(dout); free(din); return 2; }
    int64_t p = 0;
    for (int32_t v = 0; v < n; v++) for (int32_t k = 0; k < din[v]; k++) instub[p++] = v;
    {
        uint64_t key = gg_key(seed, 7);
        for (int64_t i = m - 1; i > 0; i--) {
            int64_t j = (int64_t)gg_below(gg_at(key, (uint64_t)i), (uint64_t)i + 1);
            int32_t t = instub[i]; instub[i] = instub[j]; instub[j] = t;
        }
    }
    p = 0;
    for (int32_t v = 0; v < n; v++)
        for (int32_t k = 0; k < dout[v]; k++, p++)
            keys[p] = ((uint64_t)(uint32_t)instub[p] << 32) | (uint32_t)v;
    free(instub);
    free(dout);
    free(din);
    return csr_from_keys(n, keys, m, out);
}
