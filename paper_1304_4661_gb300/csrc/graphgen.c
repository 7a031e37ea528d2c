/*
 * graphgen.c -- seeded synthetic graph and query-pair generators.
 *
 * This file holds input generation only: it builds undirected, unweighted,
 * simple graphs (symmetric CSR, sorted neighbour lists, no self-loops, no
 * duplicate arcs, uint32 offsets and column ids) and uniform query pairs.
 * It contains none of the labelling method's arithmetic; the CUDA library
 * and the CPU oracle both consume its output as plain data.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, "Scrambled linear
 * pseudorandom number generators", 2018), its 256-bit state filled from the
 * seed by splitmix64 (Steele, Lea & Flood, 2014), as the authors recommend.
 * Bounded integers use Lemire's multiply-shift with rejection ("Fast random
 * integer generation in an interval", 2019); doubles take the top 53 bits.
 * Everything is integer or exactly representable, so the same seed gives the
 * same graph on x86-64 and AArch64.
 *
 * Graph families (the workloads of the paper are power-law, small-world
 * networks, Sec. 6.1; these synthetic families stand in for them):
 *   - Barabasi-Albert: an (m+1)-clique, then each new vertex attaches to m
 *     distinct earlier vertices drawn proportionally to degree (uniform draw
 *     from the list of edge endpoints, duplicates redrawn).
 *   - Watts-Strogatz: ring lattice with k/2 neighbours per side, each lattice
 *     edge (i, i+j) rewired with probability p to (i, w), w uniform, w != i,
 *     never creating a duplicate edge.
 *   - R-MAT: ef * 2^scale edge samples, each descending `scale` levels of the
 *     adjacency matrix with quadrant probabilities (a, b, c, d); symmetrised,
 *     self-loops and duplicates dropped. No noise, no vertex permutation.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ RNG */
typedef struct { uint64_t s[4]; } gg_rng;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void rng_seed(gg_rng *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(gg_rng *r) {
    uint64_t *s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* uniform double in [0, 1) from the top 53 bits */
static inline double rng_unif(gg_rng *r) {
    return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, bound), bound >= 1 (Lemire, with rejection) */
static inline uint64_t rng_below(gg_rng *r, uint64_t bound) {
    uint64_t x = rng_next(r);
    __uint128_t m = (__uint128_t)x * bound;
    uint64_t l = (uint64_t)m;
    if (l < bound) {
        uint64_t thresh = (0 - bound) % bound;
        while (l < thresh) {
            x = rng_next(r);
            m = (__uint128_t)x * bound;
            l = (uint64_t)m;
        }
    }
    return (uint64_t)(m >> 64);
}

/* ------------------------------------------------------ graph container */
typedef struct gg_graph {
    uint32_t n;
    uint64_t nnz;   /* number of arcs = 2 x undirected edges */
    uint32_t *off;  /* n + 1 */
    uint32_t *col;  /* nnz */
} gg_graph;

/* LSD radix sort of 64-bit keys, only over the low `bits` bits. */
static int radix_sort_u64(uint64_t *a, uint64_t len, int bits) {
    if (len < 2) return 0;
    uint64_t *tmp = (uint64_t *)malloc(len * sizeof(uint64_t));
    if (!tmp) return -1;
    const int D = 11;
    const uint64_t R = 1ull << D;
    uint64_t *cnt = (uint64_t *)malloc(R * sizeof(uint64_t));
    if (!cnt) { free(tmp); return -1; }
    uint64_t *src = a, *dst = tmp;
    for (int shift = 0; shift < bits; shift += D) {
        memset(cnt, 0, R * sizeof(uint64_t));
        for (uint64_t i = 0; i < len; ++i) cnt[(src[i] >> shift) & (R - 1)]++;
        uint64_t s = 0;
        for (uint64_t d = 0; d < R; ++d) { uint64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (uint64_t i = 0; i < len; ++i) dst[cnt[(src[i] >> shift) & (R - 1)]++] = src[i];
        uint64_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, len * sizeof(uint64_t));
    free(cnt);
    free(tmp);
    return 0;
}

static int bits_for(uint32_t n) {
    int b = 1;
    while (b < 32 && ((uint64_t)1 << b) < n) ++b;
    return b;
}

/* Build a simple undirected CSR from an edge list: both directions of every
 * edge, self-loops dropped, duplicates merged, neighbour lists ascending.
 * Returns NULL on allocation failure or if an id is >= n. */
static gg_graph *csr_from_pairs(uint32_t n, uint64_t m, const uint32_t *eu, const uint32_t *ev) {
    uint64_t *keys = (uint64_t *)malloc((m ? 2 * m : 1) * sizeof(uint64_t));
    if (!keys) return NULL;
    uint64_t k = 0;
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t u = eu[i], v = ev[i];
        if (u >= n || v >= n) { free(keys); return NULL; }
        if (u == v) continue;
        keys[k++] = ((uint64_t)u << 32) | v;
        keys[k++] = ((uint64_t)v << 32) | u;
    }
    /* both halves of the key hold ids < n: sort the low bits of each half by
     * packing into a contiguous 2*bits integer first */
    int b = bits_for(n);
    for (uint64_t i = 0; i < k; ++i) keys[i] = ((keys[i] >> 32) << b) | (keys[i] & 0xffffffffull);
    if (radix_sort_u64(keys, k, 2 * b)) { free(keys); return NULL; }
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    if (!g) { free(keys); return NULL; }
    g->n = n;
    g->off = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    uint64_t uniq = 0;
    for (uint64_t i = 0; i < k; ++i)
        if (i == 0 || keys[i] != keys[i - 1]) ++uniq;
    g->col = (uint32_t *)malloc((uniq ? uniq : 1) * sizeof(uint32_t));
    if (!g->off || !g->col || uniq >= 0xffffffffull) {
        free(g->off); free(g->col); free(g); free(keys);
        return NULL;
    }
    const uint64_t mask = (b >= 32) ? 0xffffffffull : (((uint64_t)1 << b) - 1);
    uint64_t w = 0;
    for (uint64_t i = 0; i < k; ++i) {
        if (i > 0 && keys[i] == keys[i - 1]) continue;
        uint32_t u = (uint32_t)(keys[i] >> b);
        uint32_t v = (uint32_t)(keys[i] & mask);
        g->off[u + 1]++;
        g->col[w++] = v;
    }
    for (uint32_t v = 0; v < n; ++v) g->off[v + 1] += g->off[v];
    g->nnz = uniq;
    free(keys);
    return g;
}

/* ---------------------------------------------------------- public API */
gg_graph *gg_from_edges(uint32_t n, uint64_t m, const uint32_t *eu, const uint32_t *ev) {
    return csr_from_pairs(n, m, eu, ev);
}

gg_graph *gg_ba(uint32_t n, uint32_t m, uint64_t seed) {
    if (m == 0) m = 1;
    gg_rng r;
    rng_seed(&r, seed);
    uint32_t core = m + 1 < n ? m + 1 : n;
    uint64_t max_e = (uint64_t)core * (core - 1) / 2 + (uint64_t)(n > core ? n - core : 0) * m;
    uint32_t *eu = (uint32_t *)malloc((max_e ? max_e : 1) * sizeof(uint32_t));
    uint32_t *ev = (uint32_t *)malloc((max_e ? max_e : 1) * sizeof(uint32_t));
    uint32_t *ends = (uint32_t *)malloc((max_e ? 2 * max_e : 1) * sizeof(uint32_t));
    uint32_t *pick = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
    if (!eu || !ev || !ends || !pick) { free(eu); free(ev); free(ends); free(pick); return NULL; }
    uint64_t e = 0, ne = 0;
    for (uint32_t i = 0; i < core; ++i)
        for (uint32_t j = i + 1; j < core; ++j) {
            eu[e] = i; ev[e] = j; ++e;
            ends[ne++] = i; ends[ne++] = j;
        }
    for (uint32_t v = core; v < n; ++v) {
        uint32_t got = 0;
        while (got < m) {
            uint32_t x = ends[rng_below(&r, ne)];
            int dup = 0;
            for (uint32_t q = 0; q < got; ++q) if (pick[q] == x) { dup = 1; break; }
            if (!dup) pick[got++] = x;
        }
        for (uint32_t q = 0; q < m; ++q) {
            eu[e] = v; ev[e] = pick[q]; ++e;
            ends[ne++] = v; ends[ne++] = pick[q];
        }
    }
    gg_graph *g = csr_from_pairs(n, e, eu, ev);
    free(eu); free(ev); free(ends); free(pick);
    return g;
}

/* open-addressing set of undirected edges (key = min << 32 | max) */
typedef struct { uint64_t *slot; uint64_t cap; } eset;
#define ESET_EMPTY 0xffffffffffffffffull
#define ESET_TOMB  0xfffffffffffffffeull
static uint64_t ekey(uint32_t a, uint32_t b) {
    return a < b ? (((uint64_t)a << 32) | b) : (((uint64_t)b << 32) | a);
}
static uint64_t ehash(uint64_t k) { uint64_t x = k; return splitmix64_next(&x); }
static int eset_find(const eset *s, uint64_t k) {
    for (uint64_t i = ehash(k) & (s->cap - 1);; i = (i + 1) & (s->cap - 1)) {
        if (s->slot[i] == k) return 1;
        if (s->slot[i] == ESET_EMPTY) return 0;
    }
}
static void eset_add(eset *s, uint64_t k) {
    for (uint64_t i = ehash(k) & (s->cap - 1);; i = (i + 1) & (s->cap - 1)) {
        if (s->slot[i] == ESET_EMPTY || s->slot[i] == ESET_TOMB) { s->slot[i] = k; return; }
    }
}
static void eset_del(eset *s, uint64_t k) {
    for (uint64_t i = ehash(k) & (s->cap - 1);; i = (i + 1) & (s->cap - 1)) {
        if (s->slot[i] == k) { s->slot[i] = ESET_TOMB; return; }
        if (s->slot[i] == ESET_EMPTY) return;
    }
}

gg_graph *gg_ws(uint32_t n, uint32_t k, double p, uint64_t seed) {
    gg_rng r;
    rng_seed(&r, seed);
    uint32_t half = k / 2;
    if (n < 3 || half == 0 || half >= n) return csr_from_pairs(n, 0, NULL, NULL);
    uint64_t ne = (uint64_t)n * half;
    eset s;
    s.cap = 16;
    while (s.cap < 4 * ne) s.cap <<= 1;
    s.slot = (uint64_t *)malloc(s.cap * sizeof(uint64_t));
    uint32_t *deg = (uint32_t *)calloc(n, sizeof(uint32_t));
    if (!s.slot || !deg) { free(s.slot); free(deg); return NULL; }
    for (uint64_t i = 0; i < s.cap; ++i) s.slot[i] = ESET_EMPTY;
    for (uint32_t j = 1; j <= half; ++j)
        for (uint32_t i = 0; i < n; ++i) {
            uint32_t w = (i + j) % n;
            uint64_t key = ekey(i, w);
            if (!eset_find(&s, key)) { eset_add(&s, key); deg[i]++; deg[w]++; }
        }
    for (uint32_t j = 1; j <= half; ++j)
        for (uint32_t i = 0; i < n; ++i) {
            if (rng_unif(&r) >= p) continue;
            uint32_t old = (i + j) % n;
            uint64_t okey = ekey(i, old);
            if (!eset_find(&s, okey)) continue;     /* lattice edge already rewired away */
            if (deg[i] >= n - 1) continue;          /* no free endpoint */
            uint32_t w;
            do { w = (uint32_t)rng_below(&r, n); } while (w == i || eset_find(&s, ekey(i, w)));
            eset_del(&s, okey);
            deg[old]--;
            eset_add(&s, ekey(i, w));
            deg[w]++;
        }
    uint32_t *eu = (uint32_t *)malloc(ne * sizeof(uint32_t));
    uint32_t *ev = (uint32_t *)malloc(ne * sizeof(uint32_t));
    if (!eu || !ev) { free(eu); free(ev); free(s.slot); free(deg); return NULL; }
    uint64_t e = 0;
    for (uint64_t i = 0; i < s.cap; ++i) {
        uint64_t key = s.slot[i];
        if (key == ESET_EMPTY || key == ESET_TOMB) continue;
        eu[e] = (uint32_t)(key >> 32); ev[e] = (uint32_t)key; ++e;
    }
    gg_graph *g = csr_from_pairs(n, e, eu, ev);
    free(eu); free(ev); free(s.slot); free(deg);
    return g;
}

gg_graph *gg_rmat(uint32_t scale, uint32_t ef, double a, double b, double c, uint64_t seed) {
    if (scale == 0 || scale > 30) return NULL;
    gg_rng r;
    rng_seed(&r, seed);
    uint32_t n = 1u << scale;
    uint64_t m = (uint64_t)ef << scale;
    uint32_t *eu = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t *ev = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    if (!eu || !ev) { free(eu); free(ev); return NULL; }
    const double ab = a + b, abc = a + b + c;
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t u = 0, v = 0;
        for (uint32_t l = 0; l < scale; ++l) {
            double x = rng_unif(&r);
            uint32_t bu, bv;
            if (x < a) { bu = 0; bv = 0; }
            else if (x < ab) { bu = 0; bv = 1; }
            else if (x < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        eu[i] = u; ev[i] = v;
    }
    gg_graph *g = csr_from_pairs(n, m, eu, ev);
    free(eu); free(ev);
    return g;
}

uint32_t gg_n(const gg_graph *g) { return g->n; }
uint64_t gg_nnz(const gg_graph *g) { return g->nnz; }
void gg_copy(const gg_graph *g, uint32_t *off, uint32_t *col) {
    memcpy(off, g->off, ((size_t)g->n + 1) * sizeof(uint32_t));
    if (g->nnz) memcpy(col, g->col, g->nnz * sizeof(uint32_t));
}
void gg_free(gg_graph *g) {
    if (!g) return;
    free(g->off); free(g->col); free(g);
}

/* q uniform pairs (s, t) in [0, n)^2; s == t allowed */
void gg_pairs(uint32_t n, uint64_t q, uint64_t seed, uint32_t *s, uint32_t *t) {
    gg_rng r;
    rng_seed(&r, seed);
    for (uint64_t i = 0; i < q; ++i) {
        s[i] = (uint32_t)rng_below(&r, n);
        t[i] = (uint32_t)rng_below(&r, n);
    }
}

/* count doubles uniform in [0, 1) */
void gg_uniform(uint64_t seed, uint64_t count, double *out) {
    gg_rng r;
    rng_seed(&r, seed);
    for (uint64_t i = 0; i < count; ++i) out[i] = rng_unif(&r);
}

/* count integers uniform in [0, bound) */
void gg_below(uint64_t seed, uint64_t count, uint64_t bound, uint64_t *out) {
    gg_rng r;
    rng_seed(&r, seed);
    for (uint64_t i = 0; i < count; ++i) out[i] = rng_below(&r, bound);
}
