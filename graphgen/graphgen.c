/*
 * graphgen.c -- seeded synthetic graph inputs (R-MAT, 4-neighbour grid,
 * sub-sampled R-MAT for packed multi-graph batches, edge weights).
 *
 * This module holds no step of the graph method itself: it only builds the
 * inputs that both the CPU oracle and the CUDA path consume.  Everything is
 * deterministic for a given seed and independent of the thread count.
 *
 * Inputs follow the shapes the paper evaluates on (Sec. 6, Table 3): a
 * Graph500-style Kronecker / R-MAT generator with (a,b,c,d) =
 * (0.57,0.19,0.19,0.05) and edge factor 16, symmetrised, with self loops and
 * duplicates removed, stored as CSR (Sec. 6 "Storage Format"); random integer
 * weights per edge (Sec. 6, weights generated like Gunrock's); and a
 * high-diameter 4-neighbour grid standing in for the road graphs ER / RC.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based
 * hash so that every draw is a pure function of (seed, edge, level).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_EXPORT __attribute__((visibility("default")))

static inline uint64_t sm64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

/* Uniform double in [0,1) for draw (seed, counter). */
static inline double u01(uint64_t seed, uint64_t counter)
{
    uint64_t h = sm64(seed ^ sm64(counter));
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

GG_EXPORT uint64_t gg_splitmix64(uint64_t x) { return sm64(x); }

/* Hash of an unordered vertex pair, used for per-undirected-edge weights. */
static inline uint64_t pair_hash(uint64_t seed, uint32_t u, uint32_t v)
{
    uint32_t lo = u < v ? u : v, hi = u < v ? v : u;
    return sm64(seed ^ sm64(((uint64_t)lo << 32) | hi));
}

/* One R-MAT tuple: `scale` quadrant draws, most significant bit first. */
static inline void rmat_tuple(uint64_t seed, uint64_t i, int scale, double a,
                              double ab, double abc, uint32_t *pu, uint32_t *pv)
{
    uint32_t u = 0, v = 0;
    for (int l = 0; l < scale; ++l) {
        double r = u01(seed, (i << 6) | (uint64_t)l);
        uint32_t bu, bv;
        if (r < a) { bu = 0; bv = 0; }
        else if (r < ab) { bu = 0; bv = 1; }
        else if (r < abc) { bu = 1; bv = 0; }
        else { bu = 1; bv = 1; }
        u |= bu << (scale - 1 - l);
        v |= bv << (scale - 1 - l);
    }
    *pu = u;
    *pv = v;
}

/* ---------------------------------------------------------------------- */
/* Parallel LSD radix sort of 64-bit keys (11-bit digits over `bits`).    */
/* ---------------------------------------------------------------------- */
static void radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t m, int bits)
{
    const int D = 11, R = 1 << D;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    int64_t *hist = (int64_t *)malloc(sizeof(int64_t) * (size_t)nthr * R);
    uint64_t *src = keys, *dst = tmp;
    int passes = (bits + D - 1) / D;
    for (int p = 0; p < passes; ++p) {
        int shift = p * D;
        memset(hist, 0, sizeof(int64_t) * (size_t)nthr * R);
#pragma omp parallel num_threads(nthr)
        {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            int64_t lo = m * t / nthr, hi = m * (t + 1) / nthr;
            int64_t *h = hist + (size_t)t * R;
            for (int64_t i = lo; i < hi; ++i) h[(src[i] >> shift) & (R - 1)]++;
#pragma omp barrier
#pragma omp single
            {
                int64_t run = 0;
                for (int d = 0; d < R; ++d)
                    for (int tt = 0; tt < nthr; ++tt) {
                        int64_t c = hist[(size_t)tt * R + d];
                        hist[(size_t)tt * R + d] = run;
                        run += c;
                    }
            }
            for (int64_t i = lo; i < hi; ++i) {
                uint64_t k = src[i];
                dst[h[(k >> shift) & (R - 1)]++] = k;
            }
        }
        uint64_t *s = src; src = dst; dst = s;
    }
    if (src != keys) memcpy(keys, src, sizeof(uint64_t) * (size_t)m);
    free(hist);
}

/* A built graph held by the library until copied out. */
typedef struct {
    int64_t n, e;
    int64_t *offsets; /* [n+1] */
    int32_t *indices; /* [e]   */
} gg_graph;

/* Sort packed (u << vbits | v) keys, drop duplicates, emit CSR. */
static gg_graph *csr_from_keys(uint64_t *keys, int64_t m, int64_t n, int vbits)
{
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    radix_sort_u64(keys, tmp, m, 2 * vbits);
    free(tmp);
    /* unique (sequential: memory bound and simple) */
    int64_t w = 0;
    for (int64_t i = 0; i < m; ++i)
        if (w == 0 || keys[i] != keys[w - 1]) keys[w++] = keys[i];
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    g->n = n;
    g->e = w;
    g->offsets = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->indices = (int32_t *)malloc(sizeof(int32_t) * (size_t)(w > 0 ? w : 1));
    uint64_t vmask = (vbits >= 64) ? ~0ULL : ((1ULL << vbits) - 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < w; ++i) g->indices[i] = (int32_t)(keys[i] & vmask);
    /* offsets: position of the first key of each source */
    for (int64_t i = 0; i < w; ++i) g->offsets[(keys[i] >> vbits) + 1]++;
    for (int64_t v = 0; v < n; ++v) g->offsets[v + 1] += g->offsets[v];
    return g;
}

static int bits_for(int64_t n)
{
    int b = 1;
    while (((int64_t)1 << b) < n) ++b;
    return b;
}

/*
 * R-MAT at `scale` (n = 2^scale), edge_factor * n tuples, symmetrised,
 * self loops and duplicates removed.  Tuple i is a pure function of
 * (seed, i); no noise and no vertex permutation, so vertex 0 is the hub.
 */
GG_EXPORT gg_graph *gg_rmat(int scale, int edge_factor, double a, double b,
                            double c, uint64_t seed)
{
    int64_t n = (int64_t)1 << scale;
    int64_t m = (int64_t)edge_factor * n;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * m + 1));
    double ab = a + b, abc = a + b + c;
    int64_t *cnt = NULL;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    cnt = (int64_t *)calloc((size_t)nthr + 1, sizeof(int64_t));
    /* pass 1: count non-loop tuples per thread block; pass 2: write */
#pragma omp parallel num_threads(nthr)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        int64_t lo = m * t / nthr, hi = m * (t + 1) / nthr, k = 0;
        for (int64_t i = lo; i < hi; ++i) {
            uint32_t u, v;
            rmat_tuple(seed, (uint64_t)i, scale, a, ab, abc, &u, &v);
            if (u != v) ++k;
        }
        cnt[t + 1] = k;
#pragma omp barrier
#pragma omp single
        for (int tt = 0; tt < nthr; ++tt) cnt[tt + 1] += cnt[tt];
        int64_t pos = 2 * cnt[t];
        for (int64_t i = lo; i < hi; ++i) {
            uint32_t u, v;
            rmat_tuple(seed, (uint64_t)i, scale, a, ab, abc, &u, &v);
            if (u == v) continue;
            keys[pos++] = ((uint64_t)u << scale) | v;
            keys[pos++] = ((uint64_t)v << scale) | u;
        }
    }
    int64_t total = 2 * cnt[nthr];
    free(cnt);
    gg_graph *g = csr_from_keys(keys, total, n, scale);
    free(keys);
    return g;
}

/*
 * R-MAT restricted to n vertices (n <= 2^scale): tuples drawn at `scale`
 * are kept only when both endpoints are < n, until `tuples` are kept.
 * Used for the packed batch of many small graphs.
 */
GG_EXPORT gg_graph *gg_rmat_sub(int64_t n, int scale, int64_t tuples, double a,
                                double b, double c, uint64_t seed)
{
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * tuples + 1));
    double ab = a + b, abc = a + b + c;
    int64_t kept = 0, w = 0;
    for (uint64_t i = 0; kept < tuples; ++i) {
        uint32_t u, v;
        rmat_tuple(seed, i, scale, a, ab, abc, &u, &v);
        if ((int64_t)u >= n || (int64_t)v >= n) continue;
        ++kept;
        if (u == v) continue;
        keys[w++] = ((uint64_t)u << scale) | v;
        keys[w++] = ((uint64_t)v << scale) | u;
    }
    gg_graph *g = csr_from_keys(keys, w, n, scale);
    free(keys);
    return g;
}

/* rows x cols 4-neighbour grid, id = r*cols + c, no wrap-around. */
GG_EXPORT gg_graph *gg_grid(int64_t rows, int64_t cols)
{
    int64_t n = rows * cols;
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    g->n = n;
    g->offsets = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    g->offsets[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t r = v / cols, c = v % cols;
        int d = (r > 0) + (c > 0) + (c + 1 < cols) + (r + 1 < rows);
        g->offsets[v + 1] = g->offsets[v] + d;
    }
    g->e = g->offsets[n];
    g->indices = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->e > 0 ? g->e : 1));
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        int64_t r = v / cols, c = v % cols, p = g->offsets[v];
        if (r > 0) g->indices[p++] = (int32_t)(v - cols);
        if (c > 0) g->indices[p++] = (int32_t)(v - 1);
        if (c + 1 < cols) g->indices[p++] = (int32_t)(v + 1);
        if (r + 1 < rows) g->indices[p++] = (int32_t)(v + cols);
    }
    return g;
}

/* Graph from an explicit undirected edge list (both directions stored). */
GG_EXPORT gg_graph *gg_from_edges(int64_t n, int64_t m, const int32_t *src,
                                  const int32_t *dst)
{
    int vb = bits_for(n > 1 ? n : 2);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * m + 1));
    int64_t w = 0;
    for (int64_t i = 0; i < m; ++i) {
        uint32_t u = (uint32_t)src[i], v = (uint32_t)dst[i];
        if (u == v) continue;
        keys[w++] = ((uint64_t)u << vb) | v;
        keys[w++] = ((uint64_t)v << vb) | u;
    }
    gg_graph *g = csr_from_keys(keys, w, n, vb);
    free(keys);
    return g;
}

GG_EXPORT int64_t gg_n(const gg_graph *g) { return g->n; }
GG_EXPORT int64_t gg_e(const gg_graph *g) { return g->e; }

GG_EXPORT void gg_copy(const gg_graph *g, int64_t *offsets, int32_t *indices)
{
    memcpy(offsets, g->offsets, sizeof(int64_t) * (size_t)(g->n + 1));
    if (g->e) memcpy(indices, g->indices, sizeof(int32_t) * (size_t)g->e);
}

GG_EXPORT void gg_free(gg_graph *g)
{
    if (!g) return;
    free(g->offsets);
    free(g->indices);
    free(g);
}

/* Per-undirected-edge weight lo + H(seed, min(u,v), max(u,v)) mod (hi-lo+1):
 * both stored directions of an edge get the same weight. */
GG_EXPORT void gg_weights(int64_t n, const int64_t *offsets,
                          const int32_t *indices, uint64_t seed, uint32_t lo,
                          uint32_t hi, uint32_t *w)
{
    uint64_t span = (uint64_t)hi - lo + 1;
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t u = 0; u < n; ++u)
        for (int64_t p = offsets[u]; p < offsets[u + 1]; ++p)
            w[p] = lo + (uint32_t)(pair_hash(seed, (uint32_t)u,
                                             (uint32_t)indices[p]) % span);
}

/* k distinct vertices with non-zero degree, uniform, by rejection on the
 * counter-based stream (seed, draw index).  Returns the number written
 * (fewer than k only if fewer non-isolated vertices exist). */
GG_EXPORT int64_t gg_pick_sources(int64_t n, const int64_t *offsets, int64_t k,
                                  uint64_t seed, int32_t *out)
{
    int64_t nonzero = 0;
    for (int64_t v = 0; v < n; ++v) nonzero += offsets[v + 1] > offsets[v];
    if (k > nonzero) k = nonzero;
    int64_t got = 0;
    for (uint64_t i = 0; got < k; ++i) {
        int64_t v = (int64_t)(sm64(seed ^ sm64(i)) % (uint64_t)n);
        if (offsets[v + 1] == offsets[v]) continue;
        int dup = 0;
        for (int64_t j = 0; j < got; ++j) dup |= out[j] == (int32_t)v;
        if (!dup) out[got++] = (int32_t)v;
    }
    return got;
}
