/*
 * oracle.c -- plain, slow, single-threaded reference results for the graph
 * method of "SIMD-X: Programming and Processing of Graph Algorithms on GPUs"
 * (Liu & Huang).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; it exists so that tests, the smoke check and the timed CPU
 * baseline can compare the CUDA library against results computed here.  It
 * shares no code, header or table with the CUDA path.
 *
 * Each function is the textbook definition of the result the paper's
 * iterative method reaches exactly (Sec. 6):
 *   - BFS levels (Sec. 6, "BFS"): FIFO-queue breadth-first search.
 *   - SSSP distances (Sec. 2.1, Sec. 3.3): Dijkstra with a binary heap.
 *     The method (delta-stepping / frontier relaxation) reaches the same
 *     unique distances in any relaxation order.
 *   - k-core membership (Sec. 6, "k-Core"): repeatedly delete vertices of
 *     degree < k; the remaining set is the unique maximal subgraph of
 *     minimum degree >= k.
 *   - Core numbers: Batagelj & Zaversnik, "An O(m) algorithm for cores
 *     decomposition of networks" (2003), as a cross-check of k-core.
 *   - PageRank (Sec. 6, "PageRank"): Jacobi power iteration in double
 *     precision, pulling contributions from in-neighbours and summing them.
 *   - The BSP frontier relaxation of Sec. 2.1 (Fig. 1 narrative): a vertex
 *     becomes active when its distance changed in the previous iteration.
 *
 * Conventions: vertex ids int32, CSR offsets int64, unreached BFS level -1,
 * unreached distance UINT32_MAX.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ BFS */
/* Sec. 6 "BFS": level by level from src; level(src) = 0. */
OR_EXPORT int or_bfs(int64_t n, const int64_t *off, const int32_t *idx,
                     int32_t src, int32_t *level)
{
    if (src < 0 || src >= n) return 1;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t v = 0; v < n; ++v) level[v] = -1;
    int64_t head = 0, tail = 0;
    level[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int32_t v = queue[head++];
        for (int64_t p = off[v]; p < off[v + 1]; ++p) {
            int32_t u = idx[p];
            if (level[u] < 0) {
                level[u] = level[v] + 1;
                queue[tail++] = u;
            }
        }
    }
    free(queue);
    return 0;
}

/* ----------------------------------------------------------------- SSSP */
typedef struct { uint64_t d; int32_t v; } hent;

static void heap_push(hent *h, int64_t *sz, uint64_t d, int32_t v)
{
    int64_t i = (*sz)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d <= d) break;
        h[i] = h[p];
        i = p;
    }
    h[i].d = d;
    h[i].v = v;
}

static hent heap_pop(hent *h, int64_t *sz)
{
    hent top = h[0], last = h[--(*sz)];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= *sz) break;
        if (c + 1 < *sz && h[c + 1].d < h[c].d) ++c;
        if (h[c].d >= last.d) break;
        h[i] = h[c];
        i = c;
    }
    if (*sz > 0) h[i] = last;
    return top;
}

/* Dijkstra with lazy deletion.  Distances are accumulated in 64 bits; the
 * call fails (returns 2) if a reached distance does not fit below
 * UINT32_MAX, which is the unreached sentinel. */
OR_EXPORT int or_sssp(int64_t n, const int64_t *off, const int32_t *idx,
                      const uint32_t *w, int32_t src, uint32_t *dist)
{
    if (src < 0 || src >= n) return 1;
    uint64_t *d = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *done = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t cap = off[n] + 1, sz = 0;
    hent *h = (hent *)malloc(sizeof(hent) * (size_t)cap);
    for (int64_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
    d[src] = 0;
    heap_push(h, &sz, 0, src);
    while (sz > 0) {
        hent t = heap_pop(h, &sz);
        if (done[t.v]) continue;
        done[t.v] = 1;
        for (int64_t p = off[t.v]; p < off[t.v + 1]; ++p) {
            int32_t u = idx[p];
            uint64_t nd = t.d + w[p];
            if (nd < d[u]) {
                d[u] = nd;
                heap_push(h, &sz, nd, u);
            }
        }
    }
    int rc = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (d[v] == UINT64_MAX) dist[v] = UINT32_MAX;
        else if (d[v] >= UINT32_MAX) { dist[v] = UINT32_MAX; rc = 2; }
        else dist[v] = (uint32_t)d[v];
    }
    free(d);
    free(done);
    free(h);
    return rc;
}

/* The BSP frontier relaxation narrated in Sec. 2.1: start with src active;
 * in each iteration every active vertex relaxes its out-edges against the
 * distances of the previous iteration (Jacobi), and the vertices whose
 * distance changed form the next active set.  Writes the distance array
 * after each iteration into hist[it*n ...] (UINT32_MAX = infinite) for up to
 * max_it iterations and returns the number of iterations run. */
OR_EXPORT int64_t or_sssp_bsp(int64_t n, const int64_t *off, const int32_t *idx,
                              const uint32_t *w, int32_t src, int64_t max_it,
                              uint32_t *hist)
{
    uint32_t *cur = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    uint32_t *nxt = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    uint8_t *act = (uint8_t *)calloc((size_t)n, 1);
    for (int64_t v = 0; v < n; ++v) cur[v] = UINT32_MAX;
    cur[src] = 0;
    act[src] = 1;
    int64_t it = 0;
    for (; it < max_it; ++it) {
        memcpy(nxt, cur, sizeof(uint32_t) * (size_t)n);
        for (int64_t v = 0; v < n; ++v) {
            if (!act[v]) continue;
            for (int64_t p = off[v]; p < off[v + 1]; ++p) {
                uint64_t nd = (uint64_t)cur[v] + w[p];
                if (nd < nxt[idx[p]]) nxt[idx[p]] = (uint32_t)nd;
            }
        }
        int any = 0;
        for (int64_t v = 0; v < n; ++v) {
            act[v] = nxt[v] != cur[v];
            any |= act[v];
        }
        memcpy(hist + it * n, nxt, sizeof(uint32_t) * (size_t)n);
        memcpy(cur, nxt, sizeof(uint32_t) * (size_t)n);
        if (!any) { ++it; break; }
    }
    free(cur);
    free(nxt);
    free(act);
    return it;
}

/* --------------------------------------------------------------- k-core */
/* Sec. 6 "k-Core": delete every vertex whose degree is < k, updating the
 * degrees of its neighbours, until none is left to delete.  in_core[v] = 1
 * for survivors; resid[v] = number of surviving neighbours of a survivor,
 * 0 for deleted vertices. */
OR_EXPORT int or_kcore(int64_t n, const int64_t *off, const int32_t *idx,
                       uint32_t k, uint8_t *in_core, uint32_t *resid)
{
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t head = 0, tail = 0;
    for (int64_t v = 0; v < n; ++v) {
        deg[v] = off[v + 1] - off[v];
        in_core[v] = 1;
        if (deg[v] < (int64_t)k) {
            in_core[v] = 0;
            queue[tail++] = (int32_t)v;
        }
    }
    while (head < tail) {
        int32_t v = queue[head++];
        for (int64_t p = off[v]; p < off[v + 1]; ++p) {
            int32_t u = idx[p];
            if (!in_core[u]) continue;
            if (--deg[u] < (int64_t)k) {
                in_core[u] = 0;
                queue[tail++] = u;
            }
        }
    }
    for (int64_t v = 0; v < n; ++v) {
        uint32_t c = 0;
        if (in_core[v])
            for (int64_t p = off[v]; p < off[v + 1]; ++p) c += in_core[idx[p]];
        if (resid) resid[v] = c;
    }
    free(deg);
    free(queue);
    return 0;
}

/* Weakly connected components (Sec. 3.2 names WCC among the voting
 * algorithms): label[v] = the smallest vertex id of v's component.  Plain
 * definition: visit the vertices in increasing order and flood each
 * unlabelled one's component by a FIFO search, labelling it with that
 * vertex, which is then the smallest id the component holds.  Edges are
 * followed in both directions of the CSR as given (a symmetric CSR). */
OR_EXPORT int or_wcc(int64_t n, const int64_t *off, const int32_t *idx, uint32_t *label)
{
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t v = 0; v < n; ++v) label[v] = UINT32_MAX;
    for (int64_t r = 0; r < n; ++r) {
        if (label[r] != UINT32_MAX) continue;
        int64_t head = 0, tail = 0;
        label[r] = (uint32_t)r;
        queue[tail++] = r;
        while (head < tail) {
            int64_t v = queue[head++];
            for (int64_t p = off[v]; p < off[v + 1]; ++p) {
                int64_t u = idx[p];
                if (label[u] == UINT32_MAX) {
                    label[u] = (uint32_t)r;
                    queue[tail++] = u;
                }
            }
        }
    }
    free(queue);
    return 0;
}

/* Core number of every vertex (Batagelj & Zaversnik 2003): bucket the
 * vertices by degree and repeatedly remove a vertex of minimum current
 * degree; its current degree at removal is its core number. */
OR_EXPORT int or_coreness(int64_t n, const int64_t *off, const int32_t *idx,
                          uint32_t *core)
{
    if (n == 0) return 0;
    int64_t md = 0;
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) {
        deg[v] = off[v + 1] - off[v];
        if (deg[v] > md) md = deg[v];
    }
    int64_t *bin = (int64_t *)calloc((size_t)md + 2, sizeof(int64_t));
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *vert = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) bin[deg[v]]++;
    int64_t start = 0;
    for (int64_t d = 0; d <= md; ++d) {
        int64_t num = bin[d];
        bin[d] = start;
        start += num;
    }
    for (int64_t v = 0; v < n; ++v) {
        pos[v] = bin[deg[v]];
        vert[pos[v]] = v;
        bin[deg[v]]++;
    }
    for (int64_t d = md; d >= 1; --d) bin[d] = bin[d - 1];
    bin[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = vert[i];
        for (int64_t p = off[v]; p < off[v + 1]; ++p) {
            int64_t u = idx[p];
            if (deg[u] > deg[v]) {
                int64_t du = deg[u], pu = pos[u], pw = bin[du], w = vert[pw];
                if (u != w) {
                    pos[u] = pw;
                    vert[pu] = w;
                    pos[w] = pu;
                    vert[pw] = u;
                }
                bin[du]++;
                deg[u]--;
            }
        }
    }
    for (int64_t v = 0; v < n; ++v) core[v] = (uint32_t)deg[v];
    free(deg);
    free(bin);
    free(pos);
    free(vert);
    return 0;
}

/* ------------------------------------------------------------- PageRank */
/* Sec. 6 "PageRank": pull the contributions x(u)/outdeg(u) of every
 * in-neighbour u, sum them, and iterate until the ranks are stable.
 *   x_0(v)     = 1/n
 *   x_{t+1}(v) = (1-d)/n + d * ( sum_{u in N_in(v)} x_t(u)/outdeg(u) + D_t/n )
 * with D_t the rank held by vertices of out-degree 0, spread uniformly.
 * Stops after the first iteration with ||x_{t+1} - x_t||_1 < tol, or after
 * max_iter iterations; if fixed_iter >= 0, runs exactly fixed_iter
 * iterations instead.  in_off/in_idx is the in-neighbour CSR (CSC) and
 * outdeg the out-degree of each vertex.  Returns the iteration count. */
OR_EXPORT int64_t or_pagerank(int64_t n, const int64_t *in_off,
                              const int32_t *in_idx, const int64_t *outdeg,
                              double d, double tol, int64_t max_iter,
                              int64_t fixed_iter, double *x_out, double *l1_out)
{
    if (n == 0) return 0;
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) x[v] = 1.0 / (double)n;
    int64_t t = 0;
    double l1 = 0.0;
    int64_t limit = fixed_iter >= 0 ? fixed_iter : max_iter;
    while (t < limit) {
        double dangling = 0.0;
        for (int64_t u = 0; u < n; ++u)
            if (outdeg[u] == 0) dangling += x[u];
        l1 = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            double s = 0.0;
            for (int64_t p = in_off[v]; p < in_off[v + 1]; ++p) {
                int32_t u = in_idx[p];
                s += x[u] / (double)outdeg[u];
            }
            y[v] = (1.0 - d) / (double)n + d * (s + dangling / (double)n);
            l1 += fabs(y[v] - x[v]);
        }
        double *tmp = x; x = y; y = tmp;
        ++t;
        if (fixed_iter < 0 && l1 < tol) break;
    }
    memcpy(x_out, x, sizeof(double) * (size_t)n);
    if (l1_out) *l1_out = l1;
    free(x);
    free(y);
    return t;
}

/* ------------------------------------------- parallel timing variants */
/* The same results as or_bfs, or_kcore and or_pagerank, computed with
 * OpenMP on every core the process may use.  They exist only to time the
 * CPU baseline on all host cores; tests pin each one equal, element for
 * element, to its single-threaded definition above.  Built without OpenMP
 * they run on one thread and give the same results. */

/* Level-synchronous BFS: every vertex of level L offers L+1 to its
 * neighbours; the first offer to an unvisited vertex claims it with a
 * compare-and-swap and appends it to level L+1.  Levels are unique, so the
 * result equals or_bfs. */
OR_EXPORT int or_bfs_par(int64_t n, const int64_t *off, const int32_t *idx,
                         int32_t src, int32_t *level)
{
    if (src < 0 || src >= n) return 1;
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) level[v] = -1;
    level[src] = 0;
    cur[0] = src;
    int64_t ncur = 1;
    int32_t L = 0;
    while (ncur > 0) {
        int64_t nnext = 0;
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < ncur; ++i) {
            int32_t v = cur[i];
            for (int64_t p = off[v]; p < off[v + 1]; ++p) {
                int32_t u = idx[p];
                int32_t expect = -1;
                if (__atomic_load_n(&level[u], __ATOMIC_RELAXED) == -1 &&
                    __atomic_compare_exchange_n(&level[u], &expect, L + 1, 0, __ATOMIC_RELAXED,
                                                __ATOMIC_RELAXED)) {
                    int64_t slot = __atomic_fetch_add(&nnext, 1, __ATOMIC_RELAXED);
                    nxt[slot] = u;
                }
            }
        }
        int32_t *t = cur; cur = nxt; nxt = t;
        ncur = nnext;
        ++L;
    }
    free(cur);
    free(nxt);
    return 0;
}

/* k-core by level-synchronous peeling: the degrees are counted in parallel;
 * each round deletes the vertices that fell below k in the previous round
 * and decrements their surviving neighbours atomically; the decrement that
 * takes a neighbour from k to k-1 enqueues it.  The surviving set is the
 * unique maximal subgraph of minimum degree >= k, so the result equals
 * or_kcore. */
OR_EXPORT int or_kcore_par(int64_t n, const int64_t *off, const int32_t *idx,
                           uint32_t k, uint8_t *in_core, uint32_t *resid)
{
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t ncur = 0;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        deg[v] = off[v + 1] - off[v];
        in_core[v] = deg[v] >= (int64_t)k;
        if (!in_core[v]) {
            int64_t slot = __atomic_fetch_add(&ncur, 1, __ATOMIC_RELAXED);
            cur[slot] = (int32_t)v;
        }
    }
    while (ncur > 0) {
        int64_t nnext = 0;
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < ncur; ++i) {
            int32_t v = cur[i];
            for (int64_t p = off[v]; p < off[v + 1]; ++p) {
                int32_t u = idx[p];
                if (!__atomic_load_n(&in_core[u], __ATOMIC_RELAXED)) continue;
                if (__atomic_fetch_sub(&deg[u], 1, __ATOMIC_RELAXED) == (int64_t)k) {
                    __atomic_store_n(&in_core[u], 0, __ATOMIC_RELAXED);
                    int64_t slot = __atomic_fetch_add(&nnext, 1, __ATOMIC_RELAXED);
                    nxt[slot] = u;
                }
            }
        }
        int32_t *t = cur; cur = nxt; nxt = t;
        ncur = nnext;
    }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; ++v) {
        uint32_t c = 0;
        if (in_core[v])
            for (int64_t p = off[v]; p < off[v + 1]; ++p) c += in_core[idx[p]];
        if (resid) resid[v] = c;
    }
    free(deg);
    free(cur);
    free(nxt);
    return 0;
}

/* PageRank as or_pagerank, with the per-vertex pulls of an iteration run in
 * parallel (each vertex sums its in-edges in the same order as there); the
 * dangling mass and the L1 change are summed in vertex order on one thread,
 * so every value equals or_pagerank's bit for bit. */
OR_EXPORT int64_t or_pagerank_par(int64_t n, const int64_t *in_off,
                                  const int32_t *in_idx, const int64_t *outdeg,
                                  double d, double tol, int64_t max_iter,
                                  int64_t fixed_iter, double *x_out, double *l1_out)
{
    if (n == 0) return 0;
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) x[v] = 1.0 / (double)n;
    int64_t t = 0;
    double l1 = 0.0;
    int64_t limit = fixed_iter >= 0 ? fixed_iter : max_iter;
    while (t < limit) {
        double dangling = 0.0;
        for (int64_t u = 0; u < n; ++u)
            if (outdeg[u] == 0) dangling += x[u];
#pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t v = 0; v < n; ++v) {
            double s = 0.0;
            for (int64_t p = in_off[v]; p < in_off[v + 1]; ++p) {
                int32_t u = in_idx[p];
                s += x[u] / (double)outdeg[u];
            }
            y[v] = (1.0 - d) / (double)n + d * (s + dangling / (double)n);
        }
        l1 = 0.0;
        for (int64_t v = 0; v < n; ++v) l1 += fabs(y[v] - x[v]);
        double *tmp = x; x = y; y = tmp;
        ++t;
        if (fixed_iter < 0 && l1 < tol) break;
    }
    memcpy(x_out, x, sizeof(double) * (size_t)n);
    if (l1_out) *l1_out = l1;
    free(x);
    free(y);
    return t;
}

/* Threads the parallel variants use (1 when built without OpenMP). */
OR_EXPORT int or_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------ PageRank, push tail */
/* Sec. 6 "PageRank": start with pull (the Jacobi iteration of or_pagerank)
 * and, once most vertices are stable, switch to push, propagating only the
 * rank changes that are still large (the accumulative delta iteration the
 * paper cites for this switch).  The paper decides the switch by a decision
 * tree it does not describe; the rule here is a reading of it, a tree of
 * two tests made after pull iteration i >= 1 (the run not yet converged):
 * the pull contracts slowly, L1_i >= rho_min * L1_{i-1} (where it contracts
 * fast, the signed changes cancel in the pull sums and a selective push
 * loses that), and few vertices are unstable: those whose change exceeds
 * eps_i = theta * L1_{i-1} / n have fewer than E / alpha out-edges.  Both
 * hold: switch to push.  alpha <= 0 never switches.
 *
 * With M the iteration matrix of or_pagerank (x_{t+1} = (1-d)/n + M x_t),
 * the push phase keeps a pair (x, r) with x* = x + (I - M)^-1 r:
 *   switch after pull iteration i: x = x_i, r = x_{i+1} - x_i;
 *   each push iteration: L1 = ||r||_1; stop if L1 < tol; otherwise every
 *   vertex with |r(v)| > eps (eps = theta * L1_prev / n, or 0 when the
 *   previous iteration selected no vertex) moves r(v) into x(v) and sends
 *   d * r(v) / outdeg(v) to each out-neighbour (dangling vertices send
 *   d * r(v) / n to every vertex); L1_prev = L1.
 * The result is x + r, so ||x_out - x*||_1 <= d / (1 - d) * L1 < d / (1 - d)
 * * tol, the same guarantee as the pull stop.  off/idx are out-edges,
 * in_off/in_idx in-edges, outdeg = off[v+1] - off[v].  Returns the number of
 * iterations (pull + push); *pull_iters gets the pull ones. */
OR_EXPORT int64_t or_pagerank_delta(int64_t n, const int64_t *off, const int32_t *idx,
                                    const int64_t *in_off, const int32_t *in_idx,
                                    double d, double tol, int64_t max_iter, double alpha,
                                    double theta, double rho_min, double *x_out, int64_t *pull_iters,
                                    double *l1_out)
{
    if (n == 0) { *pull_iters = 0; return 0; }
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *take = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t e = off[n];
    for (int64_t v = 0; v < n; ++v) x[v] = 1.0 / (double)n;
    int64_t t = 0;
    double l1 = 0.0, l1_prev = 0.0;
    int push = 0;
    /* pull phase */
    while (t < max_iter) {
        double dangling = 0.0;
        for (int64_t u = 0; u < n; ++u)
            if (off[u + 1] == off[u]) dangling += x[u];
        l1 = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            double s = 0.0;
            for (int64_t p = in_off[v]; p < in_off[v + 1]; ++p) {
                int32_t u = in_idx[p];
                s += x[u] / (double)(off[u + 1] - off[u]);
            }
            y[v] = (1.0 - d) / (double)n + d * (s + dangling / (double)n);
            l1 += fabs(y[v] - x[v]);
        }
        ++t;
        if (l1 < tol) {  /* converged by pull alone */
            double *tmp = x; x = y; y = tmp;
            break;
        }
        if (t >= 2 && alpha > 0.0 && l1 >= rho_min * l1_prev) {
            double eps = theta * l1_prev / (double)n, m_act = 0.0;
            for (int64_t v = 0; v < n; ++v)
                if (fabs(y[v] - x[v]) > eps) m_act += (double)(off[v + 1] - off[v]);
            if (m_act * alpha < (double)e) {
                for (int64_t v = 0; v < n; ++v) r[v] = y[v] - x[v];  /* x stays x_i */
                push = 1;
                break;
            }
        }
        l1_prev = l1;
        double *tmp = x; x = y; y = tmp;
    }
    *pull_iters = t;
    if (push) {
        double unif = 0.0;   /* rank sent to every vertex by dangling vertices */
        int none = 0;
        l1_prev = l1;
        for (;;) {
            l1 = 0.0;
            for (int64_t v = 0; v < n; ++v) {
                r[v] += unif;
                l1 += fabs(r[v]);
            }
            unif = 0.0;
            if (l1 < tol || t >= max_iter) break;
            double eps = none ? 0.0 : theta * l1_prev / (double)n, dang = 0.0;
            int64_t sel = 0;
            for (int64_t v = 0; v < n; ++v) {
                take[v] = 0.0;
                if (fabs(r[v]) > eps) {
                    take[v] = r[v];
                    x[v] += r[v];
                    r[v] = 0.0;
                    ++sel;
                    if (off[v + 1] == off[v]) dang += take[v];
                }
            }
            for (int64_t v = 0; v < n; ++v) {
                if (take[v] == 0.0 || off[v + 1] == off[v]) continue;
                double c = d * take[v] / (double)(off[v + 1] - off[v]);
                for (int64_t p = off[v]; p < off[v + 1]; ++p) r[idx[p]] += c;
            }
            unif = d * dang / (double)n;
            none = sel == 0;
            l1_prev = l1;
            ++t;
        }
        for (int64_t v = 0; v < n; ++v) x[v] += r[v];
    }
    memcpy(x_out, x, sizeof(double) * (size_t)n);
    if (l1_out) *l1_out = l1;
    free(x);
    free(y);
    free(r);
    free(take);
    return t;
}
