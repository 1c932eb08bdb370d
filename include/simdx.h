/*
 * simdx.h -- C ABI of the GB300 (sm_103a) implementation of the
 * Active-Compute-Combine (ACC) graph hot path of "SIMD-X: Programming and
 * Processing of Graph Algorithms on GPUs" (Liu & Huang).
 *
 * One call runs one whole graph algorithm as ONE persistent cooperative
 * kernel (Sec. 5, "Push-Pull based kernel fusion"; Eq. 1): every BSP
 * iteration filters the active vertices into degree-binned task lists
 * (Sec. 4, online / ballot filters and the JIT controller), computes on the
 * edges of each active vertex in push or pull direction, and combines the
 * updates into vertex state (Sec. 3.2, Active / Compute / Combine), with a
 * software grid barrier between iterations that cannot deadlock because the
 * grid is sized to co-residency (Sec. 5, "Compiler-based deadlock free
 * barrier", Eq. 1) and that times out instead of hanging.
 *
 * Conventions shared by every entry point
 *   - Status codes only (simdx_status); nothing throws across the ABI.
 *   - Vertex ids are int32 in [0, n).  Graph arrays are CSR (Sec. 6,
 *     "Storage Format"): offsets[n+1] (int32 or int64, non-decreasing,
 *     offsets[0] = 0) and indices[e] (int32).
 *   - Output buffers are DEVICE memory owned by the caller and must hold n
 *     elements (k*n for batched calls).  The library writes every element.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream).  `stats`, when non-NULL, is HOST memory written by a
 *     host function enqueued on the same stream: it is valid once the stream
 *     has been synchronised.  Errors detected on the device (barrier time
 *     out) are reported in stats->status and by simdx_graph_last_status().
 *   - A graph owns one device workspace, so calls on the same graph must not
 *     overlap in time: issue them on one stream or synchronise in between.
 *     Different graphs are independent.
 *   - The library allocates device memory only in simdx_graph_create,
 *     simdx_graph_set_config (when a larger workspace is needed) and the
 *     batch / server entry points that say so; the algorithm calls allocate
 *     nothing.
 *   - CUDA graphs: simdx_bfs, simdx_sssp, simdx_kcore, simdx_kcore_decompose,
 *     simdx_kcore_batch, simdx_pagerank, simdx_bfs_batch, simdx_sssp_batch
 *     (groups of up to 64 sources) and simdx_bfs_multi can be captured into
 *     a CUDA graph (stream capture on `stream`) and replayed, each launch a
 *     cooperative kernel node (in clusters where small_frontier puts it
 *     there), when
 *     (a) stats is NULL (a captured call with stats returns EUNSUPPORTED),
 *     (b) a call of the same kind ran on the graph outside the capture
 *     before (it allocates the batch state; for simdx_bfs_multi with at
 *     least as many roots), and (c) the replays do not overlap other calls
 *     on the same graph.  Sources are kernel parameters, so a replay runs
 *     the captured query; simdx_bfs_multi stages its roots in pinned memory
 *     that a replay reads again, i.e. it replays the roots of the graph's
 *     latest captured simdx_bfs_multi call.
 */
#ifndef SIMDX_H
#define SIMDX_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SIMDX_API __attribute__((visibility("default")))
#else
#define SIMDX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIMDX_OK = 0,
    SIMDX_EINVAL = 1,             /* bad argument (range, NULL, size)           */
    SIMDX_ENOMEM = 2,             /* device or pinned host allocation failed    */
    SIMDX_ECUDA = 3,              /* a CUDA runtime call failed                 */
    SIMDX_EBARRIER_TIMEOUT = 4,   /* a grid-barrier wait ran out (device side)  */
    SIMDX_EUNSUPPORTED = 5,       /* valid request this build does not support  */
    SIMDX_EBUSY = 6,              /* resource in use / queue full               */
    SIMDX_ENOTREADY = 7           /* result not ready yet (server poll)         */
} simdx_status;

/* Graph in CSR form (Sec. 6 "Storage Format").  `e` = number of directed
 * edge entries = offsets[n]. */
typedef struct {
    int64_t n;
    int64_t e;
    int32_t offset_bits;     /* 32 or 64 */
    const void *offsets;     /* [n+1] int32 or int64 */
    const int32_t *indices;  /* [e] */
} simdx_csr;

/* simdx_graph_create flags */
#define SIMDX_INPUT_HOST 1u  /* arrays are host memory; the library copies them */
#define SIMDX_BORROW     2u  /* device arrays are used in place, not copied;
                                the caller keeps them alive until destroy     */

/* Per-call statistics, written to host memory when the stream reaches the
 * end of the call. */
typedef struct {
    int32_t status;          /* simdx_status of the device run              */
    int32_t iterations;      /* BSP iterations (PageRank: rank updates)     */
    int32_t push_iters;      /* iterations computed in push direction       */
    int32_t pull_iters;      /* iterations computed in pull direction       */
    int32_t ballot_iters;    /* iterations whose lists came from the ballot
                                filter (online filter overflowed or forced)  */
    int32_t online_iters;    /* iterations whose lists came from the online
                                filter                                       */
    int32_t phases;          /* grid barriers passed                        */
    int32_t grid_ctas;       /* CTAs of the persistent launch (Eq. 1)       */
    int64_t edges_visited;   /* edge entries read by compute                */
    int64_t frontier_sum;    /* sum over iterations of active vertices      */
    double last_l1;          /* PageRank: L1 change of the last iteration   */
    int32_t launches;        /* kernel launches the call made (fusion knob,
                                batch groups, WCC's two launches)           */
    int32_t reserved32;
    int64_t reserved[3];
} simdx_stats;

/* Tuning knobs (defaults in brackets).  BFS, SSSP, k-core, coreness and
 * component results are the same under every setting; the PageRank knobs
 * (pr_*, and the CTAs per SM, which set the summation order) change its
 * result only within the stated tolerance. */
typedef struct {
    int32_t small_max;       /* degree < small_max -> thread list [32]   (Sec. 4 "Classification") */
    int32_t med_max;         /* degree < med_max   -> warp list   [512]  (Sec. 4 finds this
                                separator insensitive in [128, 2048]) */
    int32_t huge_min;        /* degree >= huge_min -> cut into chunks of huge_min edges dealt
                                round-robin over all CTAs (push: smaller chunks when the
                                batch would not fill the grid); CTA list below [4096] */
    int32_t bin_per_thread;  /* online-filter overflow threshold per thread [64] (Sec. 4
                                "Overflow thresholds"); 0 forces the ballot filter */
    int32_t direction;       /* 0 auto, 1 push only, 2 pull only [0] (Sec. 5); SSSP's
                                automatic choice is push (pull is forced by 2) */
    int32_t filter;          /* 0 JIT (online, ballot on overflow), 2 ballot only [0] (Sec. 4) */
    float alpha;             /* BFS push->pull when frontier edges > unexplored edges / alpha [14] */
    float beta;              /* BFS pull->push when frontier vertices < n / beta [24] */
    float kcore_alpha;       /* k-core pull when removed-vertex edges > alive edges / kcore_alpha [8] */
    uint32_t delta;          /* SSSP delta-stepping bucket width, 0 = unbounded [32 in
                                simdx_config_default; a graph with weights starts at
                                16 x its largest weight] */
    int32_t ctas_per_sm;     /* 0 = occupancy maximum (Eq. 1); else clamp [0] */
    int32_t barrier_timeout_ms; /* grid-barrier wait limit [2000] */
    int32_t debug_skip_cta;  /* test knob: this CTA skips barrier arrival number
                                debug_skip_phase (-1 = off) [-1] */
    int32_t debug_skip_phase;
    int32_t batch_group;     /* simdx_sssp_batch: copies per persistent launch; 0 = as many
                                as keep one launch's distances within 128 MB [0] */
    int32_t fusion;          /* simdx_bfs / simdx_sssp kernel fusion (Sec. 5, Table 2) [0]:
                                0 all fusion: every iteration in one persistent launch;
                                1 selective (push-pull) fusion: one launch per run of
                                consecutive iterations in one direction, each from a kernel
                                compiled for that direction alone (BFS: push, pull, push =
                                3 launches; SSSP computes in one direction, so 1 launch);
                                2 no fusion: one launch per iteration.  Modes 1 and 2 wait
                                on the stream between launches (the host reads whether the
                                run finished and which direction comes next), so they
                                cannot be captured (EUNSUPPORTED while capturing).  Results
                                are identical in every mode. */
    float pr_alpha;          /* simdx_pagerank switch from pull to push (Sec. 6 "PageRank"):
                                after pull iteration t >= 2, push once the L1 change
                                contracts slowly (L1_t >= pr_rho * L1_{t-1}) and the
                                vertices whose change exceeds pr_theta * L1_{t-1} / n have
                                fewer than E / pr_alpha out-edges; 0 = pull only [8] */
    float pr_theta;          /* push threshold, in units of the mean pending change [2] */
    float pr_rho;            /* slowest pull contraction that still keeps pulling [0.6] */
    int32_t sssp_combine;    /* simdx_sssp push combine (Sec. 3.2) [0]: 0 atomicMin; 1 plain
                                stores (no atomics; a racing smaller value may be overwritten),
                                then pull sweeps over every vertex until none lowers a distance
                                (exact; symmetric graphs, all fusion, push; else EUNSUPPORTED).
                                Trace records mark plain-store iterations with bit 17 and the
                                sweeps with bit 18. */
    int32_t sssp_batch_width;  /* simdx_sssp_batch: sources per group of the shared-edge batch,
                                8, 16, 32 or 64; 0 = 32 [0]; a smaller batch uses the
                                narrowest of these that holds it (groups run one after
                                another inside one launch per 64 sources) */
    int32_t pr_row_cost;     /* simdx_pagerank: cost of finishing a row, in in-edges, in the
                                model that cuts the in-edges into equal-cost warp ranges;
                                0 = 4 [0] (changes the summation order's split, so results
                                may differ in the last bits; a given setting is deterministic) */
    int32_t stage_edges;     /* simdx_bfs / simdx_sssp (all fusion, push): 1 = the edge ranges
                                of CTA-class tasks and grid chunks are staged in shared memory
                                by the bulk copy engine (cp.async.bulk into two 8 KB buffers,
                                completion on an mbarrier), the next buffer's copy in flight
                                while the CTA relaxes the current one; 0 = plain loads [0] */
    int32_t pr_recut;        /* simdx_pagerank: after this many iterations, re-cut the warp
                                ranges of the in-edge walk so that every warp's share of the
                                walk time measured in the last iteration is equal; 0 = keep the
                                cost-model cut [0].  The summation order then follows a
                                measured cut: results stay within tolerance but may differ in
                                the last bits from run to run. */
    int32_t small_frontier;  /* simdx_bfs (all fusion): 1 = while a push frontier holds at most
                                4096 vertices and 65536 edges, its levels run on the first
                                thread-block cluster (16 CTAs, the frontier in distributed shared
                                memory, a cluster barrier per level) while the other CTAs wait;
                                the launch is then in clusters of 16 (a few CTAs fewer fit).
                                0 = every level on the whole grid.  2 [default] = 1 for graphs
                                whose largest out-degree is at most 64 (meshes, grids, road
                                networks: many small levels), else 0.  Trace records of such
                                levels carry bit 19; in a BFS record words 6 and 7 are the SM clock
                                cycles of the slowest CTA's walk and of CTA 0's counter
                                publication plus cluster barrier, in a coreness record CTA 0's
                                cycles in level scans since the previous record and the slowest
                                CTA's push walk.  simdx_kcore_decompose: 0 = every step on the
                                grid; 1 = the levels whose remaining vertices fit the cluster
                                (at most 65536) in a second launch in clusters, small steps and
                                level scans on the cluster, the densest core's push in a third,
                                plain launch; 2 = 1 for graphs of at most 2^22 vertices.
                                simdx_sssp (single source, all fusion, push): 1 = push
                                iterations whose frontier below the bucket bound fits run on
                                the cluster; 0 and 2 = the grid. */
    int32_t reserved[5];
} simdx_config;

typedef struct simdx_graph simdx_graph;
typedef struct simdx_server simdx_server;

/* ------------------------------------------------------------------ misc */
SIMDX_API const char *simdx_strerror(int status);
SIMDX_API int simdx_version(void);

/* Text of the last failing CUDA runtime call in this thread ("" if none);
 * explains SIMDX_ECUDA / SIMDX_ENOMEM. */
SIMDX_API const char *simdx_last_cuda_error(void);

/* Default knob values. */
SIMDX_API void simdx_config_default(simdx_config *cfg);

/* Eq. 1 (Sec. 5): #CTA = floor(regs_per_sm / (regs_per_thread *
 * threads_per_cta)) * n_sm.  Host arithmetic only (no GPU needed); the
 * launches themselves use the CUDA occupancy calculator, which also counts
 * shared memory and block limits.  Returns -1 on non-positive input. */
SIMDX_API int64_t simdx_eq1_ctas(int64_t regs_per_sm, int64_t regs_per_thread,
                       int64_t threads_per_cta, int64_t n_sm);

/* ----------------------------------------------------------------- graph */
/* Build a device-resident graph (Sec. 6 "Storage Format": CSR out-edges;
 * CSC in-edges for directed graphs).
 *   csr      out-neighbour CSR (required).
 *   csc      in-neighbour CSR of a directed graph, or NULL for a symmetric
 *            graph (the CSR is then used for both directions).
 *   weights  uint32[e] in CSR order, or NULL (SSSP then fails EINVAL).
 *   flags    SIMDX_INPUT_HOST, SIMDX_BORROW (not both).
 *   stream   copies are issued on it; the call returns after they finish.
 * Ownership: the library copies the arrays unless SIMDX_BORROW is given.
 * Errors: EINVAL (NULL, n < 0, e != offsets[n] when checkable, bad
 * offset_bits, n >= 2^31), ENOMEM, ECUDA.  *out is NULL on failure. */
SIMDX_API int simdx_graph_create(const simdx_csr *csr, const simdx_csr *csc,
                       const uint32_t *weights, uint32_t flags, void *stream,
                       simdx_graph **out);
SIMDX_API int simdx_graph_destroy(simdx_graph *g);

/* Size, edge count and the persistent grid (CTAs) used by this graph. */
SIMDX_API int simdx_graph_info(const simdx_graph *g, int64_t *n, int64_t *e,
                     int32_t *grid_ctas, int32_t *threads_per_cta);

/* Read / replace the tuning knobs (may reallocate the workspace). */
SIMDX_API int simdx_graph_get_config(const simdx_graph *g, simdx_config *cfg);
SIMDX_API int simdx_graph_set_config(simdx_graph *g, const simdx_config *cfg);

/* Status of the last device run on this graph (synchronises `stream`). */
SIMDX_API int simdx_graph_last_status(simdx_graph *g, void *stream);

/* Per-iteration trace of the last run on this graph (synchronises `stream`).
 * Each record is 8 int64: {direction (1 push, 2 pull) | filter << 8
 * (1 online, 2 ballot) | dense << 16 (SSSP: the iteration only lowered
 * distances, and the next filter scans every vertex), active vertices, active edges, level / bucket bound,
 * %globaltimer ns at the iteration's start and at its end (as seen by CTA 0),
 * and two algorithm-specific words: for BFS the end of the main compute phase
 * and the number of high in-degree pull candidates; for PageRank's pull the
 * slowest CTA's time in its phases (ns, 32 bits each); 0 for the others,
 * whose per-class timing was dropped (it cost 3.5 % of the grid SSSP), and
 * the cluster records described under small_frontier}.  A batched SSSP run as several launches (see
 * batch_group) numbers its records across them.  Writes up to `cap` records
 * to host memory `rec` and returns the number of iterations of the run in
 * *count. */
SIMDX_API int simdx_graph_trace(simdx_graph *g, void *stream, int64_t *rec, int64_t cap,
                      int64_t *count);

/* ------------------------------------------------------------ algorithms */
/* BFS (Sec. 6 "BFS"; voting combine, Sec. 3.2): levels[v] = hop distance
 * from src, -1 if unreachable.  Push in the first and last levels, pull in
 * between (Sec. 5).  levels: device int32[n].  Errors: EINVAL (src out of
 * range, NULL levels). */
SIMDX_API int simdx_bfs(simdx_graph *g, int32_t src, int32_t *levels, simdx_stats *stats,
              void *stream);

/* SSSP (Sec. 2.1, Sec. 3.3; aggregation combine = min): dist[v] = length
 * of a shortest path from src with the graph's uint32 weights, UINT32_MAX
 * if unreachable.  Delta-stepping: vertices whose distance changed and is
 * below the current bucket bound are active (Sec. 3.3); the bucket width is
 * the `delta` knob (a graph starts at 16 x its largest weight).  Push by
 * default; a push iteration whose task lists hold over 1/16 of the edges
 * only lowers distances, and the filter after it scans every vertex.
 * direction = 2 forces pull iterations (symmetric graphs: every vertex
 * takes the min over its frontier in-neighbours, Sec. 5).  Path
 * lengths must stay below UINT32_MAX.  dist: device uint32[n].  Errors:
 * EINVAL (no weights, src out of range, NULL dist). */
SIMDX_API int simdx_sssp(simdx_graph *g, int32_t src, uint32_t *dist, simdx_stats *stats,
               void *stream);

/* k-core (Sec. 6 "k-Core"): repeatedly deletes vertices of degree < k;
 * in_core[v] = 1 for the vertices of the maximal subgraph whose minimum
 * degree is >= k, else 0.  residual_deg[v] (optional, may be NULL) = number
 * of in-core neighbours of an in-core v, 0 for deleted vertices.  Pull
 * first, push later; a destination is no longer decremented once it is
 * deleted (Sec. 7.1, k-Core).  Needs a symmetric graph.
 * Errors: EINVAL (NULL in_core, directed graph). */
SIMDX_API int simdx_kcore(simdx_graph *g, uint32_t k, uint8_t *in_core,
                uint32_t *residual_deg, simdx_stats *stats, void *stream);

/* k-core decomposition (Sec. 6 "k-Core", run for every k): coreness[v] =
 * the largest k such that v belongs to the k-core (0 for isolated
 * vertices), so simdx_kcore(k) keeps exactly the vertices with coreness >=
 * k.  Persistent launches peel level after level (one on the grid, or,
 * with small_frontier, up to three: see there): at level K every
 * remaining vertex of residual degree <= K is deleted with coreness K, its
 * push decrements its remaining neighbours, and the decrement that takes a
 * neighbour to K deletes it at the same level; a scan of the remaining
 * vertices opens the next level (K + 1, or the smallest remaining degree).
 * Trace records carry K as their level word.  coreness: device uint32[n].
 * Needs a symmetric graph.  Errors: EINVAL (NULL coreness, directed
 * graph). */
SIMDX_API int simdx_kcore_decompose(simdx_graph *g, uint32_t *coreness, simdx_stats *stats,
                                    void *stream);

/* Batched k-core (the k-core of Sec. 6 for several k in one call): for
 * every ks[i], row i of in_core / residual_deg is what simdx_kcore(ks[i])
 * returns -- in_core[i*n + v] = 1 iff v belongs to the ks[i]-core, and
 * residual_deg[i*n + v] = the number of v's neighbours (edges) inside that
 * core for a member, 0 otherwise.  One decomposition (simdx_kcore_decompose,
 * its coreness kept in the graph's workspace) answers every k: v is in the
 * k-core exactly when coreness(v) >= k; two more launches count, per
 * vertex, the neighbours whose coreness reaches each k and write the rows
 * (a warp per vertex of up to 128 edges, a CTA per vertex of more).
 * ks: host uint32[nk], any order, repeats allowed, 1 <= nk <= 64; in_core:
 * device uint8[nk * n]; residual_deg: device uint32[nk * n] or NULL (not
 * written).  Needs a symmetric graph.  Errors: EINVAL (NULL ks or in_core,
 * nk outside [1, 64], directed graph). */
SIMDX_API int simdx_kcore_batch(simdx_graph *g, const uint32_t *ks, int32_t nk, uint8_t *in_core,
                                uint32_t *residual_deg, simdx_stats *stats, void *stream);

/* Weakly connected components (Sec. 3.2 lists WCC with the voting
 * algorithms): label[v] = the smallest vertex id of v's component, so two
 * vertices share a label exactly when a path joins them.  Two launches on
 * `stream`: a BFS from a vertex of largest degree (chosen when the graph is
 * created) labels its component with the component's smallest id; then
 * min-label propagation on the SSSP path runs over the vertices it did not
 * reach (each starts with its own id; a push offers the label to every
 * neighbour, min combine), ending when no label changes.  Stats and trace
 * records cover both launches.  label: device uint32[n].  Needs a
 * symmetric graph.  Errors: EINVAL (NULL label, directed graph). */
SIMDX_API int simdx_wcc(simdx_graph *g, uint32_t *label, simdx_stats *stats, void *stream);

/* PageRank (Sec. 6 "PageRank"; aggregation combine = sum, pull):
 *   x_0 = 1/n;  x_{t+1}(v) = (1-d)/n + d*(sum_{u in N_in(v)} x_t(u)/outdeg(u)
 *                                         + D_t/n),
 * D_t = rank on out-degree-0 vertices.  Stops after the first iteration
 * whose L1 change is < l1_tol, or after max_iter iterations.  FP32 ranks;
 * per-vertex sums in FP32 in a fixed order (cross-tile parts carried as a
 * TwoSum pair, cross-warp parts added in FP64); the L1 and dangling sums in
 * 2^-60 fixed point, whose total does not depend on order: results are
 * identical run to run for a given grid.  rank: device float[n].
 * Errors: EINVAL (NULL rank, damping outside [0,1), max_iter < 0). */
SIMDX_API int simdx_pagerank(simdx_graph *g, float damping, float l1_tol, int32_t max_iter,
                   float *rank, simdx_stats *stats, void *stream);

/* ---------------------------------------------------------------- batches */
/* Batched BFS (growth direction (a)): k sources in one persistent launch per
 * 64 sources.  Each vertex keeps a 64-bit visited mask and a 64-bit frontier
 * mask; Compute offers a neighbour's frontier mask and Combine is bitwise OR
 * (a vote combine, Sec. 3.2): the first level pushes from the sources, later
 * levels pull over the vertices some source has not reached (owner writes,
 * no atomics).  srcs: host int32[k] in [0, n).  levels: device int32[k*n],
 * row i = levels from srcs[i] (-1 unreachable), identical to k simdx_bfs
 * calls.  The first call on a graph allocates the batch state (24 bytes per
 * vertex); later calls reuse it.  Errors: EINVAL (k <= 0, source out of
 * range, NULL pointers), ENOMEM. */
SIMDX_API int simdx_bfs_batch(simdx_graph *g, const int32_t *srcs, int32_t k, int32_t *levels,
                              simdx_stats *stats, void *stream);

/* Batched SSSP (growth direction (a)): k sources, one persistent launch per
 * 64 sources.  Inside a launch the sources run in groups of
 * sssp_batch_width (default 32): a group keeps its distances vertex-major
 * (one row of group-width words per vertex) and one task per vertex for all
 * its sources whose distance there changed, so an edge is read once per
 * iteration for the whole group and the relaxations of one edge touch one
 * row (frontier Bellman-Ford per source, min combine by atomicMin).  The 64
 * sources travel as a kernel parameter (the call can be captured into a
 * CUDA graph).  srcs: host int32[k]; dist: device uint32[k*n], row i =
 * distances from srcs[i], identical to k simdx_sssp calls.  The first call
 * (or a wider group) allocates the batch state (4 x width + 16 bytes per
 * vertex); later calls reuse it.  With the batch_group knob > 0 the earlier
 * layout runs instead: virtual graph copies (state id inst * n + v) in groups
 * of at most batch_group copies sharing delta-stepping buckets, one launch
 * per group (about 45 bytes per vertex per copy; needs k * n < 2^31).
 * Errors: EINVAL, ENOMEM. */
SIMDX_API int simdx_sssp_batch(simdx_graph *g, const int32_t *srcs, int32_t k, uint32_t *dist,
                               simdx_stats *stats, void *stream);

/* BFS from several roots at once: every root is at level 0 and levels[v] is
 * the distance to the nearest root.  On a block-diagonal batch of graphs
 * (graphs packed into one CSR with their vertex ids offset) with one root per
 * graph, each graph's slice of levels equals a BFS of that graph alone:
 * growth direction (a)'s many-graphs-in-one-launch.  roots: host int32[k];
 * levels: device int32[n].  The first call (or a larger k) allocates a small
 * device copy of the roots.  Errors: EINVAL, ENOMEM. */
SIMDX_API int simdx_bfs_multi(simdx_graph *g, const int32_t *roots, int32_t k, int32_t *levels,
                              simdx_stats *stats, void *stream);

/* BFS on k separate graphs in one persistent launch (growth direction (a):
 * many graphs of uneven size in one launch; Sec. 6 "BFS" per graph).  The
 * library packs the graphs on the device into one block-diagonal CSR
 * (graph i's ids offset by the vertices of the graphs before it), runs
 * simdx_bfs_multi on the pack with root base_i + srcs[i] per block, and
 * copies block i's levels into levels[i]; no edge joins two blocks, so
 * levels[i] equals simdx_bfs(gs[i], srcs[i]).
 *   gs      k graph objects on the current device (any mix of sizes, offset
 *           widths, symmetric or directed; a graph may appear twice).
 *   srcs    host int32[k], srcs[i] in [0, n_i).
 *   levels  host array of k DEVICE pointers, levels[i] int32[n_i].
 * The pack (a copy of every graph's CSR, 4 bytes per vertex of levels and a
 * graph object over it) is built by the first call for a list and kept with
 * gs[0] (freed when gs[0] is destroyed); later calls with the same list in
 * the same order reuse it, a different list rebuilds it (allocating, and
 * waiting on `stream` while the pack's graph object is created).  Calls
 * whose first graph is the same share the pack: like calls on one graph,
 * they must not overlap in time.  The output pointer table is copied from
 * the caller's host memory, so the call cannot be captured (EUNSUPPORTED
 * while capturing).  Errors: EINVAL (k outside [1, 65535], NULL, a source
 * out of range, a graph on another device, more than 2^31 - 2 vertices in
 * all), ENOMEM, ECUDA. */
SIMDX_API int simdx_bfs_multigraph(simdx_graph *const *gs, const int32_t *srcs, int32_t k,
                                   int32_t *const *levels, void *stream);

/* ---------------------------------------------------------------- serving */
/* Query server over resident graphs (growth direction (b)): continuous
 * batching.  A dispatcher thread keeps `slots` launches in flight on their
 * own streams; whenever a slot is free it takes the oldest waiting query and
 * every waiting query compatible with it (same graph and algorithm: up to 64
 * BFS per bit-parallel launch, up to max_sssp SSSP per batched launch, all
 * k-core queries with the same k share one run) and launches them.  Queries
 * arriving while others run are admitted as soon as a slot frees up; the
 * slots' kernels run concurrently (each slot launches 1/slots of the
 * co-resident CTAs).  Every result equals the same query run alone.
 *   graphs      resident symmetric graphs (not owned; keep them alive and do
 *               not call other entry points on them while the server runs).
 *   mem_budget  device bytes the server may use; the number of slots is
 *               min(max_slots, budget / per-slot cost, CTAs per SM); ENOMEM if
 *               not even one slot fits.  All device memory is allocated here:
 *               serving allocates nothing.
 * Results are written to the `out` pointer given at submit time (device
 * memory or pinned host memory; int32[n] levels for BFS, uint32[n] distances
 * for SSSP, uint8[n] membership for k-core with arg = k). */
#define SIMDX_ALGO_BFS 1
#define SIMDX_ALGO_SSSP 2
#define SIMDX_ALGO_KCORE 3
SIMDX_API int simdx_server_create(simdx_graph *const *graphs, int32_t ng, size_t mem_budget,
                                  int32_t max_slots, int32_t max_sssp, simdx_server **out);
/* Queue one query; *ticket identifies it.  Thread safe.  EINVAL on a bad
 * graph index, algorithm or argument. */
SIMDX_API int simdx_server_submit(simdx_server *s, int32_t graph, int32_t algo, int32_t arg,
                                  void *out, uint64_t *ticket);
/* Non-blocking: *done = 1 and SIMDX_OK (or the query's error) once its result
 * is in `out` (the ticket is then released); SIMDX_ENOTREADY while pending. */
SIMDX_API int simdx_server_poll(simdx_server *s, uint64_t ticket, int32_t *done);
/* Block until the query is answered; releases the ticket. */
SIMDX_API int simdx_server_wait(simdx_server *s, uint64_t ticket);
SIMDX_API int simdx_server_info(simdx_server *s, int32_t *slots, uint64_t *launches,
                                uint64_t *served, uint64_t *queued);
/* Stop the dispatcher, finish launches in flight, free the server. */
SIMDX_API int simdx_server_destroy(simdx_server *s);

/* ------------------------------------------------------------ autotuner */
/* Choose the knobs of simdx_config for one algorithm on one graph by
 * measurement (growth direction (a): degree-class thresholds (Sec. 4
 * "Classification"), overflow threshold (Sec. 4), push/pull switch ratios
 * (Sec. 5), SSSP delta, CTAs per SM (Eq. 1)).  Coordinate descent from the
 * graph's current knobs: two passes over the knobs that apply to `algo`; each
 * candidate runs once untimed and then `reps` times timed with CUDA events on
 * `stream` (median); a candidate replaces the current setting only when it is
 * at least 2 % faster.  The winner is installed with simdx_graph_set_config
 * and returned in *best (and its median time in *best_ms, may be NULL).
 *   algo  SIMDX_ALGO_BFS / SSSP (arg = source vertex), SIMDX_ALGO_KCORE
 *         (arg = k), SIMDX_ALGO_PAGERANK (arg ignored; damping 0.85, L1
 *         tolerance 1e-6).
 *   reps  timed runs per candidate, 1..64.
 * Blocking; allocates one scratch output of 4 n bytes for its duration and
 * reallocates the graph's workspace when a knob that sizes it changes.  Knobs
 * change speed only: BFS, SSSP and k-core results are the same under every
 * setting.  Errors: EINVAL (bad algo, arg or reps), EUNSUPPORTED (SSSP on a
 * graph without weights), or the first error an algorithm call returns. */
#define SIMDX_ALGO_PAGERANK 4
SIMDX_API int simdx_autotune(simdx_graph *g, int32_t algo, int64_t arg, int32_t reps, simdx_config *best,
                             float *best_ms, void *stream);

/* The same tuner for the batched calls (growth direction (a): autotuned bin
 * thresholds for batches): algo SIMDX_ALGO_BFS times simdx_bfs_batch,
 * SIMDX_ALGO_SSSP simdx_sssp_batch and SIMDX_ALGO_BFS_MULTI simdx_bfs_multi,
 * each on the k sources (or roots) `srcs` (host int32[k]).  Knobs tried: the
 * CTAs per SM and degree-class thresholds; for the SSSP batch also the
 * overflow threshold, the bucket width and the copies per launch
 * (batch_group); for the multi-root BFS the BFS knobs.  Blocking; allocates
 * one scratch output (4 n bytes per source, 4 n for the multi-root BFS) for
 * its duration.  Results are the same under every setting.  Errors: EINVAL
 * (bad algo, k, source or reps; k * n >= 2^31 for SSSP), EUNSUPPORTED (SSSP
 * without weights), or the first error a timed call returns. */
#define SIMDX_ALGO_BFS_MULTI 5
SIMDX_API int simdx_autotune_batch(simdx_graph *g, int32_t algo, const int32_t *srcs, int32_t k, int32_t reps,
                                   simdx_config *best, float *best_ms, void *stream);

/* ------------------------------------------------- no-allocation variant */
/* BFS for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a deployment convenience).  Some callers cannot call
 * cudaMalloc: code running inside another runtime's memory pool or under a
 * fixed memory budget, code that must not allocate while a CUDA graph is
 * being captured elsewhere on the device, plugins whose host forbids
 * allocation after start-up.  This entry point allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.  All scratch (task
 * lists, online-filter bins, bitmaps, barrier words) lives in one fixed
 * device array of about 15 MB that every GPU loading the library holds until
 * the process exits.
 *   csr     device CSR of out-edges (offsets int32/int64, indices int32),
 *           symmetric or directed, 1 <= n <= 262144 (2^18) vertices; larger
 *           graphs fail with SIMDX_EINVAL.  Every level is a push level (only
 *           out-edges are read), so no in-edge array is needed.  The CSR is
 *           checked first: the call waits on `stream` for that check.
 *   src     source vertex; levels: device int32[n], written as simdx_bfs
 *           writes it (hop distance, -1 if unreachable).
 * The first call on a device looks up the scratch address on that device
 * (the device must be current); make that first call before any stream
 * capture.  Every call shares the one scratch array and it keeps the last
 * call's contents: calls whose GPU work overlaps (different streams, no
 * synchronisation) race and give wrong results, so serialise them.  Errors
 * raised on the device during the traversal are not reported here; use
 * simdx_bfs on a graph object when that matters. */
SIMDX_API int simdx_bfs_noalloc(const simdx_csr *csr, int32_t src, int32_t *levels,
                                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SIMDX_H */
