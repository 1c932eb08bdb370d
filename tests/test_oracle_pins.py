"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each check below is independent of ``oracle.c``: Floyd-Warshall on a dense
matrix, exhaustive subset / simple-path search on tiny graphs, closed forms
(grid levels, uniform PageRank on regular graphs, the star's two-equation
solution), a dense linear solve of the PageRank fixed point, and invariants
that hold at any size.  Each is chosen so that a dropped term, a wrong index
or an off-by-one in the oracle fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = np.iinfo(np.uint64).max // 4


def dense_weights(g, w=None):
    n = g.n
    m = np.full((n, n), INF, dtype=np.uint64)
    np.fill_diagonal(m, 0)
    for u in range(n):
        for p in range(g.offsets[u], g.offsets[u + 1]):
            v = g.indices[p]
            m[u, v] = min(m[u, v], 1 if w is None else int(w[p]))
    return m


def floyd_warshall(m):
    d = m.copy()
    for k in range(d.shape[0]):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    return d


def small_graphs():
    out = [gg.path(1), gg.path(2), gg.path(7), gg.star(9), gg.complete(6)]
    for seed in range(6):
        n = 5 + 9 * seed
        out.append(gg.random_graph(n, int(1.3 * n), seed=100 + seed))  # sparse, disconnected
        out.append(gg.random_graph(n, 3 * n, seed=200 + seed))
    out.append(gg.from_edges(10, [0, 1, 5, 6], [1, 2, 6, 7]))  # two components + isolated
    return out


# ---------------------------------------------------------------- generator
def test_generator_deterministic_symmetric_simple():
    g1, g2 = gg.rmat(10), gg.rmat(10)
    assert np.array_equal(g1.offsets, g2.offsets) and np.array_equal(g1.indices, g2.indices)
    n = g1.n
    src = np.repeat(np.arange(n), g1.degrees())
    dst = g1.indices
    assert np.all(src != dst), "self loop"
    key = src.astype(np.int64) * n + dst
    assert np.all(np.diff(key) > 0), "adjacency not sorted/unique"
    rev = np.sort(dst.astype(np.int64) * n + src)
    assert np.array_equal(rev, key), "not symmetric"
    assert g1.degrees()[0] == g1.degrees().max(), "vertex 0 should be the hub (no permutation)"
    w = gg.weights(g1, 7, 1, 64)
    assert w.min() >= 1 and w.max() <= 64
    wmap = {(int(a), int(b)): int(c) for a, b, c in zip(src, dst, w)}
    assert all(wmap[(b, a)] == c for (a, b), c in wmap.items()), "weights not per undirected edge"


def test_grid_structure():
    g = gg.grid(5, 7)
    assert g.n == 35 and g.e == 2 * (5 * 6 + 4 * 7)
    deg = g.degrees().reshape(5, 7)
    assert deg[0, 0] == 2 and deg[2, 3] == 4 and deg[0, 3] == 3


# ---------------------------------------------------------------------- BFS
@pytest.mark.parametrize("gi", range(18))
def test_bfs_vs_floyd_warshall(gi):
    g = small_graphs()[gi]
    d = floyd_warshall(dense_weights(g))
    for src in range(0, g.n, max(1, g.n // 5)):
        lev = oracle.bfs(g.offsets, g.indices, src)
        exp = np.where(d[src] >= INF, -1, d[src].astype(np.int64))
        assert np.array_equal(lev.astype(np.int64), exp)


def bfs_invariants(g, src, lev):
    n = g.n
    assert lev[src] == 0
    u = np.repeat(np.arange(n), g.degrees())
    v = g.indices
    lu, lv = lev[u], lev[v]
    both = (lu >= 0) & (lv >= 0)
    assert np.all(np.abs(lu[both] - lv[both]) <= 1)
    assert not np.any((lu >= 0) ^ (lv >= 0)), "reached vertex adjacent to unreached one"
    # every reached v != src has a neighbour one level closer
    has_parent = np.zeros(n, bool)
    sel = (lv >= 0) & (lu == lv - 1)
    has_parent[v[sel]] = True
    reached = lev >= 0
    reached[src] = False
    assert np.all(has_parent[reached])


def test_bfs_invariants_rmat():
    g = gg.rmat(14)
    for src in [0] + list(gg.pick_sources(g, 3, 5)):
        bfs_invariants(g, src, oracle.bfs(g.offsets, g.indices, src))


def test_bfs_grid_closed_form():
    rows, cols = 37, 53
    g = gg.grid(rows, cols)
    lev = oracle.bfs(g.offsets, g.indices, 0).reshape(rows, cols)
    r, c = np.indices((rows, cols))
    assert np.array_equal(lev, r + c)
    s = 11 * cols + 20
    lev = oracle.bfs(g.offsets, g.indices, s).reshape(rows, cols)
    assert np.array_equal(lev, np.abs(r - 11) + np.abs(c - 20))


def test_bfs_rejects_bad_source():
    g = gg.path(3)
    with pytest.raises(ValueError):
        oracle.bfs(g.offsets, g.indices, 3)


# --------------------------------------------------------------------- SSSP
@pytest.mark.parametrize("gi", range(18))
def test_sssp_vs_floyd_warshall(gi):
    g = small_graphs()[gi]
    w = gg.weights(g, 1000 + gi, 1, 64)
    d = floyd_warshall(dense_weights(g, w))
    for src in range(0, g.n, max(1, g.n // 4)):
        dist = oracle.sssp(g.offsets, g.indices, w, src)
        exp = np.where(d[src] >= INF, np.uint64(0xFFFFFFFF), d[src])
        assert np.array_equal(dist.astype(np.uint64), exp)


def simple_path_min(g, w, src):
    """Exhaustive enumeration of simple paths (tiny graphs only)."""
    n = g.n
    adj = {u: [(int(g.indices[p]), int(w[p])) for p in range(g.offsets[u], g.offsets[u + 1])]
           for u in range(n)}
    best = [None] * n

    def dfs(u, acc, seen):
        if best[u] is None or acc < best[u]:
            best[u] = acc
        for v, wt in adj[u]:
            if v not in seen:
                dfs(v, acc + wt, seen | {v})

    dfs(src, 0, {src})
    return best


@pytest.mark.parametrize("seed", range(8))
def test_sssp_vs_simple_paths(seed):
    g = gg.random_graph(8, 14, seed=300 + seed)
    w = gg.weights(g, seed, 1, 9)
    for src in range(g.n):
        dist = oracle.sssp(g.offsets, g.indices, w, src)
        exp = simple_path_min(g, w, src)
        got = [None if x == 0xFFFFFFFF else int(x) for x in dist]
        assert got == exp


def test_sssp_unit_weights_equal_bfs():
    g = gg.rmat(13)
    w = np.ones(g.e, np.uint32)
    for src in [0, 17, 4095]:
        lev = oracle.bfs(g.offsets, g.indices, src)
        dist = oracle.sssp(g.offsets, g.indices, w, src)
        assert np.array_equal(np.where(lev < 0, np.int64(0xFFFFFFFF), lev.astype(np.int64)), dist.astype(np.int64))


def sssp_invariants(g, w, src, dist):
    n = g.n
    u = np.repeat(np.arange(n), g.degrees())
    v = g.indices
    du, dv = dist[u].astype(np.uint64), dist[v].astype(np.uint64)
    fin = du != 0xFFFFFFFF
    assert np.all(dv[fin] <= du[fin] + w[fin]), "triangle inequality"
    tight = np.zeros(n, bool)
    t = fin & (dv == du + w)
    tight[v[t]] = True
    reached = dist != 0xFFFFFFFF
    reached[src] = False
    assert np.all(tight[reached]), "no tight in-edge"
    assert dist[src] == 0


def test_sssp_invariants_rmat():
    g = gg.rmat(13)
    w = gg.weights(g, gg.weight_seed(13), 1, 64)
    for src in [0, 123]:
        sssp_invariants(g, w, src, oracle.sssp(g.offsets, g.indices, w, src))


def test_sssp_grid_unit_closed_form():
    rows, cols = 20, 30
    g = gg.grid(rows, cols)
    dist = oracle.sssp(g.offsets, g.indices, np.ones(g.e, np.uint32), 0).reshape(rows, cols)
    r, c = np.indices((rows, cols))
    assert np.array_equal(dist.astype(np.int64), r + c)


def load_fig1():
    names, edges, facts, active, updated, degree = None, [], [], {}, [], {}
    with open(os.path.join(GOLDEN, "fig1_like_sssp.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "v":
                names = t[1:]
            elif t[0] == "e":
                edges.append((names.index(t[1]), names.index(t[2]), int(t[3])))
            elif t[0] == "fact":
                facts.append((int(t[1]), names.index(t[2]), int(t[3])))
            elif t[0] == "active":
                active[int(t[1])] = sorted(names.index(x) for x in t[2:])
            elif t[0] == "updated":
                updated.append((int(t[1]), names.index(t[2])))
            elif t[0] == "degree":
                degree[names.index(t[1])] = int(t[2])
    return names, edges, facts, active, updated, degree


def test_sssp_fig1_like_example():
    names, edges, facts, active, updated, degree = load_fig1()
    n = len(names)
    assert n == 9 and len(edges) == 10
    g = gg.from_edges(n, [e[0] for e in edges], [e[1] for e in edges])
    wmap = {}
    for a, b, wt in edges:
        wmap[(a, b)] = wmap[(b, a)] = wt
    src = np.repeat(np.arange(n), g.degrees())
    w = np.array([wmap[(int(a), int(b))] for a, b in zip(src, g.indices)], np.uint32)
    for v, k in degree.items():
        assert g.degrees()[v] == k
    hist = oracle.sssp_bsp(g.offsets, g.indices, w, 0)
    for it, v, dv in facts:
        assert hist[it - 1][v] == dv
    prev = np.full(n, 0xFFFFFFFF, np.uint32)
    prev[0] = 0
    changed = []
    for h in hist:
        changed.append(sorted(np.nonzero(h != prev)[0].tolist()))
        prev = h
    for it, lst in active.items():          # active at iteration `it` = changed in it-1
        assert changed[it - 2] == lst
    for it, v in updated:
        assert v in changed[it - 1]
    final = oracle.sssp(g.offsets, g.indices, w, 0)
    assert np.array_equal(hist[-1], final)
    fw = floyd_warshall(dense_weights(g, w))[0]
    assert np.array_equal(final.astype(np.uint64), fw)


# ------------------------------------------------------------------- k-core
def kcore_bruteforce(g, k):
    """Largest vertex subset whose induced minimum degree is >= k (unique)."""
    n = g.n
    nb = [set(g.indices[g.offsets[u]:g.offsets[u + 1]].tolist()) for u in range(n)]
    best = frozenset()
    for mask in range(1 << n):
        s = [u for u in range(n) if mask >> u & 1]
        if len(s) <= len(best):
            continue
        ss = set(s)
        if all(len(nb[u] & ss) >= k for u in s):
            best = frozenset(s)
    # uniqueness: every qualifying set is contained in the best one
    return best


@pytest.mark.parametrize("seed", range(6))
def test_kcore_vs_exhaustive(seed):
    g = gg.random_graph(12 + seed % 3, 30 + 3 * seed, seed=400 + seed)
    core = oracle.coreness(g.offsets, g.indices)
    for k in range(0, 7):
        inc, res = oracle.kcore(g.offsets, g.indices, k)
        exp = kcore_bruteforce(g, k)
        assert set(np.nonzero(inc)[0].tolist()) == set(exp)
        assert np.array_equal(inc.astype(bool), core >= k)
        for u in range(g.n):
            nbr = g.indices[g.offsets[u]:g.offsets[u + 1]]
            assert res[u] == (int(inc[nbr].sum()) if inc[u] else 0)


def test_kcore_special_cases_and_invariants():
    g = gg.rmat(13)
    deg = g.degrees()
    inc1, _ = oracle.kcore(g.offsets, g.indices, 1)
    assert np.array_equal(inc1.astype(bool), deg > 0)
    incbig, _ = oracle.kcore(g.offsets, g.indices, int(deg.max()) + 1)
    assert incbig.sum() == 0
    for k in (16, 32):
        inc, res = oracle.kcore(g.offsets, g.indices, k)
        assert inc.sum() > 0
        u = np.repeat(np.arange(g.n), deg)
        cnt = np.bincount(u, weights=inc[g.indices], minlength=g.n)
        assert np.all(cnt[inc.astype(bool)] >= k)
        assert np.array_equal(res, np.where(inc, cnt, 0).astype(np.uint32))
    assert oracle.kcore(gg.complete(6).offsets, gg.complete(6).indices, 5)[0].sum() == 6
    assert oracle.kcore(gg.complete(6).offsets, gg.complete(6).indices, 6)[0].sum() == 0


def test_coreness_vs_bruteforce():
    g = gg.random_graph(13, 40, seed=77)
    core = oracle.coreness(g.offsets, g.indices)
    for v in range(g.n):
        kv = max(k for k in range(0, 13) if v in kcore_bruteforce(g, k) or k == 0)
        assert core[v] == kv


# ------------------------------------------------------------------- WCC
def reach_closure(g):
    """Boolean reachability matrix (reflexive) by Floyd-Warshall on 0/1."""
    n = g.n
    r = np.eye(n, dtype=bool)
    for u in range(n):
        r[u, g.indices[g.offsets[u]:g.offsets[u + 1]]] = True
    for m in range(n):
        r |= np.outer(r[:, m], r[m, :])
    return r


@pytest.mark.parametrize("gi", range(len(small_graphs())))
def test_wcc_vs_reachability(gi):
    g = small_graphs()[gi]
    lab = oracle.wcc(g.offsets, g.indices)
    r = reach_closure(g)
    for v in range(g.n):
        assert lab[v] == np.nonzero(r[v])[0].min(), (g.name, v)


def test_wcc_invariants_and_closed_forms():
    g = gg.rmat(13)
    lab = oracle.wcc(g.offsets, g.indices).astype(np.int64)
    v = np.arange(g.n)
    assert np.all(lab <= v) and np.array_equal(lab[lab], lab)
    u = np.repeat(v, g.degrees())
    assert np.array_equal(lab[u], lab[g.indices])  # both ends of every edge agree
    for s in (0, 5, int(np.argmax(g.degrees())), g.n - 1):
        reached = oracle.bfs(g.offsets, g.indices, s) >= 0
        assert np.array_equal(reached, lab == lab[s])
    assert np.all(oracle.wcc(gg.grid(7, 9).offsets, gg.grid(7, 9).indices) == 0)
    e = gg.random_graph(40, 0, seed=1)
    assert np.array_equal(oracle.wcc(e.offsets, e.indices), np.arange(40, dtype=np.uint32))


def test_coreness_invariants_rmat():
    """At R-MAT scale: the k-core (queue peeling) is exactly {coreness >= k}
    for every k up to the largest coreness, each vertex of coreness c has at
    least c neighbours of coreness >= c, and isolated vertices have 0."""
    g = gg.rmat(12)
    core = oracle.coreness(g.offsets, g.indices).astype(np.int64)
    deg = g.degrees()
    assert np.all(core[deg == 0] == 0) and np.all(core <= deg)
    for k in range(0, int(core.max()) + 2):
        inc, _ = oracle.kcore(g.offsets, g.indices, k)
        assert np.array_equal(inc.astype(bool), core >= k), k
    u = np.repeat(np.arange(g.n), deg)
    strong = np.bincount(u, weights=(core[g.indices] >= core[u]), minlength=g.n)
    assert np.all(strong >= core)


def test_kcore_residual_from_coreness():
    """The identity the batched k-core computes from one decomposition: the
    k-core's residual degree of a member v is the number of its neighbours
    u with min(coreness(u), coreness(v)) >= k, and 0 outside the core --
    checked against the peeling oracle for every k on R-MAT 12, a grid and
    a star (the peeling and the decomposition are separate programs)."""
    for g in (gg.rmat(12), gg.grid(20, 30), gg.star(40)):
        core = oracle.coreness(g.offsets, g.indices).astype(np.int64)
        deg = g.degrees()
        u = np.repeat(np.arange(g.n), deg)
        m = np.minimum(core[u], core[g.indices])
        for k in range(0, int(core.max()) + 2):
            inc, res = oracle.kcore(g.offsets, g.indices, k)
            want = np.bincount(u, weights=(m >= k), minlength=g.n).astype(np.int64)
            want[core < k] = 0
            assert np.array_equal(inc.astype(bool), core >= k), (g.name, k)
            assert np.array_equal(res.astype(np.int64), want), (g.name, k)


# ----------------------------------------------------------------- PageRank
def pagerank_dense(g, d):
    """Fixed point of the PageRank map by a dense FP64 linear solve."""
    n = g.n
    deg = g.degrees().astype(np.float64)
    P = np.zeros((n, n))
    for u in range(n):
        for p in range(g.offsets[u], g.offsets[u + 1]):
            P[g.indices[p], u] += 1.0 / deg[u]
    dang = (deg == 0).astype(np.float64)
    A = np.eye(n) - d * P - d / n * np.outer(np.ones(n), dang)
    return np.linalg.solve(A, np.full(n, (1 - d) / n))


@pytest.mark.parametrize("gi", range(18))
def test_pagerank_vs_dense_solve(gi):
    g = small_graphs()[gi]
    if g.n == 0:
        return
    x, it, l1 = oracle.pagerank(g.offsets, g.indices, tol=1e-15, max_iter=5000)
    exp = pagerank_dense(g, 0.85)
    assert abs(x.sum() - 1.0) < 1e-12
    assert np.max(np.abs(x - exp)) < 1e-12


def test_pagerank_fixed_iterations_match_matrix_power():
    g = gg.random_graph(40, 70, seed=9)
    n, d = g.n, 0.85
    deg = g.degrees().astype(np.float64)
    x = np.full(n, 1.0 / n)
    for t in range(1, 8):
        contrib = np.where(deg > 0, x / np.maximum(deg, 1), 0.0)
        s = np.zeros(n)
        np.add.at(s, g.indices, np.repeat(contrib, g.degrees()))
        x = (1 - d) / n + d * (s + x[deg == 0].sum() / n)
        got, it, _ = oracle.pagerank(g.offsets, g.indices, fixed_iter=t)
        assert it == t
        assert np.max(np.abs(got - x)) < 1e-15


def test_pagerank_closed_forms():
    d = 0.85
    for g in (gg.complete(7), gg.from_edges(6, list(range(6)), [(i + 1) % 6 for i in range(6)])):
        x, _, _ = oracle.pagerank(g.offsets, g.indices, tol=1e-15)
        assert np.allclose(x, 1.0 / g.n, rtol=0, atol=1e-15)
    n = 11
    g = gg.star(n)
    x, _, _ = oracle.pagerank(g.offsets, g.indices, tol=1e-16, max_iter=10000)
    xl = (1 + d / (n - 1)) / (n * (1 + d))
    xc = (1 - d) / n + d * (n - 1) * xl
    assert abs(x[0] - xc) < 1e-13 and np.all(np.abs(x[1:] - xl) < 1e-13)


def test_pagerank_stop_rule():
    g = gg.rmat(12)
    x, it, l1 = oracle.pagerank(g.offsets, g.indices, tol=1e-6)
    assert l1 < 1e-6
    _, _, l1_prev = oracle.pagerank(g.offsets, g.indices, fixed_iter=it - 1)
    assert l1_prev >= 1e-6
    assert abs(x.sum() - 1) < 1e-9


# ------------------------------------------------- parallel timing variants
# The OpenMP variants time the CPU baseline on every host core.  Each must
# give the single-threaded definition's result element for element (they are
# pinned through it, not through themselves).
PAR_GRAPHS = [lambda: gg.path(1), lambda: gg.path(50), lambda: gg.star(40), lambda: gg.complete(9),
              lambda: gg.grid(37, 23), lambda: gg.from_edges(10, [0, 1, 5, 6], [1, 2, 6, 7]),
              lambda: gg.random_graph(900, 5000, seed=7), lambda: gg.rmat(13)]


@pytest.mark.parametrize("gi", range(len(PAR_GRAPHS)))
def test_parallel_variants_equal_definitions(gi):
    g = PAR_GRAPHS[gi]()
    deg = g.degrees()
    for s in sorted({0, g.n - 1, int(np.argmax(deg))}):
        assert np.array_equal(oracle.bfs_par(g.offsets, g.indices, s), oracle.bfs(g.offsets, g.indices, s))
    for k in (0, 1, 2, 3, 5, 16):
        a, b = oracle.kcore(g.offsets, g.indices, k), oracle.kcore_par(g.offsets, g.indices, k)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for kw in (dict(fixed_iter=7), dict(tol=1e-9)):
        a, b = oracle.pagerank(g.offsets, g.indices, **kw), oracle.pagerank_par(g.offsets, g.indices, **kw)
        assert np.array_equal(a[0], b[0]) and a[1:] == b[1:]
    assert oracle.threads() >= 1


# ------------------------------------------------ PageRank, push tail
# pagerank_delta pulls, then pushes the rank changes still above a threshold.
# Pinned by: (a) without a switch it is the pull iteration itself; (b) with
# every changed vertex pushed (theta = 0) each push iteration is one Jacobi
# step, so it stops at the same iteration with the same ranks; (c) with any
# threshold its result is within d / (1 - d) * tol (L1) of the fixed point
# from a dense FP64 solve, which a dropped dangling share, a wrong
# out-degree or a lost residual would break.
def test_pagerank_delta_without_switch_is_pull():
    for g in [gg.rmat(11), gg.grid(30, 20), gg.star(50)]:
        a = oracle.pagerank(g.offsets, g.indices)
        b = oracle.pagerank_delta(g.offsets, g.indices, alpha=0.0)
        assert np.array_equal(a[0], b[0]) and a[1] == b[1] == b[2]


def test_pagerank_delta_full_push_is_jacobi():
    for g in [gg.rmat(11), gg.grid(30, 20), gg.from_edges(10, [0, 1, 5, 6], [1, 2, 6, 7]), gg.path(40)]:
        x, it, pulls, _ = oracle.pagerank_delta(g.offsets, g.indices, alpha=1e-30, theta=0.0, rho_min=0.0)
        j, jt, _ = oracle.pagerank(g.offsets, g.indices)
        assert pulls == min(2, jt) and it == jt
        assert np.abs(x - j).sum() < 1e-12


@pytest.mark.parametrize("theta", [0.5, 1.0, 2.0, 4.0])
@pytest.mark.parametrize("gi", range(18))
def test_pagerank_delta_error_bound(gi, theta):
    g = small_graphs()[gi]
    if g.n == 0:
        return
    d, tol = 0.85, 1e-6
    exp = pagerank_dense(g, d)
    x, it, pulls, l1 = oracle.pagerank_delta(g.offsets, g.indices, d=d, tol=tol, alpha=1e-30, theta=theta, rho_min=0.0)
    assert np.abs(x - exp).sum() <= d / (1 - d) * tol * (1 + 1e-9) + 1e-14
    assert l1 < tol or it == 1000


def test_pagerank_delta_directed_and_grid_bound():
    from gpu_util import directed_graph
    off, idx, ioff, iidx, _ = directed_graph(300, 1500, 4)
    n = off.size - 1
    deg = np.diff(off)
    x_ref, _, _ = oracle.pagerank(ioff, iidx, outdeg=deg, tol=1e-14, max_iter=10000)
    for theta in (1.0, 2.0):
        x, it, pulls, _ = oracle.pagerank_delta(off, idx, ioff, iidx, alpha=1e-30, theta=theta, rho_min=0.0)
        assert pulls == 2 and it > 2
        assert np.abs(x - x_ref).sum() <= 0.85 / 0.15 * 1e-6 + 1e-12
    # the rule itself: on the grid the pull contracts slowly and few vertices
    # are unstable, so it switches; on R-MAT the pull contracts fast, so it
    # keeps pulling
    g = gg.grid(64, 64)
    _, it, pulls, _ = oracle.pagerank_delta(g.offsets, g.indices)
    assert 2 < pulls < it
    for r in (gg.rmat(12), gg.rmat(14)):
        _, it, pulls, _ = oracle.pagerank_delta(r.offsets, r.indices)
        assert pulls == it
    assert n == 300
