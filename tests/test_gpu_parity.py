"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

BFS levels, SSSP distances and k-core membership / residual degrees are
compared bit for bit; PageRank must be within 1e-6 relative L1 of the FP64
oracle run for the same number of iterations, and stop within one
iteration of the oracle's own stopping point.  Every forced path (push
only, pull only, ballot filter only, online-filter overflow, every degree
class, one CTA per SM) must give the same results.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_util import FORCED, assert_pagerank, check_pagerank, make, small_graphs, sources

pytestmark = pytest.mark.gpu

GRAPHS = small_graphs()
GRAPH_IDS = [f"{i}:{g.name}" for i, g in enumerate(GRAPHS)]


@pytest.fixture(scope="module", autouse=True)
def device():
    import torch
    from paper_1812_04070_gb300 import build
    build()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


@pytest.mark.parametrize("mode", list(FORCED))
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_bfs(gi, mode):
    g = GRAPHS[gi]
    G = make(g, bits=32 if gi % 2 else 64, **FORCED[mode])
    for s in sources(g):
        lev = G.bfs(s).cpu().numpy()
        assert np.array_equal(lev, oracle.bfs(g.offsets, g.indices, s)), (g.name, mode, s)
    assert G.last_status() == 0
    G.close()


@pytest.mark.parametrize("mode", list(FORCED))
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_sssp(gi, mode):
    g = GRAPHS[gi]
    w = gg.weights(g, 77 + gi, 1, 64)
    G = make(g, w, bits=64 if gi % 2 else 32, **FORCED[mode])
    for s in sources(g):
        d = G.sssp(s).cpu().numpy().view(np.uint32)
        assert np.array_equal(d, oracle.sssp(g.offsets, g.indices, w, s)), (g.name, mode, s)
    G.close()


@pytest.mark.parametrize("delta", [0, 1, 7, 64, 100000])
def test_sssp_delta(delta):
    g = gg.rmat(12)
    w = gg.weights(g, 5, 1, 1000)
    G = make(g, w, delta=delta)
    for s in sources(g):
        d = G.sssp(s).cpu().numpy().view(np.uint32)
        assert np.array_equal(d, oracle.sssp(g.offsets, g.indices, w, s))
    G.close()


@pytest.mark.parametrize("delta", [0, 1, 64, 1024])
def test_sssp_dense_iterations(delta):
    """From R-MAT's hub the second iteration holds most of the edges: it is
    dense (lowers distances with no pending flags or records), and the scan
    after it must find every improved vertex, flagging those a narrow bucket
    leaves for later."""
    g = gg.rmat(14)
    w = gg.weights(g, 9, 1, 64)
    G = make(g, w, delta=delta)
    d = G.sssp(0).cpu().numpy().view(np.uint32)
    tr = G.trace()
    assert any((int(r[0]) >> 16) & 1 for r in tr), "no dense iteration"
    assert np.array_equal(d, oracle.sssp(g.offsets, g.indices, w, 0))
    srcs = [0, 1, 2, 3]
    G.set_config(batch_group=4)  # the virtual-copy batch shares the dense iterations
    db = G.sssp_batch(srcs).cpu().numpy().view(np.uint32)
    assert any((int(r[0]) >> 16) & 1 for r in G.trace()), "no dense iteration in the batch"
    for i, s in enumerate(srcs):
        assert np.array_equal(db[i], oracle.sssp(g.offsets, g.indices, w, s)), s
    G.close()


@pytest.mark.parametrize("mode", ["default", "ballot", "overflow", "tiny_bins", "all_classes", "one_cta_per_sm",
                                  "grid_only", "cluster_all_classes"])
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_coreness(gi, mode):
    """Coreness equals Batagelj-Zaversnik's; the fixed-k kernel keeps exactly
    the vertices of coreness >= k; the coreness of every vertex with edges is
    a peeling level of the trace (isolated vertices are deleted by a scan,
    with nothing to push), and the levels only rise."""
    g = GRAPHS[gi]
    G = make(g, bits=32 if gi % 2 else 64, **FORCED[mode])
    core = G.coreness().cpu().numpy().view(np.uint32)
    exp = oracle.coreness(g.offsets, g.indices)
    assert np.array_equal(core, exp), (g.name, mode)
    assert G.last_status() == 0
    lev = [int(x) for x in G.trace()[:, 3]]
    has_edges = np.diff(g.offsets) > 0
    assert lev == sorted(lev) and set(lev) == set(int(x) for x in exp[has_edges]), (g.name, mode)
    for k in (1, 3, 16):
        inc, _ = G.kcore(k)
        assert np.array_equal(inc.cpu().numpy() == 1, core >= k), (g.name, mode, k)
    G.close()


@pytest.mark.parametrize("mode", ["default", "ballot", "overflow", "tiny_bins", "all_classes", "one_cta_per_sm"])
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_wcc(gi, mode):
    """Component labels equal the oracle's (smallest id per component)."""
    from paper_1812_04070_gb300 import simdx_stats
    import torch
    g = GRAPHS[gi]
    G = make(g, bits=64 if gi % 2 else 32, **FORCED[mode])
    st = simdx_stats()
    lab = G.wcc(stats=st).cpu().numpy().view(np.uint32)
    torch.cuda.synchronize()
    assert np.array_equal(lab, oracle.wcc(g.offsets, g.indices)), (g.name, mode)
    assert st.status == 0 and G.last_status() == 0
    G.close()


@pytest.mark.parametrize("mode", ["default", "push", "pull", "ballot", "overflow", "all_classes",
                                  "all_classes_pull", "one_cta_per_sm"])
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_kcore(gi, mode):
    g = GRAPHS[gi]
    G = make(g, **FORCED[mode])
    for k in (0, 1, 2, 3, 5, 16):
        inc, res = G.kcore(k)
        einc, eres = oracle.kcore(g.offsets, g.indices, k)
        assert np.array_equal(inc.cpu().numpy(), einc), (g.name, mode, k)
        assert np.array_equal(res.cpu().numpy().view(np.uint32), eres), (g.name, mode, k)
    G.close()


@pytest.mark.parametrize("mode", ["default", "all_classes", "one_cta_per_sm"])
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_pagerank(gi, mode):
    g = GRAPHS[gi]
    G = make(g, **FORCED[mode])
    assert_pagerank(G, g)
    G.set_config(pr_alpha=0.0)  # pull only: the Jacobi iteration throughout
    st, rel = assert_pagerank(G, g)
    assert st.push_iters == 0 and st.launches == 1
    G.close()


# The switch from pull to push (Sec. 6 "PageRank").  Forced early (pr_alpha
# tiny, pr_rho 0: after the second pull) on every graph; with pr_theta = 0
# every changed vertex pushes, which is the Jacobi step, so the result must
# match the oracle's Jacobi iterate of the same count.
@pytest.mark.parametrize("theta", [0.0, 0.5, 2.0, 8.0])
@pytest.mark.parametrize("mode", ["default", "all_classes"])
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_pagerank_push_tail(gi, mode, theta):
    import torch
    from paper_1812_04070_gb300 import simdx_stats
    g = GRAPHS[gi]
    G = make(g, bits=32 if gi % 2 else 64, pr_alpha=1e-30, pr_rho=0.0, pr_theta=theta, **FORCED[mode])
    st, err = assert_pagerank(G, g)
    jt = oracle.pagerank(g.offsets, g.indices)[1]
    if jt > 3 and g.n > 1:
        assert st.pull_iters == 2 and st.push_iters > 0 and st.launches == 2, (st.pull_iters, st.push_iters)
    if theta == 0.0 and st.push_iters > 0:
        ex, _, _ = oracle.pagerank(g.offsets, g.indices, fixed_iter=st.iterations)
        x = G.pagerank().cpu().numpy().astype(np.float64)
        assert np.abs(x - ex).sum() / np.abs(ex).sum() <= 1e-6
        assert abs(st.iterations - jt) <= 1
    a = G.pagerank().clone()
    b = G.pagerank().clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)  # bit-identical run to run
    G.close()


def test_pagerank_switch_rule():
    """Default knobs: on a grid the pull contracts slowly and few vertices are
    unstable, so the run switches after the same pull iterations as the
    oracle's rule; on R-MAT the pull contracts fast and it never switches."""
    from paper_1812_04070_gb300 import simdx_stats
    for g in [gg.grid(64, 64), gg.grid(300, 200)]:
        G = make(g)
        st, err = assert_pagerank(G, g)
        _, it, pulls, _ = oracle.pagerank_delta(g.offsets, g.indices)
        assert st.push_iters > 0 and st.pull_iters == pulls, (st.pull_iters, pulls)
        tr = G.trace()
        assert [int(r[0]) & 0xff for r in tr[:st.iterations]] == [2] * pulls + [1] * st.push_iters
        G.close()
    for g in [gg.rmat(12), gg.rmat(14)]:
        G = make(g)
        st, _ = assert_pagerank(G, g)
        assert st.push_iters == 0
        G.close()


def test_pagerank_deterministic_and_max_iter():
    import torch
    g = gg.rmat(13)
    G = make(g)
    a = G.pagerank().clone()
    b = G.pagerank().clone()
    assert torch.equal(a, b)
    x0 = G.pagerank(max_iter=0).cpu().numpy()
    assert np.all(x0 == np.float32(1.0 / g.n))
    rel, t, _, _ = check_pagerank(G, g, max_iter=3)
    assert t == 3 and rel <= 1e-6
    G.close()


def test_errors_and_validation():
    from paper_1812_04070_gb300 import Graph, SimdxError
    g = gg.path(5)
    G = make(g)
    with pytest.raises(SimdxError):
        G.bfs(5)
    with pytest.raises(SimdxError):
        G.sssp(0)  # no weights
    with pytest.raises(SimdxError):
        G.set_config(med_max=1)
    G.close()
    bad = g.indices.copy()
    bad[0] = 7  # out of range
    with pytest.raises(SimdxError):
        Graph(g.offsets, bad)
    badoff = g.offsets.copy()
    badoff[2] = badoff[3] + 1  # not monotone
    with pytest.raises(SimdxError):
        Graph(badoff, g.indices)


def test_device_input_and_borrow():
    import torch
    from paper_1812_04070_gb300 import Graph
    g = gg.rmat(11)
    off = torch.from_numpy(g.offsets).cuda()
    idx = torch.from_numpy(g.indices).cuda()
    for borrow in (False, True):
        G = Graph(off, idx, borrow=borrow)
        assert np.array_equal(G.bfs(3).cpu().numpy(), oracle.bfs(g.offsets, g.indices, 3))
        G.close()


def test_barrier_timeout_reports_error():
    """A CTA that never arrives makes the others' bounded waits run out; the
    run ends with SIMDX_EBARRIER_TIMEOUT and the context stays usable."""
    from paper_1812_04070_gb300 import simdx, simdx_stats
    import torch
    g = gg.rmat(10)
    G = make(g, debug_skip_cta=3, debug_skip_phase=2, barrier_timeout_ms=300)
    st = simdx_stats()
    G.bfs(0, stats=st)
    torch.cuda.synchronize()
    assert st.status == simdx.EBARRIER_TIMEOUT
    assert G.last_status() == simdx.EBARRIER_TIMEOUT
    G.set_config(debug_skip_cta=-1, debug_skip_phase=-1)
    assert np.array_equal(G.bfs(0).cpu().numpy(), oracle.bfs(g.offsets, g.indices, 0))
    assert G.last_status() == 0
    G.close()


def test_stats_and_trace():
    from paper_1812_04070_gb300 import simdx_stats
    import torch
    g = gg.rmat(14)
    G = make(g)
    st = simdx_stats()
    lev = G.bfs(0, stats=st).cpu().numpy()
    torch.cuda.synchronize()
    assert st.status == 0 and st.iterations == lev.max() + 1
    assert st.push_iters + st.pull_iters == st.iterations
    assert st.pull_iters >= 1  # R-MAT from the hub switches to pull (Sec. 5)
    tr = G.trace()
    assert tr.shape[0] == st.iterations
    assert list(tr[:, 3]) == list(range(st.iterations))
    G.close()


# Kernel fusion (Sec. 5, Table 2): all fusion (one launch), selective push-pull
# fusion (one launch per run of one direction) and no fusion (one launch per
# iteration) must give identical results.
FUSION = {"selective": dict(fusion=1), "none": dict(fusion=2), "none_pull": dict(fusion=2, direction=2),
          "selective_pull": dict(fusion=1, direction=2),
          "none_all_classes": dict(fusion=2, small_max=2, med_max=4, huge_min=8),
          "none_ballot": dict(fusion=2, filter=2)}


@pytest.mark.parametrize("mode", list(FUSION))
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_bfs_sssp_fusion_modes(gi, mode):
    g = GRAPHS[gi]
    w = gg.weights(g, 77 + gi, 1, 64)
    G = make(g, w, bits=32 if gi % 2 else 64, **FUSION[mode])
    for s in sources(g):
        lev = G.bfs(s).cpu().numpy()
        assert np.array_equal(lev, oracle.bfs(g.offsets, g.indices, s)), (g.name, mode, s)
        d = G.sssp(s).cpu().numpy().view(np.uint32)
        assert np.array_equal(d, oracle.sssp(g.offsets, g.indices, w, s)), (g.name, mode, s)
    assert G.last_status() == 0
    G.close()


def test_fusion_launch_counts():
    """Selective fusion launches once per run of consecutive iterations in
    one direction (push, pull, push on R-MAT: 3, as in Table 2); no fusion
    once per iteration; all fusion once.  Iterations and edge counts are the
    same in every mode."""
    from paper_1812_04070_gb300 import simdx_stats
    g = gg.rmat(14)
    w = gg.weights(g, 3, 1, 64)
    G = make(g, w, bits=32)
    st0 = simdx_stats()
    ref = G.bfs(0, stats=st0).cpu().numpy()
    dirs = [int(r[0]) & 0xff for r in G.trace()]
    assert st0.launches == 1 and dirs[0] == 1 and 2 in dirs
    runs = 1 + sum(1 for a, b in zip(dirs, dirs[1:]) if a != b)
    for fusion, want in [(1, runs), (2, len(dirs))]:
        G.set_config(fusion=fusion)
        st = simdx_stats()
        lev = G.bfs(0, stats=st).cpu().numpy()
        import torch
        torch.cuda.synchronize()
        assert np.array_equal(lev, ref)
        assert st.launches == want and st.iterations == st0.iterations, (fusion, st.launches, want)
        assert st.pull_iters == st0.pull_iters and st.edges_visited == st0.edges_visited
        assert [int(r[0]) & 0xff for r in G.trace()] == dirs
    G.set_config(fusion=0)
    sd = simdx_stats()
    d0 = G.sssp(0, stats=sd).cpu().numpy()
    G.set_config(fusion=2)
    sn = simdx_stats()
    d2 = G.sssp(0, stats=sn).cpu().numpy()
    import torch
    torch.cuda.synchronize()
    # the last launch of an SSSP run only finds that no vertex is pending
    assert np.array_equal(d0, d2) and sn.iterations == sd.iterations and sd.launches == 1
    assert sn.launches in (sn.iterations, sn.iterations + 1)
    G.close()


@pytest.mark.parametrize("mode", ["default", "all_classes", "overflow", "ballot", "one_cta_per_sm"])
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_sssp_atomic_free_combine(gi, mode):
    """SSSP push with plain-store min (no atomics) and pull sweeps until no
    distance drops: exact distances; the trace marks the plain-store
    iterations and ends with a sweep that lowered nothing."""
    g = GRAPHS[gi]
    w = gg.weights(g, 77 + gi, 1, 64)
    G = make(g, w, bits=64 if gi % 2 else 32, sssp_combine=1, **FORCED[mode])
    for s in sources(g):
        d = G.sssp(s).cpu().numpy().view(np.uint32)
        assert np.array_equal(d, oracle.sssp(g.offsets, g.indices, w, s)), (g.name, mode, s)
        tr = G.trace()
        flags = [int(r[0]) for r in tr]
        assert (flags[-1] >> 18) & 1 and int(tr[-1][2]) == 0
        assert all(((f >> 17) & 1) for f in flags if (f & 0xff) == 1)
    G.close()


def test_sssp_atomic_free_combine_rejects_directed():
    from paper_1812_04070_gb300 import SimdxError, simdx
    from gpu_util import directed_graph
    from paper_1812_04070_gb300 import Graph
    off, idx, ioff, iidx, w = directed_graph(300, 1500, 4)
    G = Graph(off, idx, weights=w, csc=(ioff, iidx))
    G.set_config(sssp_combine=1)
    with pytest.raises(SimdxError) as e:
        G.sssp(0)
    assert e.value.status == simdx.EUNSUPPORTED
    G.close()


# Bulk-copy staging of CTA-class edge ranges in shared memory (stage_edges):
# the same levels and distances as plain loads, also with tiny class
# thresholds (every task of degree >= 8 walks staged chunks).
STAGED = {"staged": dict(stage_edges=1), "staged_all_classes": dict(stage_edges=1, small_max=2, med_max=4, huge_min=8),
          "staged_one_cta_per_sm": dict(stage_edges=1, ctas_per_sm=1)}


@pytest.mark.parametrize("mode", list(STAGED))
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_bfs_sssp_staged_edges(gi, mode):
    g = GRAPHS[gi]
    w = gg.weights(g, 77 + gi, 1, 64)
    G = make(g, w, bits=32 if gi % 2 else 64, **STAGED[mode])
    for s in sources(g):
        assert np.array_equal(G.bfs(s).cpu().numpy(), oracle.bfs(g.offsets, g.indices, s)), (g.name, mode, s)
        d = G.sssp(s).cpu().numpy().view(np.uint32)
        assert np.array_equal(d, oracle.sssp(g.offsets, g.indices, w, s)), (g.name, mode, s)
    assert G.last_status() == 0
    G.close()


def test_staged_edges_unaligned_index_array():
    """A borrowed index array that is not 16-byte aligned takes the plain
    loads (bulk copies need 16-byte aligned addresses)."""
    import torch
    from paper_1812_04070_gb300 import Graph
    g = gg.rmat(12)
    w = gg.weights(g, 5, 1, 64)
    off = torch.from_numpy(g.offsets).cuda()
    buf = torch.zeros(g.e + 4, dtype=torch.int32, device="cuda")
    buf[1:g.e + 1] = torch.from_numpy(g.indices).cuda()
    idx = buf[1:g.e + 1]
    assert idx.data_ptr() % 16 != 0
    wt = torch.from_numpy(w.view(np.int32)).cuda()
    G = Graph(off, idx, weights=wt, borrow=True)
    G.set_config(stage_edges=1, small_max=2, med_max=4, huge_min=64)
    assert np.array_equal(G.bfs(0).cpu().numpy(), oracle.bfs(g.offsets, g.indices, 0))
    assert np.array_equal(G.sssp(0).cpu().numpy().view(np.uint32), oracle.sssp(g.offsets, g.indices, w, 0))
    G.close()


@pytest.mark.parametrize("recut", [1, 2, 5])
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_pagerank_recut_ranges(gi, recut):
    """Warp ranges re-cut by the measured walk time after `recut` iterations:
    the same parity as the cost-model cut (pull runs within 1e-6 of the FP64
    oracle at the same iteration count; runs that switch to push within their
    bound)."""
    g = GRAPHS[gi]
    G = make(g, bits=32 if gi % 2 else 64, pr_recut=recut)
    assert_pagerank(G, g)
    G.set_config(pr_alpha=0.0)
    st, _ = assert_pagerank(G, g)
    assert st.push_iters == 0
    G.close()


# Small frontiers on one thread-block cluster (small_frontier): the same
# levels as the grid, with the frontier in distributed shared memory.
SMALL = {"small": dict(small_frontier=1), "small_push": dict(small_frontier=1, direction=1),
         "small_all_classes": dict(small_frontier=1, small_max=2, med_max=4, huge_min=8),
         "small_ballot": dict(small_frontier=1, filter=2)}


@pytest.mark.parametrize("mode", list(SMALL))
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_bfs_small_frontier_cluster(gi, mode):
    g = GRAPHS[gi]
    G = make(g, bits=32 if gi % 2 else 64, **SMALL[mode])
    for s in sources(g):
        assert np.array_equal(G.bfs(s).cpu().numpy(), oracle.bfs(g.offsets, g.indices, s)), (g.name, mode, s)
    assert G.last_status() == 0
    G.close()


def test_bfs_small_frontier_levels_and_multi_root():
    """On a grid every frontier is small: the trace marks the cluster levels
    (bit 19) and the statistics count every level.  Every push level runs on
    the cluster (the last levels turn to pull when the frontier's edges
    outweigh the unvisited ones); push-only runs every level there.  A
    multi-root BFS over a block-diagonal pack gives each graph's levels."""
    import torch
    from paper_1812_04070_gb300 import simdx_stats
    g = gg.grid(120, 90)
    want = oracle.bfs(g.offsets, g.indices, 0)
    for direction in (0, 1):
        G = make(g, bits=64, small_frontier=1, direction=direction)
        st = simdx_stats()
        lev = G.bfs(0, stats=st).cpu().numpy()
        torch.cuda.synchronize()
        assert np.array_equal(lev, want)
        assert st.iterations == 120 + 90 - 1 and st.status == 0
        tr = G.trace()
        kind = [int(r[0]) for r in tr]
        assert all((x >> 19) & 1 for x in kind if x & 0xff == 1), direction  # every push level
        if direction == 1:
            assert len(kind) == st.iterations
            # cluster levels: start <= end; walk and barrier cycles recorded
            assert all(r[4] <= r[5] and r[6] > 0 and r[7] > 0 for r in tr)
        G.close()
    graphs, srcs = gg.multigraph_batch(count=12, n_lo=50, n_hi=2000, seed=9)
    packed, bases = gg.pack(graphs)
    roots = [int(x) for x in (srcs.astype(np.int64) + bases[:-1])]
    P = make(packed, bits=32, small_frontier=1)
    lv = P.bfs_multi(roots).cpu().numpy()
    for i, x in enumerate(graphs):
        assert np.array_equal(lv[bases[i]:bases[i + 1]], oracle.bfs(x.offsets, x.indices, int(srcs[i]))), i
    P.close()


def _layered(sizes, seed):
    """A layered graph: each vertex of a layer joins one or two random
    vertices of the layer before (so the BFS from vertex 0 has the layers as
    its frontiers), plus a few edges inside layers."""
    rng = np.random.default_rng(seed)
    first = np.concatenate([[0], np.cumsum(sizes)])
    src, dst = [], []
    for i in range(1, len(sizes)):
        v = np.arange(first[i], first[i + 1])
        for _ in range(2):
            src.append(v)
            dst.append(rng.integers(first[i - 1], first[i], v.size))
        if sizes[i] > 1:
            src.append(rng.integers(first[i], first[i + 1], sizes[i] // 4))
            dst.append(rng.integers(first[i], first[i + 1], sizes[i] // 4))
    return gg.from_edges(int(first[-1]), np.concatenate(src), np.concatenate(dst), "layered")


def test_bfs_small_frontier_wide_and_overflow():
    """Frontiers of several thousand vertices (more than 32 tasks per warp of
    the cluster: both halves of a lane's tasks), and a level in which one CTA
    of the cluster claims more vertices than its buffer holds (a hub whose
    1500 neighbours all fall to the CTA that walks it), which ends the
    episode and resumes it on the grid."""
    g = _layered([1, 40, 3500, 3900, 200, 3000, 64, 1], seed=5)
    for direction in (0, 1):  # push-only walks every layer on the cluster
        G = make(g, bits=64, small_frontier=1, direction=direction)
        assert np.array_equal(G.bfs(0).cpu().numpy(), oracle.bfs(g.offsets, g.indices, 0)), direction
        if direction == 1:
            assert all((int(r[0]) >> 19) & 1 for r in G.trace())
        G.close()
    k = 1500
    kids = 8 * np.arange(1, k + 1)
    src = np.concatenate([np.zeros(k, np.int64), kids, kids + 1])
    dst = np.concatenate([kids, kids + 1, kids + 2])
    g = gg.from_edges(8 * k + 8, src, dst, "skewed")
    for direction in (0, 1):
        G = make(g, bits=32, small_frontier=1, direction=direction)
        assert np.array_equal(G.bfs(0).cpu().numpy(), oracle.bfs(g.offsets, g.indices, 0)), direction
        assert G.last_status() == 0
        G.close()


@pytest.mark.parametrize("small", [0, 1])
def test_coreness_cluster_steps(small):
    """The k-core decomposition with its small steps on one thread-block
    cluster (small_frontier 1, the default's choice for coreness) and without
    (0): the same coreness on a graph whose levels mix large and small
    domains and frontiers (R-MAT 14, hubs) and on a grid (every level
    small); the cluster's push steps carry bit 19 in the trace."""
    for g in (gg.rmat(14), gg.grid(60, 70), _layered([1, 40, 3500, 3900, 200, 3000, 64, 1], seed=6)):
        G = make(g, bits=64, small_frontier=small)
        core = G.coreness().cpu().numpy().view(np.uint32)
        assert np.array_equal(core, oracle.coreness(g.offsets, g.indices)), (g.name, small)
        assert G.last_status() == 0
        flags = [(int(r[0]) >> 19) & 1 for r in G.trace()]
        assert (sum(flags) > 0) == bool(small), (g.name, small)
        G.close()


SSSP_SMALL = {"cluster": dict(small_frontier=1), "cluster_all_classes": dict(small_frontier=1, small_max=2, med_max=4,
                                                                            huge_min=8),
              "cluster_ballot": dict(small_frontier=1, filter=2), "cluster_delta64": dict(small_frontier=1, delta=64),
              "cluster_delta0": dict(small_frontier=1, delta=0)}


@pytest.mark.parametrize("mode", list(SSSP_SMALL))
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_sssp_small_frontier_cluster(gi, mode):
    """Single-source SSSP with its small push frontiers on one thread-block
    cluster: distances equal Dijkstra's on every graph, for narrow, wide
    and unbounded buckets."""
    g = GRAPHS[gi]
    w = gg.weights(g, 77 + gi, 1, 64)
    G = make(g, w, bits=64 if gi % 2 else 32, **SSSP_SMALL[mode])
    for s in sources(g):
        d = G.sssp(s).cpu().numpy().view(np.uint32)
        assert np.array_equal(d, oracle.sssp(g.offsets, g.indices, w, s)), (g.name, mode, s)
    assert G.last_status() == 0
    G.close()


def test_sssp_small_frontier_grid_and_layers():
    """On a grid every push frontier is small: the cluster runs them (trace
    bit 19) and the grid advances the buckets; a layered graph with wide
    layers and a skewed one (a hub whose improvements overflow the claiming
    CTA) hand back and forth."""
    for g, w in ((gg.grid(90, 70), None), (_layered([1, 40, 3500, 3900, 200, 3000, 64, 1], seed=8), None)):
        w = gg.weights(g, 31, 1, 1000)
        G = make(g, w, bits=64, small_frontier=1)
        d = G.sssp(0).cpu().numpy().view(np.uint32)
        assert np.array_equal(d, oracle.sssp(g.offsets, g.indices, w, 0)), g.name
        flags = [(int(r[0]) >> 19) & 1 for r in G.trace()]
        assert sum(flags) > 0, g.name
        G.close()
    k = 1500
    kids = 8 * np.arange(1, k + 1)
    g = gg.from_edges(8 * k + 8, np.concatenate([np.zeros(k, np.int64), kids, kids + 1]),
                      np.concatenate([kids, kids + 1, kids + 2]), "skewed")
    w = gg.weights(g, 32, 1, 64)
    G = make(g, w, bits=32, small_frontier=1)
    assert np.array_equal(G.sssp(0).cpu().numpy().view(np.uint32), oracle.sssp(g.offsets, g.indices, w, 0))
    G.close()


KCORE_BATCH_KS = [16, 0, 1, 2, 3, 5, 32, 1000, 3, 7]


@pytest.mark.parametrize("mode", ["default", "grid_only", "no_resid"])
@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=GRAPH_IDS)
def test_kcore_batch(gi, mode):
    """simdx_kcore_batch: row i equals simdx_kcore(ks[i]) and the oracle's
    peeling for that k (membership and residual degrees), for k values in
    any order with repeats, k = 0 and a k above every coreness."""
    g = GRAPHS[gi]
    knobs = dict(small_frontier=0) if mode == "grid_only" else {}
    G = make(g, bits=32 if gi % 2 else 64, **knobs)
    inc, res = G.kcore_batch(KCORE_BATCH_KS, want_resid=mode != "no_resid")
    inc = inc.cpu().numpy()
    for i, k in enumerate(KCORE_BATCH_KS):
        ei, er = oracle.kcore(g.offsets, g.indices, k)
        assert np.array_equal(inc[i], ei), (g.name, mode, k)
        if res is not None:
            assert np.array_equal(res[i].cpu().numpy().view(np.uint32), er), (g.name, mode, k)
    assert G.last_status() == 0
    G.close()


def test_kcore_batch_limits():
    """64 k values in one call; 0 or 65 values and a directed graph are
    rejected."""
    from paper_1812_04070_gb300 import SimdxError, simdx
    from gpu_util import directed_graph
    from paper_1812_04070_gb300 import Graph
    g = gg.rmat(13)
    G = make(g, bits=32)
    ks = list(range(0, 128, 2))
    inc, res = G.kcore_batch(ks)
    core = oracle.coreness(g.offsets, g.indices)
    for i, k in enumerate(ks):
        assert np.array_equal(inc[i].cpu().numpy(), (core >= k).astype(np.uint8)), k
        assert np.array_equal(res[i].cpu().numpy().view(np.uint32), oracle.kcore(g.offsets, g.indices, k)[1]), k
    for bad in ([], list(range(65))):
        with pytest.raises(SimdxError) as e:
            G.kcore_batch(bad)
        assert e.value.status == simdx.EINVAL
    G.close()
    off, idx, ioff, iidx, _ = directed_graph(300, 1500, 3)
    D = Graph(off, idx, csc=(ioff, iidx))
    with pytest.raises(SimdxError) as e:
        D.kcore_batch([2])
    assert e.value.status == simdx.EINVAL
    D.close()


def test_coreness_cluster_entry_overflow():
    """A hub of 33,000 edges alone in a pending frontier (its leaves went
    first): its pieces of at most 64 edges overflow the one CTA whose share
    it is, so the cluster walks nothing and the grid pushes it; the result
    stays exact."""
    k = 33000
    g = gg.from_edges(k + 1, np.zeros(k, np.int64), np.arange(1, k + 1), "hub")
    for small in (1, 2):
        G = make(g, bits=32, small_frontier=small)
        assert np.array_equal(G.coreness().cpu().numpy().view(np.uint32), oracle.coreness(g.offsets, g.indices))
        assert G.last_status() == 0
        G.close()
