"""GPU parity of the batched entry points (growth direction (a)).

Every row of a batched result must equal the oracle run for that query
alone, and every graph of a packed multi-graph batch must equal the oracle
on that graph alone.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_util import FORCED, make

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def device():
    import torch
    from paper_1812_04070_gb300 import build
    build()
    torch.cuda.set_device(0)


BATCH_GRAPHS = [gg.rmat(12), gg.grid(40, 50), gg.random_graph(900, 1200, seed=3), gg.star(500)]


@pytest.mark.parametrize("gi", range(len(BATCH_GRAPHS)))
@pytest.mark.parametrize("k", [1, 5, 64, 100])
def test_bfs_batch(gi, k):
    g = BATCH_GRAPHS[gi]
    srcs = gg.pick_sources(g, min(k, 60), seed=11 + k)
    srcs = np.resize(srcs, k)  # repeats are allowed
    G = make(g, bits=32 if gi % 2 else 64)
    out = G.bfs_batch(list(srcs)).cpu().numpy()
    for i, s in enumerate(srcs):
        assert np.array_equal(out[i], oracle.bfs(g.offsets, g.indices, int(s))), (g.name, k, i)
    G.close()


SSSP_BATCH_MODES = {**{m: FORCED[m] for m in ["default", "ballot", "overflow", "all_classes", "one_cta_per_sm"]},
                    "width16": dict(sssp_batch_width=16), "width32": dict(sssp_batch_width=32),
                    "width64": dict(sssp_batch_width=64),
                    "width64_all_classes": dict(sssp_batch_width=64, small_max=2, med_max=4, huge_min=8),
                    "virtual_copies": dict(batch_group=4)}


@pytest.mark.parametrize("mode", list(SSSP_BATCH_MODES))
@pytest.mark.parametrize("gi", range(len(BATCH_GRAPHS)))
def test_sssp_batch(gi, mode):
    g = BATCH_GRAPHS[gi]
    w = gg.weights(g, 5 + gi, 1, 64)
    srcs = list(gg.pick_sources(g, 9, seed=7)) + [0]
    G = make(g, w, bits=64 if gi % 2 else 32, **SSSP_BATCH_MODES[mode])
    out = G.sssp_batch(srcs).cpu().numpy().view(np.uint32)
    for i, s in enumerate(srcs):
        assert np.array_equal(out[i], oracle.sssp(g.offsets, g.indices, w, int(s))), (g.name, mode, i)
    # a second batch of another size reuses / regrows the state
    out2 = G.sssp_batch(srcs[:3]).cpu().numpy().view(np.uint32)
    for i, s in enumerate(srcs[:3]):
        assert np.array_equal(out2[i], oracle.sssp(g.offsets, g.indices, w, int(s)))
    G.close()


@pytest.mark.parametrize("mode", ["default", "push", "pull", "ballot", "all_classes"])
def test_bfs_multigraph_pack(mode):
    graphs, srcs = gg.multigraph_batch(count=24, n_lo=50, n_hi=3000, seed=0xBA7C4)
    packed, bases = gg.pack(graphs)
    roots = (srcs.astype(np.int64) + bases[:-1]).astype(np.int32)
    G = make(packed, **FORCED[mode])
    lev = G.bfs_multi(list(roots)).cpu().numpy()
    for i, g in enumerate(graphs):
        exp = oracle.bfs(g.offsets, g.indices, int(srcs[i]))
        assert np.array_equal(lev[bases[i]:bases[i + 1]], exp), (mode, i)
    # duplicate roots and a single root agree with the single-source call
    lev1 = G.bfs_multi([int(roots[0]), int(roots[0])]).cpu().numpy()
    assert np.array_equal(lev1, G.bfs(int(roots[0])).cpu().numpy())
    G.close()


@pytest.mark.parametrize("width", [8, 64])
@pytest.mark.parametrize("k", [1, 33, 64, 70, 130])
def test_sssp_batch_sizes(k, width):
    """Up to 64 sources per launch travel as a kernel parameter, in groups of
    the batch width; more than 64 take several launches."""
    import torch
    from paper_1812_04070_gb300 import simdx_stats
    g = gg.rmat(11)
    w = gg.weights(g, 99, 1, 64)
    srcs = np.resize(gg.pick_sources(g, 50, seed=k), k)
    G = make(g, w, bits=32, sssp_batch_width=width)
    st = simdx_stats()
    G.sssp_batch([int(s) for s in srcs], stats=st)
    torch.cuda.synchronize()
    assert st.status == 0 and st.launches == -(-k // 64)
    out = G.sssp_batch([int(s) for s in srcs]).cpu().numpy().view(np.uint32)
    for i, s in enumerate(srcs):
        assert np.array_equal(out[i], oracle.sssp(g.offsets, g.indices, w, int(s))), (k, i)
    G.close()


@pytest.mark.parametrize("k,group", [(10, 3), (7, 1), (140, 70)])
def test_sssp_batch_groups(k, group):
    """A batch runs its copies in groups, one persistent launch per group (the
    batch_group knob forces the split that a large graph gets by size); the
    launches share one stats record, and groups of more than 64 read their
    sources from device memory at the group's offset."""
    import torch
    from paper_1812_04070_gb300 import simdx_stats
    g = gg.rmat(11)
    w = gg.weights(g, 98, 1, 64)
    srcs = [int(s) for s in np.resize(gg.pick_sources(g, 50, seed=k), k)]
    G = make(g, w, bits=64, batch_group=group)
    st = simdx_stats()
    out = G.sssp_batch(srcs, stats=st).cpu().numpy().view(np.uint32)
    torch.cuda.synchronize()
    for i, s in enumerate(srcs):
        assert np.array_equal(out[i], oracle.sssp(g.offsets, g.indices, w, s)), (k, group, i)
    assert st.status == 0 and G.last_status() == 0
    assert st.iterations >= -(-k // group)  # every group ran at least one iteration
    tr = G.trace()  # the group launches number their records on
    assert tr.shape[0] == st.iterations and (tr[:, 4] > 0).all() and (tr[:, 5] >= tr[:, 4]).all()
    G.close()


def test_sssp_batch_directed():
    """Batched SSSP relaxes out-edges, so a directed graph (CSR + CSC) works."""
    import torch
    from paper_1812_04070_gb300 import Graph
    n = 400
    rng = np.random.default_rng(4)
    src = rng.integers(0, n, 3000)
    dst = rng.integers(0, n, 3000)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    pair = np.unique(np.stack([src, dst], 1), axis=0)
    src, dst = pair[:, 0], pair[:, 1]
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off)
    idx = dst.astype(np.int32)
    wt = (rng.integers(1, 50, len(idx))).astype(np.uint32)
    co = np.lexsort((src, dst))
    ioff = np.zeros(n + 1, np.int64)
    np.add.at(ioff, dst + 1, 1)
    ioff = np.cumsum(ioff)
    G = Graph(off, idx, weights=wt, csc=(ioff, src[co].astype(np.int32)))
    srcs = [0, 5, 77]
    out = G.sssp_batch(srcs).cpu().numpy().view(np.uint32)
    for i, s in enumerate(srcs):
        assert np.array_equal(out[i], oracle.sssp(off, idx, wt, s)), i
        assert torch.equal(torch.from_numpy(out[i].view(np.int32)), G.sssp(s).cpu())
    G.close()


def test_bfs_multigraph_separate_handles():
    """simdx_bfs_multigraph over separate graph objects: 256 R-MAT graphs of
    uneven size (n log-uniform in [1000, 100000], edge factor 8..32, the
    batching configuration's recipe), mixed offset widths, through the C ABI;
    every graph's levels equal the oracle's BFS of that graph.  A second call
    reuses the pack; a changed list (another order, a directed graph, a
    graph destroyed and re-created) rebuilds it."""
    import torch
    from paper_1812_04070_gb300 import Graph, SimdxError, bfs_multigraph, simdx
    from gpu_util import directed_graph
    graphs, srcs = gg.multigraph_batch(count=256)
    Gs = [Graph(g.offsets if i % 3 == 0 else g.offsets.astype(np.int32), g.indices) for i, g in enumerate(graphs)]
    outs = bfs_multigraph(Gs, srcs)
    torch.cuda.synchronize()
    for i, g in enumerate(graphs):
        assert np.array_equal(outs[i].cpu().numpy(), oracle.bfs(g.offsets, g.indices, int(srcs[i]))), i
    srcs2 = [int(gg.pick_sources(g, 1, seed=99 + i)[0]) for i, g in enumerate(graphs)]
    outs = bfs_multigraph(Gs, srcs2, outs=outs)  # same list: the cached pack
    torch.cuda.synchronize()
    for i, g in enumerate(graphs):
        assert np.array_equal(outs[i].cpu().numpy(), oracle.bfs(g.offsets, g.indices, srcs2[i])), i
    # another list: reversed order, a directed graph appended, one graph twice
    off, idx, ioff, iidx, _ = directed_graph(700, 3000, 2)
    D = Graph(off, idx, csc=(ioff, iidx))
    sub = list(reversed(Gs[:40])) + [D, Gs[5]]
    ss = list(reversed([int(s) for s in srcs[:40]])) + [3, int(srcs[5])]
    res = bfs_multigraph(sub, ss)
    torch.cuda.synchronize()
    want = list(reversed(graphs[:40]))
    for i, g in enumerate(want):
        assert np.array_equal(res[i].cpu().numpy(), oracle.bfs(g.offsets, g.indices, ss[i])), i
    assert np.array_equal(res[40].cpu().numpy(), oracle.bfs(off, idx, 3))
    assert np.array_equal(res[41].cpu().numpy(), oracle.bfs(graphs[5].offsets, graphs[5].indices, int(srcs[5])))
    # a graph re-created (perhaps at the same address) is a new list entry
    Gs[1].close()
    Gs[1] = Graph(graphs[1].offsets, graphs[1].indices)
    outs = bfs_multigraph(Gs[:8], srcs[:8])
    torch.cuda.synchronize()
    for i in range(8):
        g = graphs[i]
        assert np.array_equal(outs[i].cpu().numpy(), oracle.bfs(g.offsets, g.indices, int(srcs[i]))), i
    with pytest.raises(SimdxError) as e:
        bfs_multigraph(Gs[:2], [0, graphs[1].n])
    assert e.value.status == simdx.EINVAL
    for G in Gs + [D]:
        G.close()
