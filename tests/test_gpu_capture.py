"""CUDA-graph capture of the algorithm and batched calls (growth direction
(a): "captured into a CUDA graph"): a stream capture records each
persistent launch as a cooperative kernel node; replays must give the same
results as the calls, and match the oracle."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_util import make

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def device():
    import torch
    from paper_1812_04070_gb300 import build
    build()
    torch.cuda.set_device(0)


def test_capture_and_replay():
    import torch
    g = gg.rmat(12)
    w = gg.weights(g, 21, 1, 64)
    G = make(g, w, bits=32, batch_group=16)  # the SSSP batch runs as three launches
    n = g.n
    srcs = [int(x) for x in gg.pick_sources(g, 40, seed=5)]
    graphs, gsrc = gg.multigraph_batch(count=12, n_lo=50, n_hi=2000, seed=0xBA7C4)
    packed, bases = gg.pack(graphs)
    roots = [int(x) for x in (gsrc.astype(np.int64) + bases[:-1])]
    P = make(packed, bits=32)
    dev = torch.device("cuda")
    ob = torch.empty((len(srcs), n), dtype=torch.int32, device=dev)
    osb = torch.empty((len(srcs), n), dtype=torch.int32, device=dev)
    o1 = torch.empty(n, dtype=torch.int32, device=dev)
    o2 = torch.empty(n, dtype=torch.int32, device=dev)
    ok = torch.empty(n, dtype=torch.uint8, device=dev)
    orr = torch.empty(n, dtype=torch.int32, device=dev)
    opr = torch.empty(n, dtype=torch.float32, device=dev)
    om = torch.empty(packed.n, dtype=torch.int32, device=dev)

    def calls():
        G.bfs_batch(srcs, out=ob)
        G.sssp_batch(srcs, out=osb)
        G.bfs(srcs[0], out=o1)
        G.sssp(srcs[1], out=o2)
        G.kcore(4, out=ok, resid=orr)
        G.pagerank(out=opr)
        P.bfs_multi(roots, out=om)

    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        calls()  # first calls outside the capture allocate the batch states
    torch.cuda.synchronize()
    ref = [t.clone() for t in (ob, osb, o1, o2, ok, orr, opr, om)]
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=s):
        calls()
    for rep in range(3):
        for t in (ob, osb, o1, o2, orr, om):
            t.fill_(-7)
        ok.fill_(9)
        opr.fill_(-1.0)
        cg.replay()
        torch.cuda.synchronize()
        for t, r in zip((ob, osb, o1, o2, ok, orr, opr, om), ref):
            assert torch.equal(t, r), rep
    lev = ob.cpu().numpy()
    dist = osb.cpu().numpy().view(np.uint32)
    for i in (0, 17, len(srcs) - 1):
        assert np.array_equal(lev[i], oracle.bfs(g.offsets, g.indices, srcs[i]))
        assert np.array_equal(dist[i], oracle.sssp(g.offsets, g.indices, w, srcs[i]))
    lm = om.cpu().numpy()
    for i, x in enumerate(graphs):
        assert np.array_equal(lm[bases[i]:bases[i + 1]], oracle.bfs(x.offsets, x.indices, int(gsrc[i])))
    G.close()
    P.close()


def test_capture_rejects_stats():
    import torch
    from paper_1812_04070_gb300 import SimdxError, simdx_stats
    g = gg.rmat(9)
    G = make(g, bits=32)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        G.bfs(0, out=out)
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with pytest.raises(SimdxError):
        with torch.cuda.graph(cg, stream=s):
            G.bfs(0, out=out, stats=simdx_stats())
    torch.cuda.synchronize()
    G.close()


def test_capture_cluster_launches():
    """On a grid (no hubs) BFS runs its small levels in a launch in clusters,
    the k-core decomposition splits into a plain, a cluster and a plain
    launch, the batched k-core adds its row launches, and SSSP in cluster
    mode launches in clusters: a capture records them all and replays give
    the calls' results."""
    import torch
    g = gg.grid(60, 50)
    w = gg.weights(g, 4, 1, 100)
    G = make(g, w, bits=64)
    S = make(g, w, bits=32, small_frontier=1)
    n = g.n
    dev = torch.device("cuda")
    o1 = torch.empty(n, dtype=torch.int32, device=dev)
    oc = torch.empty(n, dtype=torch.int32, device=dev)
    os_ = torch.empty(n, dtype=torch.int32, device=dev)

    def calls():
        G.bfs(7, out=o1)
        G.coreness(out=oc)
        kb = G.kcore_batch([1, 2, 3])
        S.sssp(11, out=os_)
        return kb

    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        calls()
    torch.cuda.synchronize()
    ref = [t.clone() for t in (o1, oc, os_)]
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=s):
        kin, kres = calls()
    for rep in range(2):
        for t in (o1, oc, os_):
            t.fill_(-5)
        kin.fill_(7)
        cg.replay()
        torch.cuda.synchronize()
        for t, r in zip((o1, oc, os_), ref):
            assert torch.equal(t, r), rep
        core = oracle.coreness(g.offsets, g.indices)
        for i, k in enumerate([1, 2, 3]):
            assert np.array_equal(kin[i].cpu().numpy(), (core >= k).astype(np.uint8)), (rep, k)
    assert np.array_equal(o1.cpu().numpy(), oracle.bfs(g.offsets, g.indices, 7))
    assert np.array_equal(os_.cpu().numpy().view(np.uint32), oracle.sssp(g.offsets, g.indices, w, 11))
    assert np.array_equal(oc.cpu().numpy().view(np.uint32), core)
    G.close()
    S.close()
