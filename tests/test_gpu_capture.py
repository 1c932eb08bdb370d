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
