"""GPU test of the continuous-batching server (growth direction (b)).

A mix of BFS / SSSP / k-core queries over three resident graphs is submitted
from two threads while earlier queries are still running.  Every result must
equal the same query run alone (solo library call before the server starts)
and the CPU oracle, and the server must have batched (fewer launches than
queries).
"""
import threading

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def test_server_results_equal_solo_runs():
    import torch
    from paper_1812_04070_gb300 import Graph, Server, build
    build()
    torch.cuda.set_device(0)
    raw = [gg.rmat(11), gg.grid(60, 70), gg.rmat(12)]
    ws = [gg.weights(g, 31 + i, 1, 64) for i, g in enumerate(raw)]
    Gs = [Graph(g.offsets, g.indices, weights=w) for g, w in zip(raw, ws)]
    rng = np.random.default_rng(5)
    queries = []
    for _ in range(240):
        gi = int(rng.integers(0, 3))
        r = rng.random()
        algo = Server.BFS if r < 0.5 else Server.SSSP if r < 0.9 else Server.KCORE
        srcs = gg.pick_sources(raw[gi], 40, seed=gi + 100)
        arg = int(rng.choice([2, 4, 16])) if algo == Server.KCORE else int(srcs[int(rng.integers(0, len(srcs)))])
        queries.append((gi, algo, arg))
    # solo runs before the server owns the graphs
    solo = {}
    for q in set(queries):
        gi, algo, arg = q
        if algo == Server.BFS:
            solo[q] = Gs[gi].bfs(arg).cpu().numpy()
        elif algo == Server.SSSP:
            solo[q] = Gs[gi].sssp(arg).cpu().numpy()
        else:
            solo[q] = Gs[gi].kcore(arg)[0].cpu().numpy()
    torch.cuda.synchronize()
    srv = Server(Gs, mem_budget=8 << 30, max_slots=3, max_sssp=4)
    assert srv.info()["slots"] >= 1
    outs = []
    for gi, algo, arg in queries:
        dt = torch.uint8 if algo == Server.KCORE else torch.int32
        outs.append(torch.full((raw[gi].n,), 3, dtype=dt, device="cuda"))
    tickets = [None] * len(queries)

    def submit(lo, hi):
        for i in range(lo, hi):
            gi, algo, arg = queries[i]
            tickets[i] = srv.submit(gi, algo, arg, outs[i])

    half = len(queries) // 2
    t = threading.Thread(target=submit, args=(half, len(queries)))
    t.start()
    submit(0, half)
    t.join()
    for tk in tickets:
        srv.wait(tk)
    info = srv.info()
    srv.close()
    assert info["served"] == len(queries)
    assert info["launches"] < len(queries), info
    for i, q in enumerate(queries):
        got = outs[i].cpu().numpy()
        assert np.array_equal(got, solo[q]), (i, q)
    # spot-check against the oracle
    for i, (gi, algo, arg) in enumerate(queries[:30]):
        g = raw[gi]
        if algo == Server.BFS:
            exp = oracle.bfs(g.offsets, g.indices, arg)
        elif algo == Server.SSSP:
            exp = oracle.sssp(g.offsets, g.indices, ws[gi], arg).view(np.int32)
        else:
            exp = oracle.kcore(g.offsets, g.indices, arg)[0]
        assert np.array_equal(outs[i].cpu().numpy(), exp), (i, gi, algo, arg)
    for G in Gs:
        G.close()


def test_server_rejects_bad_queries():
    import torch
    from paper_1812_04070_gb300 import Graph, Server, SimdxError, build
    build()
    g = gg.rmat(9)
    G = Graph(g.offsets, g.indices)  # no weights: SSSP is rejected
    srv = Server([G], mem_budget=2 << 30, max_slots=1)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(SimdxError):
        srv.submit(1, Server.BFS, 0, out)
    with pytest.raises(SimdxError):
        srv.submit(0, Server.SSSP, 0, out)
    with pytest.raises(SimdxError):
        srv.submit(0, Server.BFS, g.n, out)
    tk = srv.submit(0, Server.BFS, 0, out)
    srv.wait(tk)
    assert np.array_equal(out.cpu().numpy(), oracle.bfs(g.offsets, g.indices, 0))
    srv.close()
    G.close()


def test_server_eight_graphs_config5():
    """The serving configuration's eight resident graphs (R-MAT scales 14-20
    and 22, weights [1,64]) and its query mix (50 % BFS, 40 % SSSP, 10 %
    k-core 16, uniform graph, uniform non-isolated source), submitted in
    bursts while earlier queries run: every result equals the same query run
    alone, and a sample equals the oracle."""
    import torch
    from paper_1812_04070_gb300 import Graph, Server, build
    build()
    torch.cuda.set_device(0)
    scales = [14, 15, 16, 17, 18, 19, 20, 22]
    raw = [gg.rmat(sc) for sc in scales]
    ws = [gg.weights(g, gg.weight_seed(sc), 1, 64) for g, sc in zip(raw, scales)]
    Gs = [Graph(g.offsets.astype(np.int32), g.indices, weights=w) for g, w in zip(raw, ws)]
    srcs = [gg.pick_sources(g, 64, 0x5E77E + i) for i, g in enumerate(raw)]
    rng = np.random.default_rng(0x5E77E)
    queries = []
    for _ in range(600):
        gi = int(rng.integers(0, len(raw)))
        r = rng.random()
        algo = Server.BFS if r < 0.5 else Server.SSSP if r < 0.9 else Server.KCORE
        arg = 16 if algo == Server.KCORE else int(srcs[gi][int(rng.integers(0, len(srcs[gi])))])
        queries.append((gi, algo, arg))
    solo = {}
    for q in set(queries):
        gi, algo, arg = q
        if algo == Server.BFS:
            solo[q] = Gs[gi].bfs(arg).cpu().numpy()
        elif algo == Server.SSSP:
            solo[q] = Gs[gi].sssp(arg).cpu().numpy()
        else:
            solo[q] = Gs[gi].kcore(arg)[0].cpu().numpy()
    torch.cuda.synchronize()
    srv = Server(Gs, mem_budget=64 << 30, max_slots=4, max_sssp=8)
    outs = [torch.full((raw[gi].n,), 3, dtype=torch.uint8 if a == Server.KCORE else torch.int32, device="cuda")
            for gi, a, _ in queries]
    tickets = []
    for lo in range(0, len(queries), 50):  # bursts of 50 while earlier ones run
        for i in range(lo, min(lo + 50, len(queries))):
            gi, algo, arg = queries[i]
            tickets.append(srv.submit(gi, algo, arg, outs[i]))
    for tk in tickets:
        srv.wait(tk)
    info = srv.info()
    srv.close()
    assert info["served"] == len(queries) and info["launches"] < len(queries), info
    for i, q in enumerate(queries):
        assert np.array_equal(outs[i].cpu().numpy(), solo[q]), (i, q)
    seen = set()
    for i, (gi, algo, arg) in enumerate(queries):
        if (gi, algo) in seen or scales[gi] > 20:
            continue
        seen.add((gi, algo))
        g = raw[gi]
        if algo == Server.BFS:
            exp = oracle.bfs(g.offsets, g.indices, arg)
        elif algo == Server.SSSP:
            exp = oracle.sssp(g.offsets, g.indices, ws[gi], arg).view(np.int32)
        else:
            exp = oracle.kcore(g.offsets, g.indices, arg)[0]
        assert np.array_equal(outs[i].cpu().numpy(), exp), (i, gi, algo, arg)
    for G in Gs:
        G.close()
