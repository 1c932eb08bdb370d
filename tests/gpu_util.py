"""Helpers shared by the GPU parity tests (not collected as tests)."""
from __future__ import annotations

import numpy as np

import graphgen as gg
import oracle

UNREACHED = np.uint32(0xFFFFFFFF)

# Knob settings that force every path of the method (results must not change).
FORCED = {
    "default": {},
    "push": dict(direction=1),
    "pull": dict(direction=2),
    "ballot": dict(filter=2),
    "overflow": dict(bin_per_thread=0),
    "tiny_bins": dict(bin_per_thread=1),
    "all_classes": dict(small_max=2, med_max=4, huge_min=8),
    "all_classes_pull": dict(small_max=2, med_max=4, huge_min=8, direction=2),
    "all_classes_ballot": dict(small_max=2, med_max=4, huge_min=8, filter=2),
    "one_cta_per_sm": dict(ctas_per_sm=1),
    "grid_only": dict(small_frontier=0),
    "cluster": dict(small_frontier=1),
    "cluster_all_classes": dict(small_frontier=1, small_max=2, med_max=4, huge_min=8),
}


def small_graphs():
    out = [gg.path(1), gg.path(2), gg.path(7), gg.star(9), gg.complete(6), gg.star(3000),
           gg.path(3000), gg.complete(70), gg.grid(33, 17), gg.from_edges(10, [0, 1, 5, 6], [1, 2, 6, 7])]
    for seed in range(4):
        n = 50 + 300 * seed
        out.append(gg.random_graph(n, int(1.3 * n), seed=100 + seed))
        out.append(gg.random_graph(n, 6 * n, seed=200 + seed))
    out += [gg.rmat(10), gg.rmat(12)]
    return out


def sources(g, k=3):
    deg = g.degrees()
    s = [0, g.n - 1]
    if g.n > 2:
        s.append(int(np.argmax(deg)))
    if g.n > 4:
        nz = np.nonzero(deg)[0]
        if nz.size:
            s.append(int(nz[len(nz) // 2]))
    return sorted(set(x for x in s if 0 <= x < g.n))[:k + 1]


def make(g, w=None, bits=64, **cfg):
    from paper_1812_04070_gb300 import Graph
    off = g.offsets if bits == 64 else g.offsets.astype(np.int32)
    G = Graph(off, g.indices, weights=w)
    if cfg:
        G.set_config(**cfg)
    return G


def assert_pagerank(G, g=None, d=0.85, tol=1e-6, max_iter=1000, in_csr=None, outdeg=None):
    """Run PageRank on the GPU and check it against the FP64 oracle.

    A run that only pulled (the Jacobi iteration) must be within 1e-6
    relative L1 of the oracle after the same number of iterations and stop
    within one iteration of the oracle's own stop.  A run that switched to
    push (Sec. 6 "PageRank") stops when the pending changes sum below tol in
    L1, which leaves its result within d / (1 - d) * tol of the fixed point;
    it must be within that bound plus 1e-6 (FP32 rounding) of the oracle's
    converged fixed point (run to 1e-13).  ``in_csr`` = (in_off, in_idx) of
    a directed graph (default: g's CSR).  Returns (stats, error)."""
    from paper_1812_04070_gb300 import simdx_stats
    import torch
    ioff, iidx = in_csr if in_csr is not None else (g.offsets, g.indices)
    st = simdx_stats()
    x = G.pagerank(d, tol, max_iter, stats=st)
    torch.cuda.synchronize()
    x = x.cpu().numpy().astype(np.float64)
    t = st.iterations
    assert st.status == 0 and st.pull_iters + st.push_iters == t
    if st.push_iters == 0:
        # the OpenMP variant returns the definition's values bit for bit (pinned)
        ex, _, _ = oracle.pagerank_par(ioff, iidx, outdeg=outdeg, d=d, fixed_iter=t)
        denom = np.abs(ex).sum()
        rel = np.abs(x - ex).sum() / denom if denom > 0 else 0.0
        assert rel <= 1e-6, rel
        _, t_stop, _ = oracle.pagerank_par(ioff, iidx, outdeg=outdeg, d=d, tol=tol, max_iter=max_iter)
        assert abs(t - t_stop) <= 1, (t, t_stop)
        return st, rel
    xc, _, _ = oracle.pagerank_par(ioff, iidx, outdeg=outdeg, d=d, tol=1e-13, max_iter=100000)
    err = np.abs(x - xc).sum()
    bound = d / (1 - d) * tol + 1e-6
    assert err <= bound, (err, bound, st.pull_iters, st.push_iters)
    assert st.last_l1 < tol or t == max_iter
    return st, err


def check_pagerank(G, g, d=0.85, tol=1e-6, max_iter=1000):
    """Jacobi parity of a pull-only run (see assert_pagerank)."""
    from paper_1812_04070_gb300 import simdx_stats
    import torch
    st = simdx_stats()
    x = G.pagerank(d, tol, max_iter, stats=st)
    torch.cuda.synchronize()
    x = x.cpu().numpy().astype(np.float64)
    t = st.iterations
    ex, _, _ = oracle.pagerank(g.offsets, g.indices, d=d, fixed_iter=t)
    denom = np.abs(ex).sum()
    rel = np.abs(x - ex).sum() / denom if denom > 0 else 0.0
    _, t_stop, _ = oracle.pagerank(g.offsets, g.indices, d=d, tol=tol, max_iter=max_iter)
    return rel, t, t_stop, st


def directed_graph(n, m, seed, wmax=64):
    """A seeded random directed graph: CSR (out-edges), CSC (in-edges) and
    weights in CSR order.  Some vertices have only out-edges, some only
    in-edges, some none."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    # a band of sources-only and sinks-only vertices
    k = max(1, n // 10)
    dst = np.where(dst < k, dst + k, dst)          # vertices [0, k) get no in-edges
    src = np.where((src >= n - k) & (n > 2 * k), src - k, src)  # vertices [n-k, n) get no out-edges
    keep = src != dst
    pairs = np.unique(np.stack([src[keep], dst[keep]], 1), axis=0)
    s, d = pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, s + 1, 1)
    off = np.cumsum(off)
    idx = d.astype(np.int32)
    order = np.lexsort((s, d))
    ioff = np.zeros(n + 1, np.int64)
    np.add.at(ioff, d + 1, 1)
    ioff = np.cumsum(ioff)
    iidx = s[order].astype(np.int32)
    w = rng.integers(1, wmax + 1, idx.size).astype(np.uint32)
    return off, idx, ioff, iidx, w
