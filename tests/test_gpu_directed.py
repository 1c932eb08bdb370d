"""GPU parity on directed graphs (CSR out-edges plus a separate CSC of
in-edges, Sec. 6 "Storage Format"): BFS in every direction mode (pull reads
the in-edges), SSSP (push along out-edges) and PageRank (pull over in-edges,
out-degree from the CSR), against the oracle; k-core needs a symmetric
graph."""
import numpy as np
import pytest

import oracle
from gpu_util import FORCED, assert_pagerank, directed_graph

pytestmark = pytest.mark.gpu

CASES = [(60, 150, 1), (700, 3000, 2), (3000, 40000, 3)]


@pytest.fixture(scope="module", autouse=True)
def device():
    import torch
    from paper_1812_04070_gb300 import build
    build()
    torch.cuda.set_device(0)


def _make(off, idx, ioff, iidx, w, bits, **cfg):
    from paper_1812_04070_gb300 import Graph
    cast = (lambda a: a.astype(np.int32)) if bits == 32 else (lambda a: a)
    G = Graph(cast(off), idx, weights=w, csc=(cast(ioff), iidx))
    if cfg:
        G.set_config(**cfg)
    return G


@pytest.mark.parametrize("mode", ["default", "push", "pull", "ballot", "all_classes", "all_classes_pull"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_directed_bfs_sssp(case, mode):
    off, idx, ioff, iidx, w = directed_graph(*CASES[case])
    G = _make(off, idx, ioff, iidx, w, bits=32 if case % 2 else 64, **FORCED[mode])
    n = off.size - 1
    for src in sorted({0, 1, n // 2, n - 1}):
        assert np.array_equal(G.bfs(src).cpu().numpy(), oracle.bfs(off, idx, src)), (case, mode, src)
        assert np.array_equal(G.sssp(src).cpu().numpy().view(np.uint32), oracle.sssp(off, idx, w, src)), \
            (case, mode, src)
    G.close()


@pytest.mark.parametrize("case", range(len(CASES)))
def test_directed_pagerank(case):
    import torch
    from paper_1812_04070_gb300 import simdx_stats
    off, idx, ioff, iidx, w = directed_graph(*CASES[case])
    G = _make(off, idx, ioff, iidx, w, bits=64 if case % 2 else 32)
    outdeg = np.diff(off)
    assert_pagerank(G, in_csr=(ioff, iidx), outdeg=outdeg)
    # deterministic
    assert np.array_equal(G.pagerank().cpu().numpy(), G.pagerank().cpu().numpy())
    # the push tail forced after two pulls: pushes run along the out-edges
    G.set_config(pr_alpha=1e-30, pr_rho=0.0)
    st, _ = assert_pagerank(G, in_csr=(ioff, iidx), outdeg=outdeg)
    assert st.push_iters > 0
    assert np.array_equal(G.pagerank().cpu().numpy(), G.pagerank().cpu().numpy())
    G.close()


def test_directed_kcore_rejected():
    from paper_1812_04070_gb300 import SimdxError
    off, idx, ioff, iidx, w = directed_graph(*CASES[0])
    G = _make(off, idx, ioff, iidx, w, bits=64)
    with pytest.raises(SimdxError):
        G.kcore(2)
    with pytest.raises(SimdxError):
        G.coreness()
    with pytest.raises(SimdxError):
        G.wcc()
    G.close()
