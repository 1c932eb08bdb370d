"""GPU tests of the autotuner (simdx_autotune): it installs the knob setting
it returns, that setting is valid, and every algorithm still matches the
oracle afterwards (knobs change speed only)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_util import assert_pagerank, make

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def device():
    import torch
    from paper_1812_04070_gb300 import build
    build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("bits", [32, 64])
def test_autotune_each_algorithm(bits):
    from paper_1812_04070_gb300 import simdx
    g = gg.rmat(13)
    w = gg.weights(g, 7, 1, 64)
    G = make(g, w, bits=bits)
    src = int(np.argmax(g.degrees()))
    for algo, arg in [(simdx.ALGO_BFS, src), (simdx.ALGO_SSSP, src), (simdx.ALGO_KCORE, 8),
                      (simdx.ALGO_PAGERANK, 0)]:
        best, ms = G.autotune(algo, arg, reps=2)
        assert ms > 0
        cfg = G.config
        for k, v in best.items():
            assert getattr(cfg, k) == pytest.approx(v), (algo, k)
        assert 1 <= cfg.small_max <= cfg.med_max <= cfg.huge_min
    assert np.array_equal(G.bfs(src).cpu().numpy(), oracle.bfs(g.offsets, g.indices, src))
    assert np.array_equal(G.sssp(src).cpu().numpy().view(np.uint32), oracle.sssp(g.offsets, g.indices, w, src))
    inc, resid = G.kcore(8)
    ei, er = oracle.kcore(g.offsets, g.indices, 8)
    assert np.array_equal(inc.cpu().numpy(), ei) and np.array_equal(resid.cpu().numpy(), er)
    assert_pagerank(G, g)
    G.close()


def test_autotune_rejects_bad_arguments():
    from paper_1812_04070_gb300 import SimdxError, simdx
    g = gg.rmat(9)
    G = make(g)  # no weights
    for algo, arg, reps in [(0, 0, 2), (5, 0, 2), (simdx.ALGO_BFS, g.n, 2), (simdx.ALGO_BFS, -1, 2),
                            (simdx.ALGO_BFS, 0, 0), (simdx.ALGO_BFS, 0, 65)]:
        with pytest.raises(SimdxError) as e:
            G.autotune(algo, arg, reps=reps)
        assert e.value.status == simdx.EINVAL
    with pytest.raises(SimdxError) as e:
        G.autotune(simdx.ALGO_SSSP, 0)
    assert e.value.status == simdx.EUNSUPPORTED
    G.close()


def test_autotune_batch_calls():
    """simdx_autotune_batch tunes the batched calls (bit-parallel BFS batch,
    SSSP batch, multi-root BFS); the results stay identical to the oracle."""
    from paper_1812_04070_gb300 import SimdxError, simdx
    g = gg.rmat(12)
    w = gg.weights(g, 4, 1, 64)
    G = make(g, w, bits=32)
    srcs = [int(s) for s in gg.pick_sources(g, 12, seed=5)]
    for algo in (simdx.ALGO_BFS, simdx.ALGO_SSSP, simdx.ALGO_BFS_MULTI):
        best, ms = G.autotune_batch(algo, srcs, reps=2)
        assert ms > 0
        for k, v in best.items():
            assert getattr(G.config, k) == pytest.approx(v), (algo, k)
    lb = G.bfs_batch(srcs).cpu().numpy()
    db = G.sssp_batch(srcs).cpu().numpy().view(np.uint32)
    for i, s in enumerate(srcs):
        assert np.array_equal(lb[i], oracle.bfs(g.offsets, g.indices, s))
        assert np.array_equal(db[i], oracle.sssp(g.offsets, g.indices, w, s))
    lm = G.bfs_multi(srcs).cpu().numpy()
    ref = np.min(np.stack([np.where(x < 0, 1 << 30, x) for x in lb]), axis=0)
    assert np.array_equal(lm, np.where(ref == 1 << 30, -1, ref))
    with pytest.raises(SimdxError) as e:
        G.autotune_batch(simdx.ALGO_KCORE, srcs)
    assert e.value.status == simdx.EINVAL
    G.close()
