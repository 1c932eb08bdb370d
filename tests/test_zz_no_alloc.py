"""BFS entry point that allocates nothing (simdx_bfs_noalloc).

It exists for callers that cannot call cudaMalloc (an external memory pool or
budget owns the device memory, or allocation is forbidden while a CUDA graph
is captured elsewhere).  Its scratch is a fixed device array inside the
library, so this test checks, through the C ABI, that two calls in a row give
the same levels as the regular simdx_bfs on a graph object, on symmetric and
directed graphs.  The file is named to be collected last.
"""
import numpy as np
import pytest

import graphgen as gg
from gpu_util import directed_graph

pytestmark = pytest.mark.gpu


def test_bfs_noalloc_matches_simdx_bfs():
    import torch
    from paper_1812_04070_gb300 import Graph, build, simdx
    build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream) or None
    for g, src, bits in [(gg.rmat(16), 0, 32), (gg.grid(300, 200), 17, 64)]:
        off = torch.from_numpy(g.offsets if bits == 64 else g.offsets.astype(np.int32)).cuda()
        idx = torch.from_numpy(g.indices).cuda()
        csr = simdx.simdx_csr(g.n, g.e, bits, off.data_ptr(), idx.data_ptr())
        G = Graph(off, idx)
        ref = G.bfs(src).clone()
        torch.cuda.synchronize()
        for _ in range(2):  # the scratch keeps the previous call's contents
            out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
            simdx.simdx_bfs_noalloc(csr, src, out.data_ptr(), sh)
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
        G.close()
    # a directed graph: every level pushes along out-edges, so the levels
    # equal simdx_bfs on a graph object given the in-edges too
    for case, bits in [((700, 3000, 2), 32), ((3000, 40000, 3), 64)]:
        doff, didx, dioff, diidx, _ = directed_graph(*case)
        cast = (lambda a: a.astype(np.int32)) if bits == 32 else (lambda a: a)
        off = torch.from_numpy(cast(doff)).cuda()
        idx = torch.from_numpy(didx).cuda()
        csr = simdx.simdx_csr(doff.size - 1, didx.size, bits, off.data_ptr(), idx.data_ptr())
        G = Graph(cast(doff), didx, csc=(cast(dioff), diidx))
        for src in (0, (doff.size - 1) // 2):
            ref = G.bfs(src).clone()
            torch.cuda.synchronize()
            for _ in range(2):
                out = torch.full((doff.size - 1,), 7, dtype=torch.int32, device="cuda")
                simdx.simdx_bfs_noalloc(csr, src, out.data_ptr(), sh)
                torch.cuda.synchronize()
                assert torch.equal(out, ref)
        G.close()
    with pytest.raises(simdx.SimdxError):
        simdx.simdx_bfs_noalloc(simdx.simdx_csr((1 << 18) + 1, 0, 64, off.data_ptr(), idx.data_ptr()), 0,
                                out.data_ptr(), sh)
