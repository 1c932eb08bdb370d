"""BFS entry point that allocates nothing (simdx_bfs_noalloc).

It exists for callers that cannot call cudaMalloc (an external memory pool or
budget owns the device memory, or allocation is forbidden while a CUDA graph
is captured elsewhere).  Its scratch is a fixed device array inside the
library, so this test checks, through the C ABI, that two calls in a row give
the same levels as the regular simdx_bfs on a graph object.  The file is
named to be collected last.
"""
import numpy as np
import pytest

import graphgen as gg

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
    with pytest.raises(simdx.SimdxError):
        simdx.simdx_bfs_noalloc(simdx.simdx_csr((1 << 18) + 1, 0, 64, off.data_ptr(), idx.data_ptr()), 0,
                                out.data_ptr(), sh)
