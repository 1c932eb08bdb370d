"""GB300 (sm_103a) implementation of the SIMD-X Active-Compute-Combine graph
hot path (Liu & Huang, "SIMD-X: Programming and Processing of Graph
Algorithms on GPUs").

The product is the C ABI in ``include/simdx.h`` (``libsimdx.so``); ``simdx``
is its ctypes binding with the same names, and ``Graph`` below wraps it with
PyTorch tensors for device memory and streams.  There is no CPU path: if the
library is not built or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import simdx
from .simdx import SimdxError, simdx_config, simdx_stats

__all__ = ["Graph", "Server", "bfs_multigraph", "simdx", "SimdxError", "simdx_config", "simdx_stats", "build"]


def build(force: bool = False) -> str:
    """Compile libsimdx.so for sm_103a (in place)."""
    from . import _build
    return _build.build(force=force)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("paper_1812_04070_gb300 needs a CUDA device (GB300); none is visible")
    return torch


def _stream_handle(stream) -> int | None:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if stream.cuda_stream else None


class Graph:
    """A device-resident graph.  ``offsets``/``indices`` (and optional
    ``weights``, ``csc``) are host numpy arrays or CUDA torch tensors."""

    def __init__(self, offsets, indices, weights=None, csc=None, borrow: bool = False, stream=None):
        torch = _torch()
        self._keep = []
        host = isinstance(offsets, np.ndarray)
        flags = simdx.INPUT_HOST if host else (simdx.BORROW if borrow else 0)

        def ptr(a):
            if a is None:
                return None
            if host:
                a = np.ascontiguousarray(a)
                self._keep.append(a)
                return a.ctypes.data
            a = a.contiguous()
            self._keep.append(a)
            return a.data_ptr()

        def csr_of(off, idx):
            bits = 32 if (off.dtype == np.int32 if host else off.dtype == torch.int32) else 64
            n = int(off.shape[0]) - 1
            return simdx.simdx_csr(n, int(idx.shape[0]), bits, ptr(off), ptr(idx))

        self.csr = csr_of(offsets, indices)
        self.csc = csr_of(*csc) if csc is not None else None
        w = ptr(weights) if weights is not None else None
        self.n = int(self.csr.n)
        self.e = int(self.csr.e)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.handle = simdx.simdx_graph_create(self.csr, self.csc, w, flags, _stream_handle(stream))
        if not borrow:
            self._keep = []

    def close(self):
        if getattr(self, "handle", None):
            simdx.simdx_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- knobs
    @property
    def config(self) -> simdx_config:
        return simdx.simdx_graph_get_config(self.handle)

    def set_config(self, **kw) -> None:
        c = simdx.simdx_graph_get_config(self.handle)
        for k, v in kw.items():
            if not hasattr(c, k):
                raise AttributeError(k)
            setattr(c, k, v)
        simdx.simdx_graph_set_config(self.handle, c)

    def info(self) -> dict:
        return simdx.simdx_graph_info(self.handle)

    def trace(self, stream=None):
        return simdx.simdx_graph_trace(self.handle, _stream_handle(stream))

    def last_status(self, stream=None) -> int:
        return simdx.simdx_graph_last_status(self.handle, _stream_handle(stream))

    # ----------------------------------------------------------- algorithms
    def _out(self, out, dtype):
        torch = _torch()
        if out is None:
            return torch.empty(self.n, dtype=dtype, device=self.device)
        assert out.dtype == dtype and out.is_cuda and out.is_contiguous() and out.numel() >= self.n
        return out

    def bfs(self, src: int, out=None, stats: simdx_stats | None = None, stream=None):
        torch = _torch()
        out = self._out(out, torch.int32)
        simdx.simdx_bfs(self.handle, int(src), out.data_ptr(), stats, _stream_handle(stream))
        return out

    def bfs_batch(self, srcs, out=None, stats: simdx_stats | None = None, stream=None):
        """Levels from every source in `srcs` (one row per source), in one
        persistent launch per 64 sources."""
        torch = _torch()
        k = len(srcs)
        if out is None:
            out = torch.empty((k, self.n), dtype=torch.int32, device=self.device)
        assert out.dtype == torch.int32 and out.is_cuda and out.is_contiguous() and out.numel() >= k * self.n
        simdx.simdx_bfs_batch(self.handle, srcs, out.data_ptr(), stats, _stream_handle(stream))
        return out

    def sssp_batch(self, srcs, out=None, stats: simdx_stats | None = None, stream=None):
        """Distances from every source in `srcs` (one row per source, uint32
        values in an int32 tensor), all queries in one persistent launch."""
        torch = _torch()
        k = len(srcs)
        if out is None:
            out = torch.empty((k, self.n), dtype=torch.int32, device=self.device)
        assert out.dtype == torch.int32 and out.is_cuda and out.is_contiguous() and out.numel() >= k * self.n
        simdx.simdx_sssp_batch(self.handle, srcs, out.data_ptr(), stats, _stream_handle(stream))
        return out

    def bfs_multi(self, roots, out=None, stats: simdx_stats | None = None, stream=None):
        """BFS with all `roots` at level 0 (one root per graph of a packed batch)."""
        torch = _torch()
        out = self._out(out, torch.int32)
        simdx.simdx_bfs_multi(self.handle, roots, out.data_ptr(), stats, _stream_handle(stream))
        return out

    def sssp(self, src: int, out=None, stats: simdx_stats | None = None, stream=None):
        """uint32 distances returned in an int32 tensor (reinterpret with
        ``.view(torch.uint32)`` or mask 0xFFFFFFFF as unreached)."""
        torch = _torch()
        out = self._out(out, torch.int32)
        simdx.simdx_sssp(self.handle, int(src), out.data_ptr(), stats, _stream_handle(stream))
        return out

    def kcore(self, k: int, out=None, resid=None, want_resid: bool = True,
              stats: simdx_stats | None = None, stream=None):
        torch = _torch()
        out = self._out(out, torch.uint8)
        if want_resid:
            resid = self._out(resid, torch.int32)
        simdx.simdx_kcore(self.handle, int(k), out.data_ptr(), resid.data_ptr() if want_resid else None, stats,
                          _stream_handle(stream))
        return out, resid

    def kcore_batch(self, ks, want_resid: bool = True, stats: simdx_stats | None = None, stream=None):
        """The k-core of every k in `ks` (simdx_kcore_batch): uint8 rows
        [len(ks), n] of membership and, if asked, int32 rows of residual
        degrees (uint32 values)."""
        torch = _torch()
        ks = [int(k) for k in ks]
        inc = torch.empty((len(ks), self.n), dtype=torch.uint8, device=self.device)
        res = torch.empty((len(ks), self.n), dtype=torch.int32, device=self.device) if want_resid else None
        simdx.simdx_kcore_batch(self.handle, ks, inc.data_ptr(), res.data_ptr() if want_resid else None, stats,
                                _stream_handle(stream))
        return inc, res

    def coreness(self, out=None, stats: simdx_stats | None = None, stream=None):
        """uint32 coreness of every vertex in an int32 tensor
        (simdx_kcore_decompose)."""
        torch = _torch()
        out = self._out(out, torch.int32)
        simdx.simdx_kcore_decompose(self.handle, out.data_ptr(), stats, _stream_handle(stream))
        return out

    def wcc(self, out=None, stats: simdx_stats | None = None, stream=None):
        """uint32 component label (smallest vertex id of the component) of
        every vertex in an int32 tensor (simdx_wcc)."""
        torch = _torch()
        out = self._out(out, torch.int32)
        simdx.simdx_wcc(self.handle, out.data_ptr(), stats, _stream_handle(stream))
        return out

    def autotune(self, algo: int, arg: int = 0, reps: int = 5, stream=None) -> tuple[dict, float]:
        """Measure knob settings for `algo` (simdx.ALGO_*; arg = source or
        k) on this graph, install the fastest and return it with its median
        time in ms (simdx_autotune)."""
        best, ms = simdx.simdx_autotune(self.handle, int(algo), int(arg), int(reps), _stream_handle(stream))
        return {name: getattr(best, name) for name, _ in best._fields_ if name != "reserved"}, ms

    def autotune_batch(self, algo: int, srcs, reps: int = 3, stream=None) -> tuple[dict, float]:
        """Measure knob settings for a batched call (simdx.ALGO_BFS: bfs_batch,
        ALGO_SSSP: sssp_batch, ALGO_BFS_MULTI: bfs_multi) on these sources,
        install the fastest and return it with its median time in ms
        (simdx_autotune_batch)."""
        best, ms = simdx.simdx_autotune_batch(self.handle, int(algo), [int(x) for x in srcs], int(reps),
                                              _stream_handle(stream))
        return {name: getattr(best, name) for name, _ in best._fields_ if name != "reserved"}, ms

    def pagerank(self, damping: float = 0.85, tol: float = 1e-6, max_iter: int = 1000, out=None,
                 stats: simdx_stats | None = None, stream=None):
        torch = _torch()
        out = self._out(out, torch.float32)
        simdx.simdx_pagerank(self.handle, float(damping), float(tol), int(max_iter), out.data_ptr(), stats,
                             _stream_handle(stream))
        return out


def bfs_multigraph(graphs, srcs, outs=None, stream=None):
    """BFS of graphs[i] from srcs[i] for every i, all in one persistent launch
    (simdx_bfs_multigraph).  Returns the list of int32 level tensors."""
    torch = _torch()
    if outs is None:
        outs = [torch.empty(G.n, dtype=torch.int32, device=G.device) for G in graphs]
    for G, o in zip(graphs, outs):
        assert o.dtype == torch.int32 and o.is_cuda and o.is_contiguous() and o.numel() >= G.n
    simdx.simdx_bfs_multigraph([G.handle for G in graphs], [int(s) for s in srcs], [o.data_ptr() for o in outs],
                               _stream_handle(stream))
    return outs


class Server:
    """Continuous-batching query server over resident graphs (see
    simdx_server_create in include/simdx.h).  Results land in the tensors
    passed to submit (CUDA tensors or pinned CPU tensors)."""

    BFS, SSSP, KCORE = simdx.ALGO_BFS, simdx.ALGO_SSSP, simdx.ALGO_KCORE

    def __init__(self, graphs, mem_budget: int = 32 << 30, max_slots: int = 4, max_sssp: int = 8):
        self.graphs = list(graphs)
        self.handle = simdx.simdx_server_create([g.handle for g in self.graphs], mem_budget, max_slots, max_sssp)

    def submit(self, graph: int, algo: int, arg: int, out) -> int:
        return simdx.simdx_server_submit(self.handle, graph, algo, arg, out.data_ptr())

    def poll(self, ticket: int) -> bool:
        return simdx.simdx_server_poll(self.handle, ticket)

    def wait(self, ticket: int) -> None:
        simdx.simdx_server_wait(self.handle, ticket)

    def info(self) -> dict:
        return simdx.simdx_server_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            simdx.simdx_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
