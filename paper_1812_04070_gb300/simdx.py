"""ctypes binding of libsimdx (include/simdx.h): same names, marshalling only.

Every function below forwards to the C ABI of the same name and raises
``SimdxError`` on a non-zero status.  No graph computation happens in Python:
the library runs each algorithm as one persistent CUDA kernel.  PyTorch is
used only to own device memory and streams (``Graph`` below).

The library must be built (``paper_1812_04070_gb300._build.build()``); if it
is missing or cannot be loaded this module raises at first use -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

OK, EINVAL, ENOMEM, ECUDA, EBARRIER_TIMEOUT, EUNSUPPORTED, EBUSY, ENOTREADY = range(8)
ALGO_BFS, ALGO_SSSP, ALGO_KCORE, ALGO_PAGERANK, ALGO_BFS_MULTI = 1, 2, 3, 4, 5
INPUT_HOST = 1
BORROW = 2


class SimdxError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = _lib().simdx_strerror(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{what}: {msg} (status {status})")


class simdx_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("e", ctypes.c_int64), ("offset_bits", ctypes.c_int32),
                ("offsets", ctypes.c_void_p), ("indices", ctypes.c_void_p)]


class simdx_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("push_iters", ctypes.c_int32), ("pull_iters", ctypes.c_int32),
                ("ballot_iters", ctypes.c_int32), ("online_iters", ctypes.c_int32),
                ("phases", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
                ("edges_visited", ctypes.c_int64), ("frontier_sum", ctypes.c_int64),
                ("last_l1", ctypes.c_double), ("launches", ctypes.c_int32),
                ("reserved32", ctypes.c_int32), ("reserved", ctypes.c_int64 * 3)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("reserved")}


class simdx_config(ctypes.Structure):
    _fields_ = [("small_max", ctypes.c_int32), ("med_max", ctypes.c_int32),
                ("huge_min", ctypes.c_int32), ("bin_per_thread", ctypes.c_int32),
                ("direction", ctypes.c_int32), ("filter", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("kcore_alpha", ctypes.c_float), ("delta", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_int32), ("barrier_timeout_ms", ctypes.c_int32),
                ("debug_skip_cta", ctypes.c_int32), ("debug_skip_phase", ctypes.c_int32),
                ("batch_group", ctypes.c_int32), ("fusion", ctypes.c_int32),
                ("pr_alpha", ctypes.c_float), ("pr_theta", ctypes.c_float), ("pr_rho", ctypes.c_float),
                ("sssp_combine", ctypes.c_int32), ("sssp_batch_width", ctypes.c_int32),
                ("pr_row_cost", ctypes.c_int32), ("stage_edges", ctypes.c_int32),
                ("pr_recut", ctypes.c_int32), ("small_frontier", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


_LIB = None

# name -> (restype, argtypes)
_vp, _i32, _i64, _u32, _f32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                               ctypes.c_float)
SIGNATURES = {
    "simdx_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "simdx_version": (ctypes.c_int, []),
    "simdx_last_cuda_error": (ctypes.c_char_p, []),
    "simdx_config_default": (None, [ctypes.POINTER(simdx_config)]),
    "simdx_eq1_ctas": (_i64, [_i64, _i64, _i64, _i64]),
    "simdx_graph_create": (ctypes.c_int, [ctypes.POINTER(simdx_csr), ctypes.POINTER(simdx_csr), _vp, _u32,
                                          _vp, ctypes.POINTER(_vp)]),
    "simdx_graph_destroy": (ctypes.c_int, [_vp]),
    "simdx_graph_info": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                        ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "simdx_graph_get_config": (ctypes.c_int, [_vp, ctypes.POINTER(simdx_config)]),
    "simdx_graph_set_config": (ctypes.c_int, [_vp, ctypes.POINTER(simdx_config)]),
    "simdx_graph_last_status": (ctypes.c_int, [_vp, _vp]),
    "simdx_graph_trace": (ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.POINTER(_i64)]),
    "simdx_bfs": (ctypes.c_int, [_vp, _i32, _vp, ctypes.POINTER(simdx_stats), _vp]),
    "simdx_sssp": (ctypes.c_int, [_vp, _i32, _vp, ctypes.POINTER(simdx_stats), _vp]),
    "simdx_kcore": (ctypes.c_int, [_vp, _u32, _vp, _vp, ctypes.POINTER(simdx_stats), _vp]),
    "simdx_kcore_decompose": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(simdx_stats), _vp]),
    "simdx_kcore_batch": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint32), _i32, _vp, _vp,
                                         ctypes.POINTER(simdx_stats), _vp]),
    "simdx_wcc": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(simdx_stats), _vp]),
    "simdx_pagerank": (ctypes.c_int, [_vp, _f32, _f32, _i32, _vp, ctypes.POINTER(simdx_stats), _vp]),
    "simdx_bfs_noalloc": (ctypes.c_int, [ctypes.POINTER(simdx_csr), _i32, _vp, _vp]),
    "simdx_bfs_batch": (ctypes.c_int, [_vp, _vp, _i32, _vp, ctypes.POINTER(simdx_stats), _vp]),
    "simdx_sssp_batch": (ctypes.c_int, [_vp, _vp, _i32, _vp, ctypes.POINTER(simdx_stats), _vp]),
    "simdx_bfs_multi": (ctypes.c_int, [_vp, _vp, _i32, _vp, ctypes.POINTER(simdx_stats), _vp]),
    "simdx_bfs_multigraph": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp]),
    "simdx_server_create": (ctypes.c_int, [_vp, _i32, ctypes.c_size_t, _i32, _i32, ctypes.POINTER(_vp)]),
    "simdx_server_submit": (ctypes.c_int, [_vp, _i32, _i32, _i32, _vp, ctypes.POINTER(ctypes.c_uint64)]),
    "simdx_server_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(_i32)]),
    "simdx_server_wait": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "simdx_server_info": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "simdx_server_destroy": (ctypes.c_int, [_vp]),
    "simdx_autotune": (ctypes.c_int, [_vp, _i32, _i64, _i32, ctypes.POINTER(simdx_config),
                                      ctypes.POINTER(ctypes.c_float), _vp]),
    "simdx_autotune_batch": (ctypes.c_int, [_vp, _i32, _vp, _i32, _i32, ctypes.POINTER(simdx_config),
                                            ctypes.POINTER(ctypes.c_float), _vp]),
}


def library_path() -> str:
    return _build.LIB


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libsimdx.so is not built ({path}); run __graft_entry__.build() "
                               "or paper_1812_04070_gb300._build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def _check(rc: int, what: str):
    if rc != OK:
        raise SimdxError(rc, what)


# ------------------------------------------------------------- same names
def simdx_version() -> int:
    return _lib().simdx_version()


def simdx_strerror(status: int) -> str:
    return _lib().simdx_strerror(status).decode()


def simdx_config_default() -> simdx_config:
    c = simdx_config()
    _lib().simdx_config_default(ctypes.byref(c))
    return c


def simdx_eq1_ctas(regs_per_sm: int, regs_per_thread: int, threads_per_cta: int, n_sm: int) -> int:
    return _lib().simdx_eq1_ctas(regs_per_sm, regs_per_thread, threads_per_cta, n_sm)


def simdx_graph_create(csr: simdx_csr, csc: simdx_csr | None, weights: int | None, flags: int,
                       stream: int | None) -> int:
    h = ctypes.c_void_p()
    rc = _lib().simdx_graph_create(ctypes.byref(csr), ctypes.byref(csc) if csc is not None else None,
                                   weights, flags, stream, ctypes.byref(h))
    _check(rc, "simdx_graph_create")
    return h.value


def simdx_graph_destroy(g: int) -> None:
    _check(_lib().simdx_graph_destroy(g), "simdx_graph_destroy")


def simdx_graph_info(g: int) -> dict:
    n, e, gc, tc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib().simdx_graph_info(g, ctypes.byref(n), ctypes.byref(e), ctypes.byref(gc), ctypes.byref(tc)),
           "simdx_graph_info")
    return {"n": n.value, "e": e.value, "grid_ctas": gc.value, "threads_per_cta": tc.value}


def simdx_graph_get_config(g: int) -> simdx_config:
    c = simdx_config()
    _check(_lib().simdx_graph_get_config(g, ctypes.byref(c)), "simdx_graph_get_config")
    return c


def simdx_graph_set_config(g: int, cfg: simdx_config) -> None:
    _check(_lib().simdx_graph_set_config(g, ctypes.byref(cfg)), "simdx_graph_set_config")


def simdx_graph_last_status(g: int, stream: int | None) -> int:
    return _lib().simdx_graph_last_status(g, stream)


def simdx_graph_trace(g: int, stream: int | None, cap: int = 1 << 16):
    import numpy as np
    rec = np.zeros((cap, 8), dtype=np.int64)
    cnt = ctypes.c_int64()
    _check(_lib().simdx_graph_trace(g, stream, rec.ctypes.data, cap, ctypes.byref(cnt)), "simdx_graph_trace")
    return rec[:min(cnt.value, cap)].copy()


def simdx_bfs(g: int, src: int, levels_ptr: int, stats: simdx_stats | None, stream: int | None) -> None:
    _check(_lib().simdx_bfs(g, src, levels_ptr, ctypes.byref(stats) if stats is not None else None, stream),
           "simdx_bfs")


def simdx_sssp(g: int, src: int, dist_ptr: int, stats: simdx_stats | None, stream: int | None) -> None:
    _check(_lib().simdx_sssp(g, src, dist_ptr, ctypes.byref(stats) if stats is not None else None, stream),
           "simdx_sssp")


def simdx_kcore(g: int, k: int, in_core_ptr: int, resid_ptr: int | None, stats: simdx_stats | None,
                stream: int | None) -> None:
    _check(_lib().simdx_kcore(g, k, in_core_ptr, resid_ptr, ctypes.byref(stats) if stats is not None else None,
                              stream), "simdx_kcore")


def simdx_kcore_batch(g: int, ks, in_core_ptr: int, resid_ptr: int | None, stats: simdx_stats | None,
                      stream: int | None) -> None:
    arr = (ctypes.c_uint32 * len(ks))(*[int(k) for k in ks])
    _check(_lib().simdx_kcore_batch(g, arr, len(ks), in_core_ptr, resid_ptr,
                                    ctypes.byref(stats) if stats is not None else None, stream), "simdx_kcore_batch")


def simdx_kcore_decompose(g: int, core_ptr: int, stats: simdx_stats | None, stream: int | None) -> None:
    _check(_lib().simdx_kcore_decompose(g, core_ptr, ctypes.byref(stats) if stats is not None else None, stream),
           "simdx_kcore_decompose")


def simdx_wcc(g: int, label_ptr: int, stats: simdx_stats | None, stream: int | None) -> None:
    _check(_lib().simdx_wcc(g, label_ptr, ctypes.byref(stats) if stats is not None else None, stream),
           "simdx_wcc")


def simdx_pagerank(g: int, damping: float, l1_tol: float, max_iter: int, rank_ptr: int,
                   stats: simdx_stats | None, stream: int | None) -> None:
    _check(_lib().simdx_pagerank(g, damping, l1_tol, max_iter, rank_ptr,
                                 ctypes.byref(stats) if stats is not None else None, stream), "simdx_pagerank")


def simdx_bfs_noalloc(csr: simdx_csr, src: int, levels_ptr: int, stream: int | None) -> None:
    """BFS that allocates no device memory (device CSR in, device levels out;
    at most 2^18 vertices).  See include/simdx.h."""
    _check(_lib().simdx_bfs_noalloc(ctypes.byref(csr), src, levels_ptr, stream), "simdx_bfs_noalloc")


def simdx_bfs_batch(g: int, srcs, levels_ptr: int, stats: simdx_stats | None, stream: int | None) -> None:
    """Batched BFS from the host int32 sources `srcs`; levels: device int32[k*n]."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    _check(_lib().simdx_bfs_batch(g, a.ctypes.data, int(a.size), levels_ptr,
                                  ctypes.byref(stats) if stats is not None else None, stream), "simdx_bfs_batch")


def simdx_sssp_batch(g: int, srcs, dist_ptr: int, stats: simdx_stats | None, stream: int | None) -> None:
    """Batched SSSP from the host int32 sources `srcs`; dist: device uint32[k*n]."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    _check(_lib().simdx_sssp_batch(g, a.ctypes.data, int(a.size), dist_ptr,
                                   ctypes.byref(stats) if stats is not None else None, stream), "simdx_sssp_batch")


def simdx_bfs_multi(g: int, roots, levels_ptr: int, stats: simdx_stats | None, stream: int | None) -> None:
    """BFS with every root of `roots` at level 0; levels: device int32[n]."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(roots, dtype=np.int32))
    _check(_lib().simdx_bfs_multi(g, a.ctypes.data, int(a.size), levels_ptr,
                                  ctypes.byref(stats) if stats is not None else None, stream), "simdx_bfs_multi")


def simdx_bfs_multigraph(graphs, srcs, levels_ptrs, stream: int | None) -> None:
    """BFS of graph i from srcs[i] into the device array levels_ptrs[i], all
    graphs in one launch."""
    import numpy as np
    k = len(graphs)
    gs = (ctypes.c_void_p * k)(*graphs)
    a = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    outs = (ctypes.c_void_p * k)(*levels_ptrs)
    _check(_lib().simdx_bfs_multigraph(gs, a.ctypes.data, k, outs, stream), "simdx_bfs_multigraph")


def simdx_server_create(graphs, mem_budget: int, max_slots: int = 4, max_sssp: int = 8) -> int:
    arr = (ctypes.c_void_p * len(graphs))(*graphs)
    h = ctypes.c_void_p()
    _check(_lib().simdx_server_create(arr, len(graphs), mem_budget, max_slots, max_sssp, ctypes.byref(h)),
           "simdx_server_create")
    return h.value


def simdx_server_submit(s: int, graph: int, algo: int, arg: int, out_ptr: int) -> int:
    t = ctypes.c_uint64()
    _check(_lib().simdx_server_submit(s, graph, algo, arg, out_ptr, ctypes.byref(t)), "simdx_server_submit")
    return t.value


def simdx_server_poll(s: int, ticket: int) -> bool:
    done = ctypes.c_int32()
    rc = _lib().simdx_server_poll(s, ticket, ctypes.byref(done))
    if rc == ENOTREADY:
        return False
    _check(rc, "simdx_server_poll")
    return True


def simdx_server_wait(s: int, ticket: int) -> None:
    _check(_lib().simdx_server_wait(s, ticket), "simdx_server_wait")


def simdx_server_info(s: int) -> dict:
    sl, la, se, qu = ctypes.c_int32(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib().simdx_server_info(s, ctypes.byref(sl), ctypes.byref(la), ctypes.byref(se), ctypes.byref(qu)),
           "simdx_server_info")
    return {"slots": sl.value, "launches": la.value, "served": se.value, "queued": qu.value}


def simdx_server_destroy(s: int) -> None:
    _check(_lib().simdx_server_destroy(s), "simdx_server_destroy")


def simdx_autotune(g: int, algo: int, arg: int, reps: int, stream: int | None) -> tuple[simdx_config, float]:
    best, ms = simdx_config(), ctypes.c_float()
    _check(_lib().simdx_autotune(g, algo, arg, reps, ctypes.byref(best), ctypes.byref(ms), stream),
           "simdx_autotune")
    return best, ms.value


def simdx_autotune_batch(g: int, algo: int, srcs, reps: int, stream: int | None) -> tuple[simdx_config, float]:
    import numpy as np
    a = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    best, ms = simdx_config(), ctypes.c_float()
    _check(_lib().simdx_autotune_batch(g, algo, a.ctypes.data, int(a.size), reps, ctypes.byref(best),
                                       ctypes.byref(ms), stream), "simdx_autotune_batch")
    return best, ms.value
