"""CPU oracle for the SIMD-X graph method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library never
loads it; it shares no code with the CUDA path (the two meet only through the
seeded inputs of ``graphgen``).

Every function is a plain, single-threaded definition written from the paper
(Liu & Huang, "SIMD-X: Programming and Processing of Graph Algorithms on
GPUs"), cited per function in ``oracle.c``:

* ``bfs``        -- Sec. 6 "BFS", FIFO-queue levels.
* ``sssp``       -- Sec. 2.1 / Sec. 3.3, Dijkstra distances.
* ``sssp_bsp``   -- Sec. 2.1, the per-iteration BSP relaxation narrative.
* ``kcore``      -- Sec. 6 "k-Core", queue peeling (membership + residual degree).
* ``coreness``   -- Batagelj-Zaversnik core numbers (cross-check of ``kcore``).
* ``wcc``        -- Sec. 3.2 (voting algorithms), component labels = the
                    smallest vertex id of each weakly connected component.
* ``pagerank``   -- Sec. 6 "PageRank", FP64 Jacobi pull iteration (readings of
                    the unstated teleport, dangling and stop rules: see the
                    function docstring).
* ``pagerank_delta`` -- Sec. 6 "PageRank" with its switch to push: FP64 pull
                    iterations, then pushes of the rank changes still above
                    a threshold (accumulative delta iteration).
* ``bfs_par``, ``kcore_par``, ``pagerank_par`` -- the same results computed
                    with OpenMP on every host core, only to time the CPU
                    baseline; pinned equal to the single-threaded functions.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` against brute force, closed forms or invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

UNREACHED_LEVEL = -1
UNREACHED_DIST = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (gcc -O2).  The definitions are
    single-threaded; only the ``*_par`` timing variants use OpenMP, and the
    library is built without it (those variants then run on one thread) if
    the compiler has no OpenMP runtime."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-fvisibility=hidden", _SRC, "-o", tmp]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], capture_output=True)
        if r.returncode != 0:
            subprocess.check_call(base + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i64, i32, u32, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_uint32, ctypes.c_double)
        lib.or_bfs.argtypes = [i64, vp, vp, i32, vp]
        lib.or_bfs.restype = ctypes.c_int
        lib.or_sssp.argtypes = [i64, vp, vp, vp, i32, vp]
        lib.or_sssp.restype = ctypes.c_int
        lib.or_sssp_bsp.argtypes = [i64, vp, vp, vp, i32, i64, vp]
        lib.or_sssp_bsp.restype = i64
        lib.or_kcore.argtypes = [i64, vp, vp, u32, vp, vp]
        lib.or_kcore.restype = ctypes.c_int
        lib.or_coreness.argtypes = [i64, vp, vp, vp]
        lib.or_coreness.restype = ctypes.c_int
        lib.or_wcc.argtypes = [i64, vp, vp, vp]
        lib.or_wcc.restype = ctypes.c_int
        lib.or_pagerank.argtypes = [i64, vp, vp, vp, dbl, dbl, i64, i64, vp, vp]
        lib.or_pagerank.restype = i64
        lib.or_pagerank_delta.argtypes = [i64, vp, vp, vp, vp, dbl, dbl, i64, dbl, dbl, dbl, vp,
                                          ctypes.POINTER(i64), ctypes.POINTER(dbl)]
        lib.or_pagerank_delta.restype = i64
        lib.or_bfs_par.argtypes = [i64, vp, vp, i32, vp]
        lib.or_bfs_par.restype = ctypes.c_int
        lib.or_kcore_par.argtypes = [i64, vp, vp, u32, vp, vp]
        lib.or_kcore_par.restype = ctypes.c_int
        lib.or_pagerank_par.argtypes = [i64, vp, vp, vp, dbl, dbl, i64, i64, vp, vp]
        lib.or_pagerank_par.restype = i64
        lib.or_threads.argtypes = []
        lib.or_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _csr(off, idx):
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    return off, idx, (idx.ctypes.data if idx.size else None)


def bfs(off, idx, src: int) -> np.ndarray:
    """BFS level of every vertex from `src` (-1 if unreached)."""
    off, idx, ip = _csr(off, idx)
    n = off.size - 1
    lev = np.empty(n, dtype=np.int32)
    if _load().or_bfs(n, off.ctypes.data, ip, int(src), lev.ctypes.data) != 0:
        raise ValueError("source out of range")
    return lev


def sssp(off, idx, w, src: int) -> np.ndarray:
    """Shortest-path distance of every vertex from `src` (UINT32_MAX if unreached)."""
    off, idx, ip = _csr(off, idx)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    n = off.size - 1
    dist = np.empty(n, dtype=np.uint32)
    rc = _load().or_sssp(n, off.ctypes.data, ip, w.ctypes.data if w.size else None, int(src),
                         dist.ctypes.data)
    if rc == 1:
        raise ValueError("source out of range")
    if rc == 2:
        raise OverflowError("a distance does not fit in uint32")
    return dist


def sssp_bsp(off, idx, w, src: int, max_it: int = 64) -> np.ndarray:
    """Distance arrays after each BSP iteration (shape [iterations, n])."""
    off, idx, ip = _csr(off, idx)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    n = off.size - 1
    hist = np.empty((max_it, n), dtype=np.uint32)
    it = _load().or_sssp_bsp(n, off.ctypes.data, ip, w.ctypes.data if w.size else None,
                             int(src), max_it, hist.ctypes.data)
    return hist[:it].copy()


def kcore(off, idx, k: int):
    """(in_core uint8[n], resid uint32[n]) of the k-core by peeling."""
    off, idx, ip = _csr(off, idx)
    n = off.size - 1
    inc = np.empty(n, dtype=np.uint8)
    res = np.empty(n, dtype=np.uint32)
    _load().or_kcore(n, off.ctypes.data, ip, int(k), inc.ctypes.data, res.ctypes.data)
    return inc, res


def coreness(off, idx) -> np.ndarray:
    """Core number of every vertex (Batagelj-Zaversnik)."""
    off, idx, ip = _csr(off, idx)
    n = off.size - 1
    core = np.zeros(n, dtype=np.uint32)
    _load().or_coreness(n, off.ctypes.data, ip, core.ctypes.data)
    return core


def wcc(off, idx) -> np.ndarray:
    """Label of every vertex: the smallest vertex id of its component."""
    off, idx, ip = _csr(off, idx)
    n = off.size - 1
    label = np.empty(n, dtype=np.uint32)
    _load().or_wcc(n, off.ctypes.data, ip, label.ctypes.data)
    return label


def pagerank(in_off, in_idx, outdeg=None, d: float = 0.85, tol: float = 1e-6,
             max_iter: int = 1000, fixed_iter: int = -1):
    """FP64 Jacobi PageRank.

    Readings of what the paper leaves unstated (Sec. 6 "PageRank" gives only
    "pull, sum, iterate until stable"): teleport (1-d)/n, start x_0 = 1/n,
    rank of out-degree-0 vertices spread uniformly over all vertices, stop
    after the first iteration whose L1 change is below `tol`.  For a
    symmetric graph pass the CSR itself as ``in_off/in_idx``; ``outdeg``
    defaults to its degrees.  Returns (x float64[n], iterations, last L1).
    """
    off, idx, ip = _csr(in_off, in_idx)
    n = off.size - 1
    od = np.diff(off) if outdeg is None else np.asarray(outdeg)
    od = np.ascontiguousarray(od, dtype=np.int64)
    x = np.empty(max(n, 1), dtype=np.float64)
    l1 = ctypes.c_double(0.0)
    it = _load().or_pagerank(n, off.ctypes.data, ip, od.ctypes.data, float(d), float(tol),
                             int(max_iter), int(fixed_iter), x.ctypes.data, ctypes.byref(l1))
    return x[:n], int(it), float(l1.value)


def pagerank_delta(off, idx, in_off=None, in_idx=None, d: float = 0.85, tol: float = 1e-6,
                   max_iter: int = 1000, alpha: float = 8.0, theta: float = 2.0, rho_min: float = 0.6):
    """FP64 PageRank that pulls first and, once the pull contracts slowly
    (L1 at least rho_min times the previous L1) and the vertices whose
    change exceeds theta * (previous L1) / n hold fewer than E / alpha
    out-edges, pushes the remaining rank changes (Sec. 6 "PageRank": pull,
    then push when most vertices are stable; the switch rule is a reading
    of the paper's undescribed decision tree).  Out-edges ``off/idx``; in-edges
    ``in_off/in_idx`` (default: the CSR itself, a symmetric graph).  Stops
    when the L1 change (pull) or the L1 of the pending changes (push) is
    below ``tol``; the result is then within d / (1 - d) * tol of the fixed
    point in L1.  Returns (x float64[n], iterations, pull iterations, last
    L1)."""
    off, idx, ip = _csr(off, idx)
    if in_off is None:
        ioff, iidx, iip = off, idx, ip
    else:
        ioff, iidx, iip = _csr(in_off, in_idx)
    n = off.size - 1
    x = np.empty(max(n, 1), dtype=np.float64)
    pulls = ctypes.c_int64(0)
    l1 = ctypes.c_double(0.0)
    it = _load().or_pagerank_delta(n, off.ctypes.data, ip, ioff.ctypes.data, iip, float(d), float(tol),
                                   int(max_iter), float(alpha), float(theta), float(rho_min), x.ctypes.data,
                                   ctypes.byref(pulls), ctypes.byref(l1))
    return x[:n], int(it), int(pulls.value), float(l1.value)


# ------------------------------------------------ parallel timing variants
def threads() -> int:
    """Threads the ``*_par`` variants run on (OpenMP's default team size)."""
    return int(_load().or_threads())


def bfs_par(off, idx, src: int) -> np.ndarray:
    """``bfs`` computed level-synchronously on all host cores."""
    off, idx, ip = _csr(off, idx)
    n = off.size - 1
    lev = np.empty(n, dtype=np.int32)
    if _load().or_bfs_par(n, off.ctypes.data, ip, int(src), lev.ctypes.data) != 0:
        raise ValueError("source out of range")
    return lev


def kcore_par(off, idx, k: int):
    """``kcore`` computed by level-synchronous peeling on all host cores."""
    off, idx, ip = _csr(off, idx)
    n = off.size - 1
    inc = np.empty(n, dtype=np.uint8)
    res = np.empty(n, dtype=np.uint32)
    _load().or_kcore_par(n, off.ctypes.data, ip, int(k), inc.ctypes.data, res.ctypes.data)
    return inc, res


def pagerank_par(in_off, in_idx, outdeg=None, d: float = 0.85, tol: float = 1e-6,
                 max_iter: int = 1000, fixed_iter: int = -1):
    """``pagerank`` with each iteration's per-vertex pulls on all host cores
    (same values bit for bit)."""
    off, idx, ip = _csr(in_off, in_idx)
    n = off.size - 1
    od = np.diff(off) if outdeg is None else np.asarray(outdeg)
    od = np.ascontiguousarray(od, dtype=np.int64)
    x = np.empty(max(n, 1), dtype=np.float64)
    l1 = ctypes.c_double(0.0)
    it = _load().or_pagerank_par(n, off.ctypes.data, ip, od.ctypes.data, float(d), float(tol),
                                 int(max_iter), int(fixed_iter), x.ctypes.data, ctypes.byref(l1))
    return x[:n], int(it), float(l1.value)
