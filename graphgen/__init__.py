"""Seeded synthetic graph inputs shared by the CPU oracle and the CUDA path.

This module holds none of the graph method's arithmetic: it only builds
inputs (CSR graphs, edge weights, source vertices).  The shapes follow the
paper's workloads (Sec. 6, Table 3): Graph500-style R-MAT / Kronecker graphs
with (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), symmetrised, self loops and
duplicate edges removed, in CSR (Sec. 6, "Storage Format"); random integer
edge weights (Sec. 6); and a 4-neighbour grid as the high-diameter stand-in
for the road graphs ER and RC.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None

RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile libgraphgen.so in place (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-fvisibility=hidden", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i64, u64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        lib.gg_rmat.argtypes = [i32, i32, dbl, dbl, dbl, u64]
        lib.gg_rmat.restype = vp
        lib.gg_rmat_sub.argtypes = [i64, i32, i64, dbl, dbl, dbl, u64]
        lib.gg_rmat_sub.restype = vp
        lib.gg_grid.argtypes = [i64, i64]
        lib.gg_grid.restype = vp
        lib.gg_from_edges.argtypes = [i64, i64, vp, vp]
        lib.gg_from_edges.restype = vp
        lib.gg_n.argtypes = [vp]
        lib.gg_n.restype = i64
        lib.gg_e.argtypes = [vp]
        lib.gg_e.restype = i64
        lib.gg_copy.argtypes = [vp, vp, vp]
        lib.gg_copy.restype = None
        lib.gg_free.argtypes = [vp]
        lib.gg_free.restype = None
        lib.gg_weights.argtypes = [i64, vp, vp, u64, ctypes.c_uint32, ctypes.c_uint32, vp]
        lib.gg_weights.restype = None
        lib.gg_pick_sources.argtypes = [i64, vp, i64, u64, vp]
        lib.gg_pick_sources.restype = i64
        lib.gg_splitmix64.argtypes = [u64]
        lib.gg_splitmix64.restype = u64
        _lib = lib
    return _lib


@dataclass
class Graph:
    """A symmetric graph in CSR: offsets int64[n+1], indices int32[e]."""
    offsets: np.ndarray
    indices: np.ndarray
    name: str = ""
    weights: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def e(self) -> int:
        return int(self.indices.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)


def _take(handle, name: str) -> Graph:
    lib = _load()
    try:
        n, e = lib.gg_n(handle), lib.gg_e(handle)
        off = np.empty(n + 1, dtype=np.int64)
        idx = np.empty(max(e, 0), dtype=np.int32)
        lib.gg_copy(handle, off.ctypes.data, idx.ctypes.data if e else None)
    finally:
        lib.gg_free(handle)
    return Graph(off, idx, name)


def graph_seed(scale: int) -> int:
    """Seed of the R-MAT graph at `scale`."""
    return 0x51D0000 + scale


def weight_seed(scale: int) -> int:
    return graph_seed(scale) ^ 0xFFFF


def rmat(scale: int, edge_factor: int = 16, seed: int | None = None,
         abc: tuple = RMAT_ABC) -> Graph:
    """Symmetrised R-MAT graph with 2^scale vertices and edge_factor*2^scale tuples."""
    seed = graph_seed(scale) if seed is None else seed
    g = _take(_load().gg_rmat(scale, edge_factor, abc[0], abc[1], abc[2], seed),
              f"rmat{scale}_ef{edge_factor}")
    g.meta.update(kind="rmat", scale=scale, edge_factor=edge_factor, seed=seed)
    return g


def rmat_sub(n: int, tuples: int, seed: int, abc: tuple = RMAT_ABC) -> Graph:
    """R-MAT restricted to vertices < n (drawn at scale ceil(log2 n))."""
    scale = max(1, int(np.ceil(np.log2(max(n, 2)))))
    g = _take(_load().gg_rmat_sub(n, scale, tuples, abc[0], abc[1], abc[2], seed),
              f"rmatsub{n}")
    g.meta.update(kind="rmat_sub", n=n, tuples=tuples, seed=seed)
    return g


def grid(rows: int, cols: int) -> Graph:
    """rows x cols 4-neighbour grid, vertex id r*cols + c, no wrap-around."""
    g = _take(_load().gg_grid(rows, cols), f"grid{rows}x{cols}")
    g.meta.update(kind="grid", rows=rows, cols=cols)
    return g


def from_edges(n: int, src, dst, name: str = "edges") -> Graph:
    """Symmetric CSR from an undirected edge list (loops and duplicates dropped)."""
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32))
    assert s.shape == d.shape
    if s.size and (s.min() < 0 or d.min() < 0 or max(s.max(), d.max()) >= n):
        raise ValueError("edge endpoint out of range")
    h = _load().gg_from_edges(n, s.size, s.ctypes.data if s.size else None,
                              d.ctypes.data if d.size else None)
    return _take(h, name)


def weights(g: Graph, seed: int, lo: int = 1, hi: int = 64) -> np.ndarray:
    """uint32 weights in [lo, hi], one value per undirected edge (both directions agree)."""
    w = np.empty(g.e, dtype=np.uint32)
    if g.e:
        _load().gg_weights(g.n, g.offsets.ctypes.data, g.indices.ctypes.data, seed, lo, hi,
                           w.ctypes.data)
    return w


def pick_sources(g: Graph, k: int, seed: int) -> np.ndarray:
    """k distinct non-isolated vertices, uniform, seeded."""
    out = np.empty(max(k, 1), dtype=np.int32)
    got = _load().gg_pick_sources(g.n, g.offsets.ctypes.data, k, seed, out.ctypes.data)
    return out[:got].copy()


def splitmix64(x: int) -> int:
    return int(_load().gg_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def _u01(seed: int, i: int) -> float:
    return (splitmix64(seed ^ splitmix64(i)) >> 11) / float(1 << 53)


def random_graph(n: int, m: int, seed: int) -> Graph:
    """Small Erdos-Renyi-like multigraph draw (m tuples), deduplicated."""
    if n == 0:
        return Graph(np.zeros(1, np.int64), np.zeros(0, np.int32), "empty")
    src = [int(_u01(seed, 2 * i) * n) for i in range(m)]
    dst = [int(_u01(seed, 2 * i + 1) * n) for i in range(m)]
    return from_edges(n, src, dst, f"er{n}_{m}")


def star(n: int) -> Graph:
    return from_edges(n, [0] * (n - 1), list(range(1, n)), f"star{n}")


def path(n: int) -> Graph:
    return from_edges(n, list(range(n - 1)), list(range(1, n)), f"path{n}")


def complete(n: int) -> Graph:
    s, d = np.triu_indices(n, 1)
    return from_edges(n, s, d, f"complete{n}")


def multigraph_batch(count: int = 256, seed: int = 0xBA7C4, n_lo: int = 1000,
                     n_hi: int = 100000, ef_lo: int = 8, ef_hi: int = 32):
    """`count` independent R-MAT graphs (n log-uniform in [n_lo, n_hi], edge factor
    uniform in [ef_lo, ef_hi]) and one non-isolated source per graph."""
    graphs, sources = [], []
    for i in range(count):
        n = int(round(np.exp(np.log(n_lo) + _u01(seed, 3 * i) * (np.log(n_hi) - np.log(n_lo)))))
        ef = ef_lo + int(_u01(seed, 3 * i + 1) * (ef_hi - ef_lo + 1))
        gs = splitmix64(seed + i)
        g = rmat_sub(n, ef * n, gs)
        src = pick_sources(g, 1, gs ^ 0x5A5A)
        graphs.append(g)
        sources.append(int(src[0]) if src.size else 0)
    return graphs, np.asarray(sources, dtype=np.int32)


def pack(graphs) -> tuple[Graph, np.ndarray]:
    """Block-diagonal packing; returns the packed graph and per-graph vertex bases."""
    bases = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        bases[i + 1] = bases[i] + g.n
    offs = [np.zeros(1, np.int64)]
    idxs = []
    run = 0
    for i, g in enumerate(graphs):
        offs.append(g.offsets[1:] + run)
        idxs.append(g.indices + np.int32(bases[i]))
        run += g.e
    off = np.concatenate(offs)
    idx = np.concatenate(idxs) if idxs else np.zeros(0, np.int32)
    return Graph(off, idx.astype(np.int32), f"pack{len(graphs)}"), bases
