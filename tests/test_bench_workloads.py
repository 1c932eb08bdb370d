"""Host logic of bench.py on CPU: every single-query workload's algorithms
have work accounting and a hashable kernel source, and the algorithmic byte
counts follow their stated formulas on a small graph."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import graphgen as gg  # noqa: E402
import oracle  # noqa: E402


@pytest.mark.parametrize("name", [k for k, v in bench.WORKLOADS.items() if v["kind"] in ("rmat", "grid")])
def test_workload_algorithms_are_accounted(name):
    g = gg.rmat(8)
    for alg in bench.WORKLOADS[name]["algs"]:
        out = np.zeros(g.n, dtype=np.int32)
        if alg == "sssp":
            out = np.zeros(g.n, dtype=np.uint32)
        edges, nbytes = bench.algorithmic(alg, g, bench.WORKLOADS[name]["bits"], out, 3)
        assert edges > 0 and nbytes > 0, (name, alg)
        assert len(bench.kernel_source_hash(alg + "_kernel")) == 16


def test_algorithmic_bytes_formulas():
    g = gg.rmat(9)
    n, e = g.n, g.e
    lev = oracle.bfs(g.offsets, g.indices, 0)
    reached = lev >= 0
    e_c = int(g.degrees()[reached].sum())
    n_c = int(reached.sum())
    assert bench.algorithmic("bfs", g, 32, lev, 1) == (e_c // 2, 4 * e_c + 20 * n_c)
    assert bench.algorithmic("bfs", g, 64, lev, 1) == (e_c // 2, 4 * e_c + 28 * n_c)
    assert bench.algorithmic("kcore", g, 32, None, 1) == (e // 2, 4 * e + 9 * n)
    assert bench.algorithmic("coreness", g, 64, None, 1) == (e // 2, 4 * e + 24 * n)
    assert bench.algorithmic("wcc", g, 32, None, 1) == (e // 2, 4 * e + 20 * n)
    assert bench.algorithmic("pagerank", g, 32, None, 7) == ((e // 2) * 7, (4 * e + 20 * n) * 7)


def test_kernel_sources_map_to_files():
    csrc = os.path.join(ROOT, "paper_1812_04070_gb300", "csrc")
    for kernel in ("bfs_kernel", "sssp_kernel", "kcore_kernel", "pagerank_kernel", "coreness_kernel", "wcc_kernel"):
        own = bench.KERNEL_FILES.get(kernel, kernel.replace("_kernel", "") + ".cu")
        assert os.path.exists(os.path.join(csrc, own)), kernel
    # a coreness record follows kcore.cu, a WCC record sssp.cu
    assert bench.KERNEL_FILES["coreness_kernel"] == "kcore.cu"
    assert bench.KERNEL_FILES["wcc_kernel"] == "sssp.cu"


def test_traffic_records_name_existing_summaries():
    import json
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        recs = json.load(f)
    for key, rec in recs.items():
        workload, kernel = key.split(":")
        assert workload in bench.WORKLOADS, key
        assert os.path.exists(os.path.join(ROOT, rec["summary"])), key
        assert rec["bytes_per_launch"] > 0 and len(rec["source_hash"]) == 16


def test_kernel_hash_ignores_comments_only():
    a = "__global__ void k(int* p) { p[0] = 1; }  // store\n"
    b = "/* the kernel */\n__global__ void k(int* p) {\n  p[0] = 1;\n}\n"
    c = "__global__ void k(int* p) { p[0] = 2; }\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)


def test_inspected_bytes_and_defaults():
    class St:
        edges_visited = 1000
    assert bench.inspected_bytes("bfs", 64, St, 10) == 4 * 1000 + 28 * 10
    assert bench.inspected_bytes("sssp", 32, St, 10) == 8 * 1000 + 20 * 10
    assert bench.inspected_bytes("pagerank", 32, St, 10) is None
    assert set(bench.BYTES_BASIS) >= {"bfs", "sssp", "kcore", "coreness", "wcc", "pagerank"}
    # the headline configuration is the default line
    import sys as _s
    argv, _s.argv = _s.argv, ["bench.py"]
    try:
        assert bench.parse().workload == "rmat24-bfs"
    finally:
        _s.argv = argv


def test_cpu_leg_parallel_and_serial_agree_on_work():
    g = gg.rmat(10)
    w = gg.weights(g, 1, 1, 64)
    bench.WORKLOADS["_tiny"] = dict(kind="rmat", scale=10, bits=32, algs=["bfs", "kcore", "pagerank"], desc="")
    try:
        a = bench.cpu_leg("_tiny", g, w, 0.0, parallel=True)
        b = bench.cpu_leg("_tiny", g, w, 0.0, parallel=False)
    finally:
        del bench.WORKLOADS["_tiny"]
    assert a["cores"] == oracle.threads() and b["cores"] == 1
    assert a["value"] > 0 and b["value"] > 0 and "OpenMP" in a["sample"]
