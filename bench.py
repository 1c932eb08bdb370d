#!/usr/bin/env python3
"""Benchmark of the ACC graph hot path on GB300.

Default workload (the headline configuration): BFS from vertex 0 on a
symmetrised R-MAT graph at scale 24 (16,777,216 vertices, edge factor 16,
a/b/c/d = 0.57/0.19/0.19/0.05, 520,767,798 directed edges), int64 offsets
and int32 indices, one persistent kernel per query through the C ABI.
Other workloads (--workload): rmat20 (SSSP + k-core 16 + PageRank on R-MAT
scale 20, int32 CSR), rmat16-bfs, rmat24-sssp, rmat24-pagerank,
rmat24-kcore, rmat20-coreness, rmat24-coreness (k-core decomposition),
rmat20-wcc, rmat24-wcc (connected components), rmat22-bfs, rmat22-sssp
(profiling sizes), grid4096-bfs, grid4096-sssp, batch22, serve.

Metric: GTEPS = traversed undirected edges per second (Graph500 counting:
BFS / SSSP count the edges of the component reached from the source, k-core
counts every edge once, PageRank counts every edge once per iteration).

Timing: W untimed warm-up steps, then K timed steps.  A step is a batch of
R queries of the workload (R chosen so that a step holds about 0.125 s of
GPU time, or --queries); before every query the L2 is flushed (a 512 MB
write) outside the timed brackets, and every kernel launch is bracketed by
CUDA events on the launching stream.  `value` = edges of all timed queries
over the sum of their kernel times.  The roofline object reports the
dominant kernel's bytes three ways: the algorithmic bytes of the scope
table, the bytes of the edges the kernel actually inspected (its own edge
counter), and the DRAM bytes of one ncu capture when one was taken on the
current kernel sources.  `e2e` repeats a query through the public API with
HOST buffers: the graph is uploaded from pinned memory
(simdx_graph_create) and the result is read back, all inside the timed
region.  `cpu_baseline` times the oracle on the host cores: its OpenMP
variants on every core (BFS, k-core, PageRank) and the single-threaded
definitions.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

L2_FLUSH_BYTES = 512 << 20

WORKLOADS = {
    "rmat20": dict(kind="rmat", scale=20, bits=32, algs=["sssp", "kcore", "pagerank"],
                   desc="R-MAT scale 20 (n=1,048,576, ef 16), int32 CSR, w in [1,64]: "
                        "SSSP src 0 + k-core k=16 + PageRank d=0.85 tol 1e-6"),
    "rmat24-bfs": dict(kind="rmat", scale=24, bits=64, algs=["bfs"],
                       desc="R-MAT scale 24 (n=16,777,216, ef 16), int64 offsets: BFS src 0"),
    "rmat24-sssp": dict(kind="rmat", scale=24, bits=64, algs=["sssp"],
                        desc="R-MAT scale 24, int64 offsets, w in [1,64]: SSSP src 0"),
    "rmat24-pagerank": dict(kind="rmat", scale=24, bits=64, algs=["pagerank"],
                            desc="R-MAT scale 24, int64 offsets: PageRank d=0.85 tol 1e-6"),
    "rmat24-kcore": dict(kind="rmat", scale=24, bits=64, algs=["kcore"],
                         desc="R-MAT scale 24, int64 offsets: k-core k=16"),
    "rmat20-kcore": dict(kind="rmat", scale=20, bits=32, algs=["kcore"],
                         desc="R-MAT scale 20, int32 CSR: k-core k=16 (profiling size)"),
    "rmat20-pagerank": dict(kind="rmat", scale=20, bits=32, algs=["pagerank"],
                            desc="R-MAT scale 20, int32 CSR: PageRank d=0.85 tol 1e-6 (profiling size)"),
    "rmat20-sssp": dict(kind="rmat", scale=20, bits=32, algs=["sssp"],
                        desc="R-MAT scale 20, int32 CSR, w in [1,64]: SSSP src 0 (profiling size)"),
    "rmat20-coreness": dict(kind="rmat", scale=20, bits=32, algs=["coreness"],
                            desc="R-MAT scale 20, int32 CSR: k-core decomposition (coreness of every vertex)"),
    "rmat24-coreness": dict(kind="rmat", scale=24, bits=64, algs=["coreness"],
                            desc="R-MAT scale 24, int64 offsets: k-core decomposition (coreness of every vertex)"),
    "rmat20-wcc": dict(kind="rmat", scale=20, bits=32, algs=["wcc"],
                       desc="R-MAT scale 20, int32 CSR: weakly connected components (min-label propagation)"),
    "rmat24-wcc": dict(kind="rmat", scale=24, bits=64, algs=["wcc"],
                       desc="R-MAT scale 24, int64 offsets: weakly connected components"),
    "rmat22-bfs": dict(kind="rmat", scale=22, bits=32, algs=["bfs"],
                       desc="R-MAT scale 22 (n=4,194,304, ef 16), int32 CSR: BFS src 0 (profiling size)"),
    "rmat22-sssp": dict(kind="rmat", scale=22, bits=32, algs=["sssp"],
                        desc="R-MAT scale 22 (n=4,194,304, ef 16), int32 CSR, w in [1,64]: SSSP src 0 (profiling size)"),
    "rmat16-bfs": dict(kind="rmat", scale=16, bits=32, algs=["bfs"],
                       desc="R-MAT scale 16 (n=65,536, ef 16), int32 CSR: BFS src 0"),
    "grid4096-bfs": dict(kind="grid", rows=4096, bits=64, algs=["bfs"],
                         desc="4096x4096 4-neighbour grid: BFS from corner 0"),
    "grid4096-sssp": dict(kind="grid", rows=4096, bits=64, algs=["sssp"], wmax=1000,
                          desc="4096x4096 4-neighbour grid, w in [1,1000]: SSSP from corner 0"),
    "grid4096-pagerank": dict(kind="grid", rows=4096, bits=64, algs=["pagerank"],
                              desc="4096x4096 4-neighbour grid: PageRank d=0.85 tol 1e-6 (pull, then push once "
                                   "the pull contracts slowly and few vertices are unstable)"),
    "grid4096-ablation": dict(kind="ablation", graph="grid", rows=4096, bits=64, algs=["bfs", "sssp"],
                              wmax=1000,
                              desc="4096x4096 4-neighbour grid (w in [1,1000]), BFS / SSSP from corner 0: all, "
                                   "selective and no kernel fusion (Sec. 5, Table 2); JIT vs ballot-only filter"),
    "grid4096-pr-ablation": dict(kind="ablation", graph="grid", rows=4096, bits=64, algs=["pagerank"],
                                 desc="4096x4096 4-neighbour grid: PageRank pull then push (Sec. 6) vs pull only"),
    "rmat20-ablation": dict(kind="ablation", graph="rmat", scale=20, bits=32,
                            algs=["pagerank", "sssp", "kcore", "bfs"],
                            desc="R-MAT scale 20, int32 CSR: the ablations of rmat24-ablation at the default "
                                 "workload's size"),
    "rmat24-ablation": dict(kind="ablation", graph="rmat", scale=24, bits=64,
                            algs=["bfs", "sssp", "kcore", "pagerank"],
                            desc="R-MAT scale 24, int64 offsets: BFS / SSSP src 0, k-core 16 and PageRank under all, "
                                 "selective and no kernel fusion (BFS, SSSP); JIT vs ballot-only filter (Sec. 4); PageRank switch to push vs pull only"),
    "batch22": dict(kind="batch", scale=22, bits=32,
                    desc="R-MAT scale 22 (n=4,194,304, ef 16, w in [1,64]): 64 BFS + 64 SSSP sources uniform over "
                         "non-isolated vertices (seed 0xBA7C4), batched vs one call per query; plus 256 R-MAT "
                         "graphs (n log-uniform in [1k,100k], ef 8..32) packed block-diagonally, multi-root BFS vs "
                         "256 calls"),
    "serve": dict(kind="serve", bits=32,
                  desc="8 resident R-MAT graphs (scales 14,15,16,17,18,19,20,22; w in [1,64]); Poisson arrivals "
                       "1k..50k/s; mix 50% BFS / 40% SSSP / 10% k-core(16); graph uniform; source uniform "
                       "non-isolated (seed 0x5E77E); continuous-batching server vs one call per query"),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="simdx", choices=["simdx", "reference"])
    p.add_argument("--workload", default="rmat24-bfs", choices=list(WORKLOADS))
    p.add_argument("--queries", type=int, default=0,
                   help="queries per step (0: as many as make about 0.125 s of GPU time)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--autotune", action="store_true",
                   help="before warm-up, tune each algorithm's knobs (simdx_autotune) on its own copy of the "
                        "graph; the timed steps and e2e use the tuned knobs")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def max_over_ranks(x: float, world: int) -> float:
    """The largest x over all ranks (a job lasts as long as its slowest
    rank).  Every rank must call it."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput of `world` replicas that each processed
    `units_per_rank` units: all units over the slowest rank's time."""
    return units_per_rank * world / max_over_ranks(seconds, world)


def make_graph(wl):
    import graphgen as gg
    if wl["kind"] == "rmat" or wl.get("graph") == "rmat":
        g = gg.rmat(wl["scale"])
        w = gg.weights(g, gg.weight_seed(wl["scale"]), 1, wl.get("wmax", 64))
    else:
        g = gg.grid(wl["rows"], wl["rows"])
        w = gg.weights(g, 0x6121D ^ 0xFFFF, 1, wl.get("wmax", 1000))
    return g, w


def s_off(bits):
    return bits // 8


# ------------------------------------------------------------ clocks sampling
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={','.join(self.FIELDS)}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KERNEL_FILES = {"coreness_kernel": "kcore.cu", "wcc_kernel": "sssp.cu"}  # kernels not in <algorithm>.cu


def _code_only(text: str) -> str:
    """Source text without comments and with whitespace runs collapsed, so
    that editing a comment does not count as changing a kernel."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(kernel: str) -> str:
    """Hash of the code a kernel is built from (comments and layout
    ignored): its own file (<algorithm>.cu for <algorithm>_kernel) and the
    shared device headers (*.cuh; the host-side header declares no device
    code)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1812_04070_gb300", "csrc")
    own = KERNEL_FILES.get(kernel, kernel.replace("_kernel", "") + ".cu")
    headers = sorted(os.path.basename(p) for p in glob.glob(os.path.join(csrc, "*.cuh")))
    for fn in [own] + headers:
        with open(os.path.join(csrc, fn), encoding="utf-8") as f:
            h.update(fn.encode())
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        rec = d[f"{workload}:{kernel}"]
        if rec.get("source_hash") != kernel_source_hash(kernel):
            return None
        return float(rec["bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


# ------------------------------------------------------------ work accounting
def reached_edges(g, reached_mask):
    deg = g.degrees()
    e_c = int(deg[reached_mask].sum())
    return e_c, int(reached_mask.sum())


def algorithmic(alg, g, bits, out, iters, st=None):
    """(undirected traversed edges, algorithmic bytes) of one call.  A
    PageRank run that switched to push counts its pull iterations as above
    and each push iteration as a scan of the pending changes (8 bytes per
    vertex) plus 12 bytes per pushed edge (index, 64-bit add), with the
    pushed edges from the run's own edge counter."""
    so = s_off(bits)
    n, e = g.n, g.e
    if alg == "bfs":
        e_c, n_c = reached_edges(g, out >= 0)
        return e_c // 2, 4 * e_c + (2 * so + 4 + 8) * n_c
    if alg == "sssp":
        e_c, n_c = reached_edges(g, out != 0xFFFFFFFF)
        return e_c // 2, 8 * e_c + (2 * so + 4 + 8) * n_c
    if alg == "kcore":
        return e // 2, 4 * e + (2 * so + 1) * n
    if alg == "coreness":
        return e // 2, 4 * e + (2 * so + 8) * n
    if alg == "wcc":
        return e // 2, 4 * e + (2 * so + 12) * n
    if alg == "pagerank":
        if st is not None and st.push_iters > 0:
            pulls = st.pull_iters
            pushed = max(0, st.edges_visited - pulls * e)
            return (e // 2) * pulls + pushed // 2, (4 * e + (2 * so + 12) * n) * pulls + \
                st.push_iters * 8 * n + 12 * pushed
        return (e // 2) * iters, (4 * e + (2 * so + 12) * n) * iters
    raise ValueError(alg)


BYTES_BASIS = {
    "bfs": "4*E_c + (2*s_off + 4 + 8)*n_c: every edge of the reached component read once",
    "sssp": "8*E_c + (2*s_off + 4 + 8)*n_c: every edge (index + weight) of the reached component once",
    "kcore": "4*E + (2*s_off + 1)*n",
    "coreness": "4*E + (2*s_off + 8)*n",
    "wcc": "4*E + (2*s_off + 12)*n",
    "pagerank": "(4*E + (2*s_off + 12)*n) per iteration",
}
INSPECTED_BASIS = {
    "bfs": "4*(edge entries the kernel read) + (2*s_off + 12)*n_c; pull levels stop at the first frontier "
           "in-neighbour",
    "sssp": "8*(edge entries the kernel relaxed, re-relaxations included) + (2*s_off + 12)*n_c",
}


def inspected_bytes(alg, bits, st, n_c):
    """Bytes of the edges a launch actually read (its own counter), with the
    same per-vertex term as the algorithmic count; None where the two are
    the same by construction."""
    so = s_off(bits)
    if alg == "bfs":
        return 4 * st.edges_visited + (2 * so + 12) * n_c
    if alg == "sssp":
        return 8 * st.edges_visited + (2 * so + 12) * n_c
    return None


# ------------------------------------------------------------ the GPU arm
def run_simdx(args, rank, world, local):
    import torch
    from paper_1812_04070_gb300 import Graph, build, simdx_stats

    wl = WORKLOADS[args.workload]
    torch.cuda.set_device(local)
    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
    build()
    g, w = make_graph(wl)
    bits = wl["bits"]
    off = g.offsets if bits == 64 else g.offsets.astype(np.int32)
    G = Graph(off, g.indices, weights=w)
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", local)
    algs = wl["algs"]
    graphs = {a: G for a in algs}
    tuned, tuned_full, tune_s = {}, {}, 0.0
    if args.autotune and not {"coreness", "wcc"} & set(algs):
        from paper_1812_04070_gb300 import simdx
        code = {"bfs": simdx.ALGO_BFS, "sssp": simdx.ALGO_SSSP, "kcore": simdx.ALGO_KCORE,
                "pagerank": simdx.ALGO_PAGERANK}
        arg = {"bfs": 0, "sssp": 0, "kcore": 16, "pagerank": 0}
        default = {k: getattr(G.config, k) for k, _ in G.config._fields_ if k != "reserved"}
        t0 = time.time()
        for i, a in enumerate(algs):
            Ga = G if i == 0 else Graph(off, g.indices, weights=w)
            best, _ = Ga.autotune(code[a], arg[a], reps=3)
            graphs[a] = Ga
            tuned_full[a] = best
            tuned[a] = {k: v for k, v in best.items() if v != default[k]}
        tune_s = time.time() - t0
    outs = {
        "bfs": torch.empty(g.n, dtype=torch.int32, device=dev),
        "sssp": torch.empty(g.n, dtype=torch.int32, device=dev),
        "kcore": (torch.empty(g.n, dtype=torch.uint8, device=dev), torch.empty(g.n, dtype=torch.int32, device=dev)),
        "pagerank": torch.empty(g.n, dtype=torch.float32, device=dev),
        "coreness": torch.empty(g.n, dtype=torch.int32, device=dev),
        "wcc": torch.empty(g.n, dtype=torch.int32, device=dev),
    }
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def launch(alg, st=None):
        Ga = graphs[alg]
        if alg == "bfs":
            Ga.bfs(0, out=outs["bfs"], stats=st)
        elif alg == "sssp":
            Ga.sssp(0, out=outs["sssp"], stats=st)
        elif alg == "kcore":
            Ga.kcore(16, out=outs["kcore"][0], resid=outs["kcore"][1], stats=st)
        elif alg == "coreness":
            Ga.coreness(out=outs["coreness"], stats=st)
        elif alg == "wcc":
            Ga.wcc(out=outs["wcc"], stats=st)
        else:
            Ga.pagerank(0.85, 1e-6, 1000, out=outs["pagerank"], stats=st)

    calls = {"wcc": 2}  # kernel launches per call (WCC: hub BFS + propagation)
    evs = {a: [] for a in algs}

    def query(record):
        flush.zero_()
        for a in algs:
            if record:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            launch(a)
            if record:
                e1.record(stream)
                evs[a].append((e0, e1))

    for _ in range(max(args.warmup, 3)):
        query(False)
    torch.cuda.synchronize()
    # queries per step: about 0.125 s of GPU time, so that K steps span
    # seconds of clock samples (20 steps: about 2.5 s)
    if args.queries > 0:
        R = args.queries
    else:
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(3):
            query(False)
        q1.record(stream)
        torch.cuda.synchronize()
        R = int(min(4096, max(1, round(0.125 / (q0.elapsed_time(q1) / 3 / 1e3)))))
    for _ in range(args.warmup):
        for _ in range(R):
            query(False)
    torch.cuda.synchronize()
    # per-algorithm work (iterations are stable run to run)
    stats = {}
    for a in algs:
        st = simdx_stats()
        launch(a, st)
        torch.cuda.synchronize()
        stats[a] = st
        assert st.status == 0, f"{a} status {st.status}"
    work, n_reached = {}, {}
    for a in algs:
        o = outs[a]
        if a in ("kcore", "coreness", "wcc"):
            host = None
            n_reached[a] = g.n
        elif a == "sssp":
            host = o.cpu().numpy().view(np.uint32)
            n_reached[a] = int((host != 0xFFFFFFFF).sum())
        else:
            host = o.cpu().numpy()
            n_reached[a] = int((host >= 0).sum()) if a == "bfs" else g.n
        work[a] = algorithmic(a, g, bits, host, stats[a].iterations, stats[a])
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.2)
    wall0 = time.time()
    for _ in range(args.steps):
        for _ in range(R):
            query(True)
    torch.cuda.synchronize()
    wall = time.time() - wall0
    clocks = clk.stop()
    if world > 1:
        torch.distributed.barrier()
    kern_ms = {a: [x.elapsed_time(y) for x, y in evs[a]] for a in algs}
    total_ms = max_over_ranks(float(sum(sum(v) for v in kern_ms.values())), world)
    edges_query = sum(work[a][0] for a in algs)
    value = job_rate(edges_query * R * args.steps, total_ms / 1e3, world) / 1e9
    # dominant kernel and its roofline
    mean_k = {a: statistics.mean(kern_ms[a]) for a in algs}
    dom = max(algs, key=lambda a: mean_k[a])
    peak, peak_kind = measured_peaks()
    t_dom = mean_k[dom] / 1e3
    achieved = work[dom][1] / t_dom / 1e9
    kname = f"{dom}_kernel"
    traffic = ncu_traffic(kname, args.workload)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": kname,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s", "algorithmic_bytes_per_launch": work[dom][1],
                "bytes_basis": BYTES_BASIS[dom], "mean_launch_ms": round(mean_k[dom], 4),
                "launches_timed": len(kern_ms[dom])}
    ib = inspected_bytes(dom, bits, stats[dom], n_reached[dom])
    if ib is not None:
        roofline["inspected"] = {"bytes_per_launch": ib, "achieved": round(ib / t_dom / 1e9, 1),
                                 "frac": round(ib / t_dom / 1e9 / peak, 4),
                                 "edges_inspected": stats[dom].edges_visited,
                                 "basis": INSPECTED_BASIS[dom]}
    if traffic:
        roofline["dram"] = {"bytes_per_launch": traffic, "achieved": round(traffic / t_dom / 1e9, 1),
                            "frac": round(traffic / t_dom / 1e9 / peak, 4),
                            "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch, "
                                      "profiles/ncu_traffic.json"}
    per_kernel = {a: {"mean_ms": round(mean_k[a], 4), "median_ms": round(statistics.median(kern_ms[a]), 4),
                      "min_ms": round(min(kern_ms[a]), 4), "max_ms": round(max(kern_ms[a]), 4),
                      "iterations": stats[a].iterations, "gteps": round(work[a][0] / (mean_k[a] / 1e3) / 1e9, 3),
                      "gbs": round(work[a][1] / (mean_k[a] / 1e3) / 1e9, 1),
                      "frac_of_peak": round(work[a][1] / (mean_k[a] / 1e3) / 1e9 / peak, 4),
                      "push_iters": stats[a].push_iters, "pull_iters": stats[a].pull_iters,
                      "ballot_iters": stats[a].ballot_iters, "online_iters": stats[a].online_iters,
                      "edges_inspected": stats[a].edges_visited, "grid_ctas": stats[a].grid_ctas}
                  for a in algs}
    # ---- e2e through the C ABI with host buffers (--e2e-steps 0 skips it, for profiling runs)
    e2e = run_e2e(args, g, w, bits, algs, edges_query, world, tuned_full) if args.e2e_steps > 0 else None
    res = {
        "metric": "GTEPS", "value": round(value, 3), "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic (seeded R-MAT / grid)",
        "config": {"workload": args.workload, "description": wl["desc"], "n": g.n, "directed_edges": g.e,
                   "queries_per_step": R,
                   "l2": "flushed before every query (512 MB write, outside the timed brackets)",
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "knobs": ({"autotuned": tuned, "tune_s": round(tune_s, 2)} if args.autotune else "defaults")},
        "roofline": roofline, "kernels": per_kernel, "e2e": e2e,
        "gpu_launches": sum(calls.get(a, 1) for a in algs) * R * args.steps,
        "clocks": clocks, "wall_s_timed": round(wall, 3),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args.workload, g, w)
    G.close()
    return res


def run_e2e(args, g, w, bits, algs, edges_step, world, tuned_full=None):
    import torch
    from paper_1812_04070_gb300 import Graph

    off = g.offsets if bits == 64 else g.offsets.astype(np.int32)
    p_off = torch.from_numpy(off).pin_memory()
    p_idx = torch.from_numpy(g.indices).pin_memory()
    p_w = torch.from_numpy(w.view(np.int32)).pin_memory()
    host_out = {"bfs": torch.empty(g.n, dtype=torch.int32).pin_memory(),
                "sssp": torch.empty(g.n, dtype=torch.int32).pin_memory(),
                "kcore": (torch.empty(g.n, dtype=torch.uint8).pin_memory(),
                          torch.empty(g.n, dtype=torch.int32).pin_memory()),
                "pagerank": torch.empty(g.n, dtype=torch.float32).pin_memory(),
                "coreness": torch.empty(g.n, dtype=torch.int32).pin_memory(),
                "wcc": torch.empty(g.n, dtype=torch.int32).pin_memory()}
    h2d = p_off.numel() * p_off.element_size() + p_idx.numel() * 4 + (p_w.numel() * 4 if "sssp" in algs else 0)
    d2h = 0
    for a in algs:
        d2h += g.n * (4 if a in ("bfs", "sssp", "pagerank", "coreness", "wcc") else 5)

    split = {"create": 0.0, "run": 0.0}

    def one():
        t0 = time.perf_counter()
        G = Graph(p_off.numpy(), p_idx.numpy(), weights=p_w.numpy().view(np.uint32) if "sssp" in algs else None)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        split["create"] += t1 - t0
        for a in algs:
            if tuned_full:
                G.set_config(**tuned_full[a])
            if a == "bfs":
                host_out[a].copy_(G.bfs(0), non_blocking=True)
            elif a == "sssp":
                host_out[a].copy_(G.sssp(0), non_blocking=True)
            elif a == "kcore":
                ic, rs = G.kcore(16)
                host_out[a][0].copy_(ic, non_blocking=True)
                host_out[a][1].copy_(rs, non_blocking=True)
            elif a == "coreness":
                host_out[a].copy_(G.coreness(), non_blocking=True)
            elif a == "wcc":
                host_out[a].copy_(G.wcc(), non_blocking=True)
            else:
                host_out[a].copy_(G.pagerank(0.85, 1e-6, 1000), non_blocking=True)
        torch.cuda.synchronize()
        split["run"] += time.perf_counter() - t1
        G.close()

    one()
    split["create"] = split["run"] = 0.0
    ts = []
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        one()
        ts.append(time.perf_counter() - t0)
    tot = max_over_ranks(sum(ts), world)
    return {"value": round(job_rate(edges_step * len(ts), tot, world) / 1e9, 3), "unit": "GTEPS",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": round(tot / len(ts) * 1e3, 3),
            "ms_create_per_step": round(split["create"] / len(ts) * 1e3, 3),
            "ms_algorithms_and_d2h_per_step": round(split["run"] / len(ts) * 1e3, 3),
            "note": "host pinned CSR -> simdx_graph_create -> algorithms -> results to host, per step"}


# ------------------------------------------------------------ batch / serve
def _ev_time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def run_batch(args, rank, world, local):
    """Queries per second of the batched entry points vs one call per query
    (configuration of the batching workload; identical outputs are checked)."""
    import torch
    import graphgen as gg
    from paper_1812_04070_gb300 import Graph, build, simdx_stats
    torch.cuda.set_device(local)
    build()
    wl = WORKLOADS[args.workload]
    g = gg.rmat(wl["scale"])
    w = gg.weights(g, gg.weight_seed(wl["scale"]), 1, 64)
    G = Graph(g.offsets.astype(np.int32), g.indices, weights=w)
    srcs = [int(x) for x in gg.pick_sources(g, 64, 0xBA7C4)]
    ob = torch.empty((64, g.n), dtype=torch.int32, device="cuda")
    o1 = torch.empty((64, g.n), dtype=torch.int32, device="cuda")
    reps = max(1, min(args.steps, 5))
    res = {}
    tuned = {}
    if args.autotune:
        from paper_1812_04070_gb300 import simdx
        default = {k: getattr(G.config, k) for k, _ in G.config._fields_ if k != "reserved"}
        for name, algo in [("bfs", simdx.ALGO_BFS), ("sssp", simdx.ALGO_SSSP)]:
            Gt = Graph(g.offsets.astype(np.int32), g.indices, weights=w)
            best, ms = Gt.autotune_batch(algo, srcs, reps=2)
            Gt.close()
            tuned[name] = {k: v for k, v in best.items() if v != default[k]}
            tuned[name + "_full"] = best
    for name, bat, one in [("bfs", lambda: G.bfs_batch(srcs, out=ob), lambda: [G.bfs(s, out=o1[i]) for i, s in enumerate(srcs)]),
                           ("sssp", lambda: G.sssp_batch(srcs, out=ob), lambda: [G.sssp(s, out=o1[i]) for i, s in enumerate(srcs)])]:
        ts = _ev_time(one, reps)  # one call per query, default knobs
        if name + "_full" in tuned:
            G.set_config(**tuned[name + "_full"])
        st = simdx_stats()
        G.bfs_batch(srcs, out=ob, stats=st) if name == "bfs" else G.sssp_batch(srcs, out=ob, stats=st)
        torch.cuda.synchronize()
        tb = _ev_time(bat, reps)
        same = bool(torch.equal(ob, o1))
        res[name] = {"batched_qps": round(64 / tb * 1e3, 1), "per_query_qps": round(64 / ts * 1e3, 1),
                     "batched_ms": round(tb, 3), "per_query_ms": round(ts, 3), "identical": same,
                     "launches": st.launches, "iterations": st.iterations}
        if name + "_full" in tuned:
            res[name]["knobs"] = tuned[name]
            G.set_config(**{k: v for k, v in default.items()})
    # the shared-edge batch at every group width
    for width in (8, 16, 32, 64):
        G.set_config(sssp_batch_width=width)
        G.sssp_batch(srcs, out=ob)
        torch.cuda.synchronize()
        tw = _ev_time(lambda: G.sssp_batch(srcs, out=ob), reps)
        res[f"sssp_width{width}"] = {"batched_qps": round(64 / tw * 1e3, 1), "batched_ms": round(tw, 3),
                                     "identical": bool(torch.equal(ob, o1))}
    G.set_config(sssp_batch_width=0)
    # the earlier batched SSSP layout for comparison: virtual graph copies in
    # cache-sized groups, one launch per group (batch_group knob)
    G.set_config(batch_group=8)
    st = simdx_stats()
    G.sssp_batch(srcs, out=ob, stats=st)
    torch.cuda.synchronize()
    tg = _ev_time(lambda: G.sssp_batch(srcs, out=ob), reps)
    res["sssp_virtual_copies"] = {"batched_qps": round(64 / tg * 1e3, 1), "batched_ms": round(tg, 3),
                                  "launches": st.launches, "identical": bool(torch.equal(ob, o1))}
    G.set_config(batch_group=0)
    # k-core for 64 values of k (1..64): one decomposition and one row launch
    # against 64 fixed-k runs
    ks = list(range(1, 65))
    kin = torch.empty((64, g.n), dtype=torch.uint8, device="cuda")
    krs = torch.empty((64, g.n), dtype=torch.int32, device="cuda")

    def kone():
        for i, k in enumerate(ks):
            G.kcore(k, out=kin[i], resid=krs[i])

    tk1 = _ev_time(kone, reps)
    kb_in, kb_rs = G.kcore_batch(ks)
    torch.cuda.synchronize()
    tkb = _ev_time(lambda: G.kcore_batch(ks), reps)
    res["kcore_k1_64"] = {"batched_qps": round(64 / tkb * 1e3, 1), "per_query_qps": round(64 / tk1 * 1e3, 1),
                          "batched_ms": round(tkb, 3), "per_query_ms": round(tk1, 3),
                          "identical": bool(torch.equal(kb_in, kin) and torch.equal(kb_rs, krs)),
                          "note": "simdx_kcore_batch (one decomposition, then the rows) against simdx_kcore per k"}
    G.close()
    graphs, gsrc = gg.multigraph_batch(count=256)
    packed, bases = gg.pack(graphs)
    roots = [int(x) for x in (gsrc.astype(np.int64) + bases[:-1])]
    P = Graph(packed.offsets.astype(np.int32), packed.indices)
    op = torch.empty(packed.n, dtype=torch.int32, device="cuda")
    Gs = [Graph(x.offsets.astype(np.int32), x.indices) for x in graphs]
    outs = [torch.empty(x.n, dtype=torch.int32, device="cuda") for x in graphs]
    tb = _ev_time(lambda: P.bfs_multi(roots, out=op), reps)
    ts = _ev_time(lambda: [Gi.bfs(int(s), out=o) for Gi, s, o in zip(Gs, gsrc, outs)], reps)
    same = all(torch.equal(op[int(bases[i]):int(bases[i + 1])], outs[i]) for i in range(len(graphs)))
    res["multigraph_bfs"] = {"batched_qps": round(256 / tb * 1e3, 1), "per_query_qps": round(256 / ts * 1e3, 1),
                             "batched_ms": round(tb, 3), "per_query_ms": round(ts, 3), "identical": same,
                             "note": "caller-packed CSR (simdx_bfs_multi)"}
    # the same 256 graphs as separate objects (simdx_bfs_multigraph: the
    # library packs them on the device, once per list, and scatters levels)
    from paper_1812_04070_gb300 import bfs_multigraph
    outs_m = [torch.empty(x.n, dtype=torch.int32, device="cuda") for x in graphs]
    t0 = time.perf_counter()
    bfs_multigraph(Gs, gsrc, outs=outs_m)
    torch.cuda.synchronize()
    first_ms = (time.perf_counter() - t0) * 1e3
    tm = _ev_time(lambda: bfs_multigraph(Gs, gsrc, outs=outs_m), reps)
    same = all(torch.equal(outs_m[i], outs[i]) for i in range(len(graphs)))
    res["multigraph_handles_bfs"] = {"batched_qps": round(256 / tm * 1e3, 1), "per_query_qps": round(256 / ts * 1e3, 1),
                                     "batched_ms": round(tm, 3), "per_query_ms": round(ts, 3), "identical": same,
                                     "first_call_ms": round(first_ms, 3),
                                     "note": "separate graph objects (simdx_bfs_multigraph); the first call "
                                             "builds the pack"}
    for Gi in Gs:
        Gi.close()
    P.close()
    tot_b = 64 / res["bfs"]["batched_qps"] + 64 / res["sssp"]["batched_qps"] + 256 / res["multigraph_bfs"]["batched_qps"]
    value = job_rate(64 + 64 + 256, tot_b, world)
    return {"metric": "queries/s (batched)", "value": round(value, 1), "unit": "queries/s", "n_gpus": world,
            "steps": reps, "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic (seeded R-MAT)", "config": {"workload": args.workload,
                                                                          "description": wl["desc"]},
            "batches": res}


def run_serve(args, rank, world, local):
    """Open-loop Poisson serving: queries/s and p50/p99 latency (arrival to
    result ready) per offered rate, vs one call per query."""
    import torch
    import graphgen as gg
    from paper_1812_04070_gb300 import Graph, Server, build
    torch.cuda.set_device(local)
    build()
    wl = WORKLOADS[args.workload]
    scales = [14, 15, 16, 17, 18, 19, 20, 22]
    raw = [gg.rmat(sc) for sc in scales]
    ws = [gg.weights(g, gg.weight_seed(sc), 1, 64) for g, sc in zip(raw, scales)]
    Gs = [Graph(g.offsets.astype(np.int32), g.indices, weights=w) for g, w in zip(raw, ws)]
    srcs = [gg.pick_sources(g, 256, 0x5E77E + i) for i, g in enumerate(raw)]
    rng = np.random.default_rng(0x5E77E)

    def make(m):
        q = []
        for _ in range(m):
            gi = int(rng.integers(0, len(raw)))
            r = rng.random()
            algo = Server.BFS if r < 0.5 else Server.SSSP if r < 0.9 else Server.KCORE
            arg = 16 if algo == Server.KCORE else int(srcs[gi][int(rng.integers(0, len(srcs[gi])))])
            q.append((gi, algo, arg))
        return q

    qs = make(400)
    o32 = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in raw]
    o8 = [torch.empty(g.n, dtype=torch.uint8, device="cuda") for g in raw]
    # capacity model: GPU time per query of each (graph, algorithm) when the
    # server forms full batches (64 BFS, max_sssp SSSP per launch; one k-core
    # run answers every waiting k-core query, counted here as one run per
    # query), on the whole GPU; the mix weights them (graph uniform, 50/40/10)
    max_sssp = 8
    ob = torch.empty((64, max(g.n for g in raw)), dtype=torch.int32, device="cuda")
    cost = {}
    for gi, g in enumerate(raw):
        s64 = [int(x) for x in srcs[gi][:64]]
        # the cheaper of a full batch (per query) and a single call
        tb = min(_ev_time(lambda: Gs[gi].bfs_batch(s64, out=ob), 3) / 64,
                 _ev_time(lambda: Gs[gi].bfs(s64[0], out=o32[gi]), 3))
        ts = min(_ev_time(lambda: Gs[gi].sssp_batch(s64[:max_sssp], out=ob), 3) / max_sssp,
                 _ev_time(lambda: Gs[gi].sssp(s64[0], out=o32[gi]), 3))
        tk = _ev_time(lambda: Gs[gi].kcore(16, out=o8[gi], want_resid=False), 3)
        cost[scales[gi]] = {"bfs_ms": round(tb, 4), "sssp_ms": round(ts, 4), "kcore_ms": round(tk, 4)}
    per_q_ms = sum(0.5 * c["bfs_ms"] + 0.4 * c["sssp_ms"] + 0.1 * c["kcore_ms"] for c in cost.values()) / len(raw)
    ceiling = 1e3 / per_q_ms
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for gi, a, arg in qs:
        if a == Server.BFS:
            Gs[gi].bfs(arg, out=o32[gi])
        elif a == Server.SSSP:
            Gs[gi].sssp(arg, out=o32[gi])
        else:
            Gs[gi].kcore(arg, out=o8[gi])
    torch.cuda.synchronize()
    per_query = len(qs) / (time.perf_counter() - t0)
    srv = Server(Gs, mem_budget=64 << 30, max_slots=4, max_sssp=max_sssp)
    rates = []
    for rate in [1000, 2000, 5000, 10000, 20000, 50000]:
        m = min(4000, rate * 2)
        q = make(m)
        bufs = [torch.empty(raw[gi].n, dtype=(torch.uint8 if a == Server.KCORE else torch.int32), device="cuda")
                for gi, a, _ in q]
        gaps = rng.exponential(1.0 / rate, size=m)
        t_sub, t_done, tk = np.zeros(m), np.zeros(m), [None] * m
        pending, i = [], 0  # in submission order
        start = time.perf_counter()
        nxt = start
        while i < m or pending:
            now = time.perf_counter()
            while i < m and now >= nxt:
                gi, a, arg = q[i]
                tk[i] = srv.submit(gi, a, arg, bufs[i])
                t_sub[i] = nxt
                pending.append(i)
                nxt += gaps[i]
                i += 1
            # poll the oldest 64 queries only: the client's loop stays O(1) per
            # query at high rates (a query answered out of order is seen once
            # it is among the oldest, which adds at most the wait for those)
            keep = []
            for idx, j in enumerate(pending):
                if idx < 64 and srv.poll(tk[j]):
                    t_done[j] = time.perf_counter()
                else:
                    keep.append(j)
            pending = keep
        tot = time.perf_counter() - start
        lat = (t_done - t_sub) * 1e3
        rates.append({"offered_qps": rate, "served_qps": round(job_rate(m, tot, world), 1),
                      "p50_ms": round(float(np.percentile(lat, 50)), 3),
                      "p99_ms": round(float(np.percentile(lat, 99)), 3)})
    info = srv.info()
    srv.close()
    for G in Gs:
        G.close()
    best = max(r["served_qps"] for r in rates)
    return {"metric": "queries/s (served)", "value": best, "unit": "queries/s", "n_gpus": world, "steps": len(rates),
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded R-MAT)", "config": {"workload": args.workload, "description": wl["desc"]},
            "per_query_qps": round(per_query, 1), "rates": rates, "server": info,
            "capacity_model": {"gpu_ms_per_query_full_batches": round(per_q_ms, 4),
                               "ceiling_qps": round(ceiling, 1), "served_over_ceiling": round(best / ceiling, 3),
                               "cost_by_scale": cost}}


def run_ablation(args, rank, world, local):
    """Kernel fusion (Sec. 5, Table 2) and task management (Sec. 4) ablations
    on one graph: every algorithm under all fusion (one persistent launch),
    selective push-pull fusion (one launch per run of one direction) and no
    fusion (one launch per iteration), and under the JIT filter (online,
    ballot on overflow) against the ballot filter alone.  Times are CUDA
    events around each call (median of the repetitions, L2 flushed before
    each); every mode's output is checked equal to the all-fusion JIT run."""
    import torch
    from paper_1812_04070_gb300 import Graph, build, simdx_stats
    torch.cuda.set_device(local)
    build()
    wl = WORKLOADS[args.workload]
    g, w = make_graph(wl)
    bits = wl["bits"]
    off = g.offsets if bits == 64 else g.offsets.astype(np.int32)
    G = Graph(off, g.indices, weights=w)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = torch.empty(g.n, dtype=torch.int32, device=dev)
    out8 = torch.empty(g.n, dtype=torch.uint8, device=dev)
    reps = max(3, min(args.steps, 7))
    default_delta = G.config.delta
    fl = lambda f, x: (f"fusion={['all', 'selective', 'none'][f]} filter={'JIT' if x == 0 else 'ballot'}",
                       dict(fusion=f, filter=x))
    modes = {"bfs": [fl(0, 0), fl(1, 0), fl(2, 0), fl(0, 2), fl(2, 2),
                     ("edges staged by bulk copy", dict(fusion=0, filter=0, stage_edges=1)),
                     ("small frontiers on one cluster", dict(stage_edges=0, small_frontier=1))],
             "sssp": [fl(0, 0), fl(2, 0), fl(0, 2), fl(2, 2),
                      ("combine=plain stores + pull sweeps (no atomics)", dict(fusion=0, filter=0, sssp_combine=1)),
                      ("edges staged by bulk copy", dict(sssp_combine=0, stage_edges=1)),
                      ("delta=64", dict(stage_edges=0, delta=64)), ("delta=256", dict(delta=256)),
                      ("delta=unbounded", dict(delta=0)), ("pull every iteration", dict(delta=default_delta,
                                                                                         direction=2)),
                      ("small frontiers on one cluster", dict(direction=0, small_frontier=1)),
                      ("delta=64, small frontiers on one cluster", dict(delta=64)),
                      ("delta=64, grid only", dict(small_frontier=0))],
             "kcore": [fl(0, 0), fl(0, 2)],
             "pagerank": [("pull, then push (default switch rule)", dict(pr_alpha=8.0)),
                          ("pull only", dict(pr_alpha=0.0))] +
                         [(f"pull only, row cost {rc}", dict(pr_alpha=0.0, pr_row_cost=rc)) for rc in (1, 2, 8, 16, 32)] +
                         [(f"pull only, ranges re-cut by measured time after {r}", dict(pr_alpha=0.0, pr_row_cost=0,
                                                                                          pr_recut=r))
                          for r in (1, 2)] +
                         [("pull then push, re-cut after 2", dict(pr_alpha=8.0, pr_recut=2))]}

    outf = torch.empty(g.n, dtype=torch.float32, device=dev)

    def call(a, st=None):
        if a == "bfs":
            G.bfs(0, out=out, stats=st)
        elif a == "sssp":
            G.sssp(0, out=out, stats=st)
        elif a == "pagerank":
            G.pagerank(0.85, 1e-6, 1000, out=outf, stats=st)
        else:
            G.kcore(16, out=out8, want_resid=False, stats=st)

    res = {}
    for a in wl["algs"]:
        ref = None
        rows = []
        G.set_config(delta=default_delta, direction=0, stage_edges=0, small_frontier=0)
        for label, knobs in modes[a]:
            G.set_config(**knobs)
            st = simdx_stats()
            call(a, st)
            torch.cuda.synchronize()
            o = (out8 if a == "kcore" else outf if a == "pagerank" else out).clone()
            if ref is None:
                ref = o
            ts = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call(a)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            row = {"mode": label, "ms": round(ms, 3), "iterations": st.iterations, "launches": st.launches,
                   "us_per_iteration": round(ms * 1e3 / max(1, st.iterations), 2),
                   "pull_iters": st.pull_iters, "push_iters": st.push_iters, "ballot_iters": st.ballot_iters,
                   "edges_inspected": st.edges_visited}
            if a == "pagerank":
                # the two modes reach the fixed point by different paths: both are
                # within d / (1 - d) * tol of it, so they are compared in L1
                row["l1_vs_first_mode"] = float((o.double() - ref.double()).abs().sum())
            else:
                row["identical"] = bool(torch.equal(o, ref))
            rows.append(row)
        res[a] = rows
        G.set_config(fusion=0, filter=0, pr_alpha=8.0, sssp_combine=0, delta=default_delta, direction=0,
                     pr_row_cost=0, stage_edges=0, pr_recut=0, small_frontier=2)
    G.close()
    base = res[wl["algs"][0]][0]
    return {"metric": f"us per iteration ({wl['algs'][0]}, all fusion)", "value": base["us_per_iteration"],
            "unit": "us", "n_gpus": world, "steps": reps, "warmup": 1, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded R-MAT / grid)",
            "config": {"workload": args.workload, "description": wl["desc"], "n": g.n, "directed_edges": g.e,
                       "l2": "flushed before every timed call"},
            "ablation": res}


# ------------------------------------------------------------ CPU oracle legs
def cpu_leg(workload, g, w, budget_s, parallel):
    """The oracle on a bounded sample of the workload, repeated until about
    budget_s seconds have passed (at least once): GTEPS with the GPU's edge
    counting.  parallel=True takes the OpenMP variants where the oracle has
    them (BFS, k-core, PageRank) and the single-threaded definition
    elsewhere (SSSP stays Dijkstra; coreness and components)."""
    import oracle
    wl = WORKLOADS[workload]
    t_tot, edges, reps = 0.0, 0, 0
    parts = []
    while True:
        for a in wl["algs"]:
            t0 = time.perf_counter()
            par = parallel and a in ("bfs", "kcore", "pagerank")
            if a == "bfs":
                lev = (oracle.bfs_par if par else oracle.bfs)(g.offsets, g.indices, 0)
                m = int(g.degrees()[lev >= 0].sum()) // 2
                part = "bfs full"
            elif a == "sssp":
                d = oracle.sssp(g.offsets, g.indices, w, 0)
                m = int(g.degrees()[d != 0xFFFFFFFF].sum()) // 2
                part = "sssp full"
            elif a == "kcore":
                (oracle.kcore_par if par else oracle.kcore)(g.offsets, g.indices, 16)
                m = g.e // 2
                part = "kcore full"
            elif a == "coreness":
                oracle.coreness(g.offsets, g.indices)
                m = g.e // 2
                part = "coreness full"
            elif a == "wcc":
                oracle.wcc(g.offsets, g.indices)
                m = g.e // 2
                part = "wcc full"
            else:
                iters = 5
                (oracle.pagerank_par if par else oracle.pagerank)(g.offsets, g.indices, fixed_iter=iters)
                m = (g.e // 2) * iters
                part = f"pagerank {iters} iterations"
            t_tot += time.perf_counter() - t0
            edges += m
            if reps == 0:
                parts.append(part + (" (OpenMP)" if par else " (1 thread)"))
        reps += 1
        if t_tot >= budget_s or reps >= 50:
            break
    threads = oracle.threads() if parallel else 1
    return {"value": round(edges / t_tot / 1e9, 4), "unit": "GTEPS", "cores": threads, "kind": "oracle",
            "sample": f"{workload}: {reps} x (" + ", ".join(parts) + f") ({t_tot:.1f} s)"}


def cpu_baseline(workload, g, w, budget_s=12.0):
    """The oracle as it stands, timed on the host cores: the OpenMP variants
    on every core the process may use (the line's value) and the
    single-threaded definitions beside them."""
    par = cpu_leg(workload, g, w, budget_s, parallel=True)
    ser = cpu_leg(workload, g, w, budget_s * 0.6, parallel=False)
    par["affinity_cores"] = len(os.sched_getaffinity(0))
    par["serial"] = {"value": ser["value"], "cores": 1, "sample": ser["sample"]}
    return par


def run_reference(args, rank, world):
    if rank != 0:
        return None
    wl = WORKLOADS[args.workload]
    g, w = make_graph(wl)
    cb = cpu_leg(args.workload, g, w, 5.0, parallel=True)  # warm-up of the sample
    vals = []
    for _ in range(max(1, args.steps if args.steps <= 3 else 3)):
        vals.append(cpu_leg(args.workload, g, w, 10.0, parallel=True)["value"])
    v = statistics.median(vals)
    return {"impl": "reference", "metric": "GTEPS", "value": v, "unit": "GTEPS", "n_gpus": world,
            "steps": len(vals), "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32+f64", "data": "synthetic (seeded R-MAT / grid)",
            "config": {"workload": args.workload, "description": wl["desc"]},
            "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"], "affinity_cores": len(os.sched_getaffinity(0))},
            "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    elif WORKLOADS[args.workload]["kind"] == "batch":
        res = run_batch(args, rank, world, local)
    elif WORKLOADS[args.workload]["kind"] == "ablation":
        res = run_ablation(args, rank, world, local)
    elif WORKLOADS[args.workload]["kind"] == "serve":
        res = run_serve(args, rank, world, local)
    else:
        res = run_simdx(args, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
