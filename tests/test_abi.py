"""The C-ABI library loads and exports every symbol include/simdx.h declares;
host-only entry points work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(simdx_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_04070_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_declarations():
    from paper_1812_04070_gb300 import simdx
    names = declared_functions()
    assert set(names) <= set(simdx.SIGNATURES), set(names) - set(simdx.SIGNATURES)


def test_eq1_worked_example(lib):
    # Sec. 5, Eq. 1 worked example: 65,536 registers per SMX, 110 registers
    # per thread, 128 threads per CTA, 15 SMX -> floor(4.65) * 15 = 60 CTAs.
    from paper_1812_04070_gb300 import simdx
    assert simdx.simdx_eq1_ctas(65536, 110, 128, 15) == 60
    assert simdx.simdx_eq1_ctas(65536, 48, 128, 15) == 150
    assert simdx.simdx_eq1_ctas(0, 1, 1, 1) == -1


def test_host_only_calls(lib):
    from paper_1812_04070_gb300 import simdx
    assert simdx.simdx_strerror(simdx.EBARRIER_TIMEOUT) == "grid barrier wait timed out"
    c = simdx.simdx_config_default()
    assert (c.small_max, c.bin_per_thread) == (32, 64)  # Sec. 4: thread/warp separator 32, threshold 64
    assert 128 <= c.med_max <= 2048  # Sec. 4: the warp/CTA separator is insensitive in [128, 2048]
    assert simdx.simdx_version() >= 10000


def test_config_layout_matches_header(lib):
    """The binding's simdx_config mirrors the header field for field (the
    batch_group, fusion and PageRank switch knobs took reserved words, so the size is
    unchanged); simdx_config_default writes the whole struct."""
    import ctypes
    from paper_1812_04070_gb300 import simdx
    text = open(os.path.join(ROOT, "include", "simdx.h")).read()
    end = text.index("} simdx_config;")
    body = text[text.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:int32_t|uint32_t|float)\s+([a-z_0-9]+)(\[(\d+)\])?;", body)
    assert [f[0] for f in fields] == [f[0] for f in simdx.simdx_config._fields_]
    words = sum(int(n) if n else 1 for _, _, n in fields)
    assert ctypes.sizeof(simdx.simdx_config) == 4 * words
    c = simdx.simdx_config_default()
    assert c.batch_group == 0 and c.fusion == 0 and c.sssp_combine == 0 and c.sssp_batch_width == 0
    assert c.pr_row_cost == 0 and c.stage_edges == 0 and c.pr_recut == 0 and c.small_frontier == 2
    assert list(c.reserved) == [0] * 5
    assert (c.pr_alpha, c.pr_theta, c.pr_rho) == (8.0, 2.0, pytest.approx(0.6))


def test_stats_layout_matches_header():
    """simdx_stats keeps its size: the launch count took reserved words."""
    import ctypes
    from paper_1812_04070_gb300 import simdx
    text = open(os.path.join(ROOT, "include", "simdx.h")).read()
    end = text.index("} simdx_stats;")
    body = text[text.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(int32_t|int64_t|double)\s+([a-z_0-9]+)(\[(\d+)\])?;", body)
    assert [f[1] for f in fields] == [f[0] for f in simdx.simdx_stats._fields_]
    size = sum({"int32_t": 4, "int64_t": 8, "double": 8}[t] * (int(n) if n else 1) for t, _, _, n in fields)
    assert ctypes.sizeof(simdx.simdx_stats) == size == 88
