"""CPU-only checks of the C-ABI library: it builds, loads, exports every symbol
include/gbx.h declares, and its host-side logic (descriptor defaults, status
names, argument validation that fails before any device work) behaves as
documented.  No compute call runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
from paper_1804_03327_gb300 import build as gbx_build
from paper_1804_03327_gb300 import gbx, roofline

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gbx_build.build()
    return gbx.load()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gbx_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(gbx.EXPORTED) == set(names)


def test_library_links_no_torch(lib):
    # the boundary is plain C: no torch symbol is referenced by the library
    data = open(gbx_build.LIB_PATH, "rb").read()
    assert b"libtorch" not in data and b"c10::" not in data


def test_desc_defaults_follow_section_6_3(lib):
    d = gbx.desc_init()
    assert d.transpose == 1 and d.early_exit == 1 and d.masking == 1 and d.operand_reuse == 1
    assert d.mask_complement == 0 and d.accum == 0 and d.trace == 0
    assert d.direction == gbx.DIR_AUTO and d.heuristic == gbx.HEUR_RATIO
    assert abs(d.alpha - 0.01) < 1e-7 and abs(d.beta - 0.01) < 1e-7
    assert d.pull_probe == 0 and d.blocks_per_sm == 0 and d.push_sort == 0 and list(d.reserved) == [0] * 2


def test_status_names_and_version(lib):
    assert gbx.status_string(gbx.OK) == "GBX_OK"
    assert gbx.status_string(gbx.ERR_TIMEOUT) == "GBX_ERR_TIMEOUT"
    assert gbx.status_string(999) == "GBX_ERR_UNKNOWN"
    assert gbx.version() == 100


def test_validation_before_device_work(lib):
    h = ctypes.c_void_p()
    src = np.zeros(1, np.int32)
    assert lib.gbx_graph_build(None, 4, 1, src.ctypes.data, src.ctypes.data, 0, None) == gbx.ERR_NULL_POINTER
    assert lib.gbx_graph_build(ctypes.byref(h), 0, 1, src.ctypes.data, src.ctypes.data, 0, None) == \
        gbx.ERR_INVALID_VALUE
    assert "n must be" in lib.gbx_last_error().decode()
    assert lib.gbx_graph_build(ctypes.byref(h), 4, -1, src.ctypes.data, src.ctypes.data, 0, None) == \
        gbx.ERR_INVALID_VALUE
    assert lib.gbx_graph_build(ctypes.byref(h), 4, 1, None, None, 0, None) == gbx.ERR_NULL_POINTER
    assert lib.gbx_graph_build(ctypes.byref(h), 4, 1, src.ctypes.data, src.ctypes.data, 0x80, None) == \
        gbx.ERR_INVALID_VALUE
    assert lib.gbx_bfs(None, 0, None, None, None, None) == gbx.ERR_NULL_POINTER
    assert lib.gbx_graph_free(None) == gbx.OK
    w = gbx.Vector(gbx.DENSE, 4, None, None, 0)
    assert lib.gbx_mxv(ctypes.byref(w), None, gbx.LOR_LAND, None, ctypes.byref(w), None, None) == \
        gbx.ERR_NULL_POINTER
    assert lib.gbx_set_wait_timeout_ns(5_000_000_000) == gbx.OK


def test_python_binding_raises_with_message(lib):
    with pytest.raises(gbx.GbxError) as e:
        gbx.graph_build(0, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert e.value.status == gbx.ERR_INVALID_VALUE


def test_byte_model_on_oracle_trace():
    """The roofline byte model evaluated on the oracle's own level trace (same
    fields the device records) for the star closed form."""
    k = 9
    g = oracle.graph(*synth.star_edges(k))
    depth, _, levels = oracle.bfs(g, 1)
    tr = oracle.bfs_trace(g, depth, levels)
    dirs = oracle.direction_schedule(tr, g.n, mode="push")
    rec = np.zeros(len(tr), dtype=[(f, np.int64) for f in gbx.LEVEL_FIELDS])
    for f in tr.dtype.names:
        rec[f] = tr[f]
    rec["direction"] = [roofline.PUSH if d == "push" else roofline.PULL for d in dirs]
    n = g.n
    bm = (n + 7) // 8
    want = 8 * n + sum(12 * r["nf"] + 4 * r["mf"] + 12 * r["n_new"] + bm for r in tr)
    assert roofline.bfs_bytes(rec, n) == want
    assert roofline.reached_edges(rec) == k  # star: k undirected edges, all reached


def test_server_config_validation_on_host(lib):
    c = gbx.ServerConfig()
    lib.gbx_server_config_init(ctypes.byref(c))
    assert (c.max_batch, c.slots, c.depth_type, c.max_pending, c.memory_budget) == (64, 2, 0, 1 << 16, 0)
    h = ctypes.c_void_p()
    for field, bad in [("max_batch", 0), ("slots", 17), ("depth_type", 5), ("max_pending", 0), ("memory_budget", -1)]:
        c2 = gbx.ServerConfig()
        lib.gbx_server_config_init(ctypes.byref(c2))
        setattr(c2, field, bad)
        assert lib.gbx_server_create(ctypes.byref(h), ctypes.byref(c2)) == gbx.ERR_INVALID_VALUE, field
    assert lib.gbx_server_submit(None, 0, 0, None, 0) == gbx.ERR_NULL_POINTER
    assert lib.gbx_server_destroy(None) == gbx.OK
