"""GPU parity of gbx_mxv (the four matvec variants of Table 1, Eq 2-5) against
the CPU oracle's definition, bit-exact, for every flag and vector format."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth
from paper_1804_03327_gb300 import gbx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

_cache = {}


def graph(name):
    if name not in _cache:
        if name == "rmat11":
            n, s, d = synth.rmat_edges(11, 16, seed=5)
            sym = True
        elif name == "rmat11-directed":
            n, s, d = synth.rmat_edges(11, 8, seed=6)
            sym = False
        elif name == "grid":
            n, s, d = synth.grid_edges(50, 41, p_delete=0.01, seed=2)  # ragged: n not a multiple of 32
            sym = True
        _cache[name] = (n, oracle.graph(n, s, d, symmetrize=sym), gbx.graph_build(n, s, d, symmetrize=sym))
    return _cache[name]


def to_vec(x: np.ndarray, fmt: int, n: int):
    """Device vector from a 0/1 byte array; returns (gbx.Vector, keepalive)."""
    if fmt == gbx.DENSE:
        t = torch.from_numpy(x.astype(np.uint8)).cuda()
        return gbx.dense(t), (t,)
    idx = np.flatnonzero(x).astype(np.int32)
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    t[: len(idx)] = torch.from_numpy(idx).cuda()
    c = torch.tensor([len(idx)], dtype=torch.int32, device="cuda")
    return gbx.sparse(t, c, n), (t, c)


def out_vec(fmt: int, n: int, w_old: np.ndarray):
    return to_vec(w_old, fmt, n)


def read_vec(v, keep, fmt: int, n: int) -> np.ndarray:
    torch.cuda.synchronize()
    if fmt == gbx.DENSE:
        return keep[0].cpu().numpy()
    cnt = int(keep[1].item())
    idx = keep[0][:cnt].cpu().numpy()
    assert np.all(np.diff(idx) > 0), "sparse output must be sorted and unique"
    out = np.zeros(n, np.uint8)
    out[idx] = 1
    return out


CASES = list(itertools.product(
    [gbx.DIR_PUSH, gbx.DIR_PULL, gbx.DIR_AUTO],  # direction
    [0, 1],                                      # transpose
    ["none", "dense", "sparse"],                 # mask
    [0, 1],                                      # complement
    [0, 1],                                      # accum
))


@pytest.mark.parametrize("direction,transpose,mask_kind,complement,accum", CASES)
def test_mxv_all_flags(direction, transpose, mask_kind, complement, accum):
    for name in ["rmat11", "rmat11-directed"]:
        n, og, g = graph(name)
        for k, (ud, md) in enumerate([(0.001, 0.5), (0.02, 0.9), (0.3, 0.1)]):
            u = synth.vertex_set(n, ud, seed=10 + k)
            m = synth.vertex_set(n, md, seed=20 + k)
            w_old = synth.vertex_set(n, 0.2, seed=30 + k)
            want = oracle.mxv(n, n, og.out_ptr, og.out_col, u, None if mask_kind == "none" else m,
                              transpose=bool(transpose), complement=bool(complement), accum=bool(accum),
                              w_old=w_old)
            for ufmt, wfmt in [(gbx.DENSE, gbx.DENSE), (gbx.SPARSE, gbx.SPARSE), (gbx.SPARSE, gbx.DENSE)]:
                uv, ukeep = to_vec(u, ufmt, n)
                wv, wkeep = out_vec(wfmt, n, w_old)
                mv = None
                if mask_kind != "none":
                    mv, mkeep = to_vec(m, gbx.DENSE if mask_kind == "dense" else gbx.SPARSE, n)
                for ee in (0, 1):
                    wv, wkeep = out_vec(wfmt, n, w_old)
                    desc = gbx.desc_init(direction=direction, transpose=transpose, mask_complement=complement,
                                         accum=accum, early_exit=ee)
                    gbx.mxv(wv, mv, gbx.LOR_LAND, g, uv, desc)
                    got = read_vec(wv, wkeep, wfmt, n)
                    assert np.array_equal(got, want), (name, k, ufmt, wfmt, ee)


def test_mxv_ragged_grid_and_extremes():
    n, og, g = graph("grid")
    assert n % 32 != 0
    for ud in [0.0, 1e-3, 0.5, 1.0]:
        u = synth.vertex_set(n, ud, seed=3) if 0 < ud < 1 else np.full(n, int(ud), np.uint8)
        for md in [0.0, 0.5, 1.0]:
            m = synth.vertex_set(n, md, seed=4) if 0 < md < 1 else np.full(n, int(md), np.uint8)
            want = oracle.mxv(n, n, og.out_ptr, og.out_col, u, m, transpose=True, complement=True)
            for direction in (gbx.DIR_PUSH, gbx.DIR_PULL, gbx.DIR_AUTO):
                uv, uk = to_vec(u, gbx.SPARSE, n)
                mv, mk = to_vec(m, gbx.DENSE, n)
                wv, wk = to_vec(np.zeros(n, np.uint8), gbx.SPARSE, n)
                gbx.mxv(wv, mv, gbx.LOR_LAND, g, uv, gbx.desc_init(direction=direction, mask_complement=1))
                assert np.array_equal(read_vec(wv, wk, gbx.SPARSE, n), want)


def test_mxv_figure3_example():
    ex = json.load(open(os.path.join(GOLDEN, "fig3_example.json")))
    names = ex["stated_by_the_paper"]["vertices"]
    idx = {c: i for i, c in enumerate(names)}
    edges = ex["chosen_by_this_test"]["edges"]
    src = np.array([idx[a] for a, _ in edges], np.int32)
    dst = np.array([idx[b] for _, b in edges], np.int32)
    g = gbx.graph_build(8, src, dst)
    f = oracle.to_dense([idx[c] for c in ex["stated_by_the_paper"]["frontier"]], 8)
    v = oracle.to_dense([idx[c] for c in ex["stated_by_the_paper"]["visited"]], 8)
    for direction in (gbx.DIR_PUSH, gbx.DIR_PULL):
        uv, uk = to_vec(f, gbx.SPARSE, 8)
        mv, mk = to_vec(v, gbx.DENSE, 8)
        wv, wk = to_vec(np.zeros(8, np.uint8), gbx.SPARSE, 8)
        gbx.mxv(wv, mv, gbx.LOR_LAND, g, uv, gbx.desc_init(direction=direction, mask_complement=1))
        got = [names[i] for i in np.flatnonzero(read_vec(wv, wk, gbx.SPARSE, 8))]
        assert got == ex["stated_by_the_paper"]["push_result_after_visited_filter"]


def test_mxv_stats_count_table1_terms():
    n, og, g = graph("rmat11")
    u = synth.vertex_set(n, 0.01, seed=1)
    m = synth.vertex_set(n, 0.3, seed=2)
    uv, uk = to_vec(u, gbx.SPARSE, n)
    mv, mk = to_vec(m, gbx.DENSE, n)
    wv, wk = to_vec(np.zeros(n, np.uint8), gbx.DENSE, n)
    gbx.mxv(wv, mv, gbx.LOR_LAND, g, uv, gbx.desc_init(direction=gbx.DIR_PUSH, trace=1))
    st = gbx.mxv_stats(g)
    deg = np.diff(og.out_ptr)
    assert st["u_nnz"] == u.sum() and st["edges"] == deg[u.astype(bool)].sum()
    gbx.mxv(wv, mv, gbx.LOR_LAND, g, uv, gbx.desc_init(direction=gbx.DIR_PULL, early_exit=0, trace=1))
    st = gbx.mxv_stats(g)
    rows = m.astype(bool) & (deg > 0)
    assert st["rows"] == rows.sum() and st["examined"] == deg[rows].sum()


def test_mxv_rejects_bad_arguments():
    n, og, g = graph("rmat11")
    t = torch.zeros(n, dtype=torch.uint8, device="cuda")
    small = torch.zeros(n - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(gbx.GbxError) as e:
        gbx.mxv(gbx.dense(t), None, 7, g, gbx.dense(torch.zeros_like(t)))
    assert e.value.status == gbx.ERR_NOT_SUPPORTED
    with pytest.raises(gbx.GbxError) as e:
        gbx.mxv(gbx.dense(t), None, gbx.LOR_LAND, g, gbx.dense(small))
    assert e.value.status == gbx.ERR_DIMENSION_MISMATCH
    with pytest.raises(gbx.GbxError) as e:
        gbx.mxv(gbx.dense(t), None, gbx.LOR_LAND, g, gbx.dense(t))
    assert e.value.status == gbx.ERR_INVALID_VALUE
    idx = torch.zeros(10, dtype=torch.int32, device="cuda")
    c = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(gbx.GbxError) as e:  # sparse output needs capacity >= n
        gbx.mxv(gbx.sparse(idx, c, n), None, gbx.LOR_LAND, g, gbx.dense(t))
    assert e.value.status == gbx.ERR_INVALID_VALUE


# ---- Algorithm 3: the paper's sort-based push (desc.push_sort) gives the same w

SORT_CASES = list(itertools.product(
    [gbx.DIR_PUSH, gbx.DIR_AUTO],  # direction (AUTO with alpha 1 always pushes)
    [0, 1],                        # transpose
    ["none", "dense", "sparse"],   # mask
    [0, 1],                        # complement
    [0, 1],                        # accum
))


@pytest.mark.parametrize("direction,transpose,mask_kind,complement,accum", SORT_CASES)
def test_mxv_sorted_push_all_flags(direction, transpose, mask_kind, complement, accum):
    for name in ["rmat11", "rmat11-directed"]:
        n, og, g = graph(name)
        for k, (ud, md) in enumerate([(0.001, 0.5), (0.02, 0.9), (0.3, 0.1)]):
            u = synth.vertex_set(n, ud, seed=40 + k)
            m = synth.vertex_set(n, md, seed=50 + k)
            w_old = synth.vertex_set(n, 0.2, seed=60 + k)
            want = oracle.mxv(n, n, og.out_ptr, og.out_col, u, None if mask_kind == "none" else m,
                              transpose=bool(transpose), complement=bool(complement), accum=bool(accum),
                              w_old=w_old)
            for ufmt, wfmt in [(gbx.DENSE, gbx.DENSE), (gbx.SPARSE, gbx.SPARSE), (gbx.DENSE, gbx.SPARSE)]:
                uv, ukeep = to_vec(u, ufmt, n)
                mv = None
                if mask_kind != "none":
                    mv, mkeep = to_vec(m, gbx.DENSE if mask_kind == "dense" else gbx.SPARSE, n)
                wv, wkeep = out_vec(wfmt, n, w_old)
                desc = gbx.desc_init(direction=direction, transpose=transpose, mask_complement=complement,
                                     accum=accum, push_sort=1, alpha=1.0)
                gbx.mxv(wv, mv, gbx.LOR_LAND, g, uv, desc)
                assert np.array_equal(read_vec(wv, wkeep, wfmt, n), want), (name, k, ufmt, wfmt)


def test_mxv_sorted_push_large_and_extremes():
    """Many gather tiles and radix passes (RMAT scale 16 with hubs; the 50x41 grid,
    n not a multiple of 32), empty and full frontiers, empty and full masks."""
    n16, s16, d16 = synth.rmat_edges(16, 16, seed=8)
    og16 = oracle.graph(n16, s16, d16)
    g16 = gbx.graph_build(n16, s16, d16)
    n, og, g = graph("grid")
    for (nn, ogx, gx) in [(n16, og16, g16), (n, og, g)]:
        for ud in [0.0, 1e-3, 0.5, 1.0]:
            u = synth.vertex_set(nn, ud, seed=13) if 0 < ud < 1 else np.full(nn, int(ud), np.uint8)
            for md in [0.0, 0.5, 1.0]:
                m = synth.vertex_set(nn, md, seed=14) if 0 < md < 1 else np.full(nn, int(md), np.uint8)
                want = oracle.mxv(nn, nn, ogx.out_ptr, ogx.out_col, u, m, transpose=True, complement=True)
                uv, uk = to_vec(u, gbx.SPARSE, nn)
                mv, mk = to_vec(m, gbx.DENSE, nn)
                wv, wk = to_vec(np.zeros(nn, np.uint8), gbx.SPARSE, nn)
                gbx.mxv(wv, mv, gbx.LOR_LAND, gx, uv,
                        gbx.desc_init(direction=gbx.DIR_PUSH, mask_complement=1, push_sort=1, trace=1))
                assert np.array_equal(read_vec(wv, wk, gbx.SPARSE, nn), want), (nn, ud, md)
                st = gbx.mxv_stats(gx)
                deg = np.diff(ogx.out_ptr)
                assert st["u_nnz"] == u.sum() and st["edges"] == deg[u.astype(bool)].sum()
    g16.free()


def test_push_sort_is_mxv_only():
    n, og, g = graph("rmat11")
    depth = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(gbx.GbxError) as e:
        gbx.bfs(g, 0, depth, None, gbx.desc_init(push_sort=1))
    assert e.value.status == gbx.ERR_NOT_SUPPORTED
    with pytest.raises(gbx.GbxError) as e:
        gbx.bfs_batch(g, np.array([0, 1], np.int32), torch.zeros((2, n), dtype=torch.int32, device="cuda"),
                      desc=gbx.desc_init(push_sort=1))
    assert e.value.status == gbx.ERR_NOT_SUPPORTED
    t = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(gbx.GbxError) as e:
        gbx.mxv(gbx.dense(t), None, gbx.LOR_LAND, g, gbx.dense(torch.zeros_like(t)), gbx.desc_init(push_sort=2))
    assert e.value.status == gbx.ERR_INVALID_VALUE
