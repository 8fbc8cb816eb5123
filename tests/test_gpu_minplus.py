"""GPU parity of the (min, +) semiring (Section 5.6): edge weights, the masked
min-plus matvec and the direction-optimised Bellman-Ford SSSP, against the
CPU oracle.  Each matvec output is one binary32 addition followed by exact
minima, and rounding is monotonic, so the device result equals the oracle's
double-precision result rounded to binary32 -- compared exactly.  SSSP
distances equal the oracle's binary32 Bellman-Ford exactly (non-negative
weights: the rounded fixpoint does not depend on the relaxation order)."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from paper_1804_03327_gb300 import gbx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

_cache = {}


def weights(m, seed, integer):
    rng = np.random.default_rng(seed)
    if integer:
        return rng.integers(1, 65, size=m).astype(np.float32)
    return (rng.random(m) * 8.0 + 1e-3).astype(np.float32)


def wgraph(name, integer=False):
    key = (name, integer)
    if key not in _cache:
        if name == "rmat12":
            (n, s, d), sym = synth.rmat_edges(12, 16, seed=71), True
        elif name == "rmat11-directed":
            (n, s, d), sym = synth.rmat_edges(11, 8, seed=72), False
        elif name == "grid":
            (n, s, d), sym = synth.grid_edges(45, 37, p_delete=0.02, seed=73), True
        elif name == "dups":  # parallel pairs with different weights, directed
            n, s, d = synth.er_edges(400, 0.01, seed=74, directed=True)
            s, d, sym = np.concatenate([s, s[:300]]), np.concatenate([d, d[:300]]), False
        w = weights(len(s), 75, integer)
        og = oracle.graph_weighted(n, s, d, w, symmetrize=sym)
        g = gbx.graph_build(n, s, d, symmetrize=sym)
        gbx.graph_set_weights(g, s, d, w)
        _cache[key] = (n, s, d, w, og, g)
    return _cache[key]


@pytest.mark.parametrize("name", ["rmat12", "rmat11-directed", "dups"])
def test_weights_match_oracle(name):
    n, s, d, w, og, g = wgraph(name)
    assert np.array_equal(gbx.graph_weights(g), og.out_val.astype(np.float32))
    assert np.array_equal(gbx.graph_weights(g, transpose=True), og.in_val.astype(np.float32))


def test_weights_from_device_arrays_and_errors():
    n, s, d, w, og, g = wgraph("rmat11-directed")
    g2 = gbx.graph_build(n, s, d, symmetrize=False)
    gbx.graph_set_weights(g2, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(w).cuda())
    assert np.array_equal(gbx.graph_weights(g2), og.out_val.astype(np.float32))
    bad = w.copy()
    bad[3] = np.nan
    with pytest.raises(gbx.GbxError) as e:
        gbx.graph_set_weights(g2, s, d, bad)
    assert e.value.status == gbx.ERR_INVALID_VALUE
    other = synth.er_edges(n, 0.001, seed=99, directed=True)
    with pytest.raises(gbx.GbxError) as e:  # pairs the graph does not store
        gbx.graph_set_weights(g2, other[1], other[2], np.ones(len(other[1]), np.float32))
    assert e.value.status == gbx.ERR_INVALID_VALUE
    g3 = gbx.graph_build(n, s, d, symmetrize=False)
    dist = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(gbx.GbxError) as e:  # no weights
        gbx.sssp(g3, 0, dist)
    assert e.value.status == gbx.ERR_INVALID_VALUE
    g2.free()
    g3.free()


CASES = list(itertools.product([gbx.DIR_PUSH, gbx.DIR_PULL, gbx.DIR_AUTO], [0, 1], ["none", "dense", "sparse"],
                               [0, 1], [0, 1]))


def to_mask(m, kind, n):
    if kind == "dense":
        t = torch.from_numpy(m.astype(np.uint8)).cuda()
        return gbx.dense(t), (t,)
    idx = np.flatnonzero(m).astype(np.int32)
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    t[: len(idx)] = torch.from_numpy(idx).cuda()
    c = torch.tensor([len(idx)], dtype=torch.int32, device="cuda")
    return gbx.sparse(t, c, n), (t, c)


@pytest.mark.parametrize("direction,transpose,mask_kind,complement,accum", CASES)
def test_mxv_minplus_all_flags(direction, transpose, mask_kind, complement, accum):
    for name in ["rmat12", "rmat11-directed", "dups"]:
        n, s, d, w, og, g = wgraph(name)
        rng = np.random.default_rng(5)
        for k, dens in enumerate([0.002, 0.05, 0.6]):
            u = np.where(rng.random(n) < dens, (rng.random(n) * 100).astype(np.float32), np.float32(np.inf))
            w_old = np.where(rng.random(n) < 0.3, (rng.random(n) * 100).astype(np.float32), np.float32(np.inf))
            m = synth.vertex_set(n, 0.5, seed=80 + k)
            want = oracle.mxv_minplus(n, n, og.out_ptr, og.out_col, og.out_val, u.astype(np.float64),
                                      None if mask_kind == "none" else m, transpose=bool(transpose),
                                      complement=bool(complement), accum=bool(accum),
                                      w_old=w_old.astype(np.float64)).astype(np.float32)
            ut = torch.from_numpy(u).cuda()
            wt = torch.from_numpy(w_old).cuda()
            mv, mk = (None, None) if mask_kind == "none" else to_mask(m, mask_kind, n)
            desc = gbx.desc_init(direction=direction, transpose=transpose, mask_complement=complement, accum=accum,
                                 alpha=0.05)
            gbx.mxv(gbx.dense_f32(wt), mv, gbx.MIN_PLUS_F32, g, gbx.dense_f32(ut), desc)
            got = wt.cpu().numpy()
            assert np.array_equal(got, want), (name, k)


def test_mxv_minplus_rejects_bad_combinations():
    n, s, d, w, og, g = wgraph("rmat12")
    f = torch.zeros(n, dtype=torch.float32, device="cuda")
    b = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(gbx.GbxError) as e:  # Boolean vectors with the tropical semiring
        gbx.mxv(gbx.dense(b), None, gbx.MIN_PLUS_F32, g, gbx.dense(torch.zeros_like(b)))
    assert e.value.status == gbx.ERR_INVALID_VALUE
    with pytest.raises(gbx.GbxError) as e:  # float vectors with the Boolean semiring
        gbx.mxv(gbx.dense_f32(f), None, gbx.LOR_LAND, g, gbx.dense_f32(torch.zeros_like(f)))
    assert e.value.status == gbx.ERR_INVALID_VALUE
    with pytest.raises(gbx.GbxError) as e:
        gbx.mxv(gbx.dense_f32(f), None, gbx.MIN_PLUS_F32, g, gbx.dense_f32(torch.zeros_like(f)),
                gbx.desc_init(push_sort=1))
    assert e.value.status == gbx.ERR_NOT_SUPPORTED


@pytest.mark.parametrize("name", ["rmat12", "rmat11-directed", "grid", "dups"])
@pytest.mark.parametrize("integer", [True, False])
def test_sssp_matches_oracle_every_direction(name, integer):
    n, s, d, w, og, g = wgraph(name, integer)
    dist = torch.zeros(n, dtype=torch.float32, device="cuda")
    for src in synth.sources(n, s, d, 3, seed=6):
        want, _ = oracle.sssp(og, int(src))
        for desc in [gbx.desc_init(), gbx.desc_init(beta=0.0), gbx.desc_init(direction=gbx.DIR_PUSH),
                     gbx.desc_init(direction=gbx.DIR_PULL), gbx.desc_init(alpha=0.0005),
                     gbx.desc_init(blocks_per_sm=1), gbx.desc_init(blocks_per_sm=3),
                     gbx.desc_init(direction=gbx.DIR_PUSH, blocks_per_sm=3)]:
            gbx.sssp(g, int(src), dist, desc)
            gbx.graph_sync(g)
            assert np.array_equal(dist.cpu().numpy(), want), (name, src, desc.direction, desc.alpha, desc.beta,
                                                              desc.blocks_per_sm)


def test_sssp_unit_weights_equal_bfs_depth_and_trace():
    n, s, d = synth.rmat_edges(13, 16, seed=91)
    g = gbx.graph_build(n, s, d)
    gbx.graph_set_weights(g, s, d, np.ones(len(s), np.float32))
    og = oracle.graph(n, s, d)
    dist = torch.zeros(n, dtype=torch.float32, device="cuda")
    for k, src in enumerate(synth.sources(n, s, d, 3, seed=7)):
        depth, _, _ = oracle.bfs(og, int(src))
        gbx.sssp(g, int(src), dist, gbx.desc_init(trace=1, blocks_per_sm=3 if k == 1 else 0))  # k = 1: lean build
        tr = gbx.sssp_trace(g)
        want = np.where(depth >= 0, depth.astype(np.float32), np.float32(np.inf))
        assert np.array_equal(dist.cpu().numpy(), want)
        assert tr["n_new"][-1] == 0 and np.all(tr["n_new"][:-1] > 0)
        assert set(tr["direction"].tolist()) <= {gbx.DIR_PUSH, gbx.DIR_PULL}
        assert tr["direction"][0] == gbx.DIR_PUSH
        # a push iteration relaxes exactly the out-edges of the queued vertices, a pull every in-edge
        push = tr["direction"] == gbx.DIR_PUSH
        assert np.array_equal(tr["e_exam"][push], tr["mf"][push])
        assert np.all(tr["e_exam"][~push] == og.nnz)
        assert tr["nf"][0] == 1 and np.array_equal(tr["nf"][1:], tr["n_new"][:-1])
    g.free()


def test_sssp_isolated_source_and_bad_arguments():
    n, s, d, w, og, g = wgraph("dups")
    dist = torch.zeros(n, dtype=torch.float32, device="cuda")
    deg = np.diff(og.out_ptr)
    iso = int(np.flatnonzero(deg == 0)[0]) if np.any(deg == 0) else None
    if iso is not None:
        gbx.sssp(g, iso, dist)
        gbx.graph_sync(g)
        want = np.full(n, np.inf, np.float32)
        want[iso] = 0.0
        assert np.array_equal(dist.cpu().numpy(), want)
    with pytest.raises(gbx.GbxError) as e:
        gbx.sssp(g, n, dist)
    assert e.value.status == gbx.ERR_INVALID_INDEX
    with pytest.raises(gbx.GbxError) as e:
        gbx.sssp(g, 0, dist, gbx.desc_init(push_sort=1))
    assert e.value.status == gbx.ERR_NOT_SUPPORTED


def _pull_shape(shape):
    """Graphs whose in-edge lists cut across the pull's equal per-warp chunks in every way: a hub
    row spanning many chunks, long runs of one-edge rows (rows ending at lane and chunk borders),
    and rows with in-edges interleaved with many rows without any."""
    rng = np.random.default_rng(81)
    if shape == "star":  # vertex 0 is every other vertex's neighbour, plus a weighted path
        n = 20001
        s = np.concatenate([np.arange(1, n), np.arange(1, n - 1)])
        d = np.concatenate([np.zeros(n - 1, np.int64), np.arange(2, n)])
        return n, s, d, True
    if shape == "cycle":  # directed: every row has exactly one in-edge, n iterations deep
        n = 2000
        s = np.arange(n)
        return n, s, (s + 1) % n, False
    # mixed: sparse random edges on a third of the vertices, a hub to 4000 of them, the rest isolated
    n = 30000
    live = rng.choice(n, n // 3, replace=False)
    s = live[rng.integers(0, len(live), 3 * len(live))]
    d = live[rng.integers(0, len(live), 3 * len(live))]
    hub = int(live[0])
    fan = live[rng.choice(len(live), 4000, replace=False)]
    return n, np.concatenate([s, np.full(len(fan), hub)]), np.concatenate([d, fan]), True


@pytest.mark.parametrize("shape", ["star", "cycle", "mixed"])
def test_sssp_pull_chunk_borders(shape):
    n, s, d, sym = _pull_shape(shape)
    w = weights(len(s), 82, True)
    og = oracle.graph_weighted(n, s, d, w, symmetrize=sym)
    g = gbx.graph_build(n, s, d, symmetrize=sym)
    gbx.graph_set_weights(g, s, d, w)
    dist = torch.zeros(n, dtype=torch.float32, device="cuda")
    srcs = [0, 1, n // 2] if shape != "mixed" else [int(x) for x in synth.sources(n, s, d, 3, seed=8)]
    for src in srcs:
        want, _ = oracle.sssp(og, src)
        for desc in [gbx.desc_init(direction=gbx.DIR_PULL), gbx.desc_init(), gbx.desc_init(direction=gbx.DIR_PUSH),
                     gbx.desc_init(alpha=0.2, beta=0.3)]:
            gbx.sssp(g, src, dist, desc)
            gbx.graph_sync(g)
            assert np.array_equal(dist.cpu().numpy(), want), (shape, src, desc.direction, desc.alpha)
    g.free()
