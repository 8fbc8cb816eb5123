"""GPU parity of the batched multi-source BFS (gbx_bfs_batch): every lane's
depth row must equal the CPU oracle's single-source BFS from that lane's
source, bit-exactly, whatever the direction schedule, lane count (ragged last
word), depth type or repeated sources."""
import numpy as np
import pytest

import oracle
import synth
from paper_1804_03327_gb300 import gbx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

_cache = {}


def graph(name):
    if name not in _cache:
        if name == "rmat12":
            n, s, d = synth.rmat_edges(12, 16, seed=31)
            sym = True
        elif name == "rmat11-directed":
            n, s, d = synth.rmat_edges(11, 8, seed=32)
            sym = False
        elif name == "grid":
            n, s, d = synth.grid_edges(70, 45, p_delete=0.01, seed=33)
            sym = True
        _cache[name] = (n, s, d, oracle.graph(n, s, d, symmetrize=sym), gbx.graph_build(n, s, d, symmetrize=sym))
    return _cache[name]


def run_batch(g, n, sources, desc=None, dtype=torch.int32):
    depth = torch.full((len(sources), n), 1234, dtype=dtype, device="cuda")
    gbx.bfs_batch(g, sources, depth, desc)
    gbx.graph_sync(g)
    return depth.cpu().numpy().astype(np.int32)


@pytest.mark.parametrize("name", ["rmat12", "rmat11-directed", "grid"])
@pytest.mark.parametrize("S", [1, 5, 64, 65, 200, 256])
@pytest.mark.parametrize("direction", [gbx.DIR_AUTO, gbx.DIR_PUSH, gbx.DIR_PULL])
def test_batch_lanes_equal_single_source(name, S, direction):
    n, s, d, og, g = graph(name)
    srcs = list(synth.sources(n, s, d, S, seed=S))
    if len(srcs) > 3:
        srcs[-1] = srcs[0]  # a repeated source
    got = run_batch(g, n, srcs, gbx.desc_init(direction=direction))
    want = oracle.ms_bfs(og, srcs)
    assert np.array_equal(got, want)


def test_batch_int16_depth_and_trace():
    n, s, d, og, g = graph("grid")
    srcs = synth.sources(n, s, d, 130, seed=4)
    got = run_batch(g, n, srcs, gbx.desc_init(), dtype=torch.int16)
    want = oracle.ms_bfs(og, srcs)
    assert np.array_equal(got, want)
    tr = gbx.bfs_batch_trace(g)
    assert len(tr) == want.max() + 1
    assert tr["n_new"][-1] == 0
    # pairs found per level sum to the reached (vertex, lane) pairs minus the sources
    assert tr["n_new"].sum() == np.sum(want > 0)
    assert set(tr["direction"]) <= {gbx.DIR_PUSH, gbx.DIR_PULL}


def test_batch_alpha_extremes_force_each_direction():
    n, s, d, og, g = graph("rmat12")
    srcs = synth.sources(n, s, d, 100, seed=7)
    want = oracle.ms_bfs(og, srcs)
    for alpha, expect in [(1e9, gbx.DIR_PUSH), (0.0, gbx.DIR_PULL)]:
        got = run_batch(g, n, srcs, gbx.desc_init(alpha=alpha))
        assert np.array_equal(got, want)
        tr = gbx.bfs_batch_trace(g)
        assert set(tr["direction"]) == {expect}


def test_batch_then_single_source_share_scratch():
    n, s, d, og, g = graph("rmat12")
    srcs = synth.sources(n, s, d, 70, seed=9)
    got = run_batch(g, n, srcs)
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    gbx.bfs(g, int(srcs[3]), depth, None)
    gbx.graph_sync(g)
    assert np.array_equal(depth.cpu().numpy(), got[3])
    got2 = run_batch(g, n, srcs[:10])
    assert np.array_equal(got2, got[:10])


@pytest.mark.parametrize("name", ["rmat12", "rmat11-directed", "grid"])
@pytest.mark.parametrize("S", [64, 100, 200])
def test_batch_every_build_and_block_cap(name, S):
    """blocks_per_sm 1 and 2 cap the default build, 3 and more select the
    register-lean build (at most 128 sources); every choice gives the oracle's
    depths in each direction."""
    n, s, d, og, g = graph(name)
    srcs = synth.sources(n, s, d, S, seed=S + 11)
    want = oracle.ms_bfs(og, srcs)
    for bps in (1, 2, 3, 7):
        for direction in (gbx.DIR_AUTO, gbx.DIR_PUSH, gbx.DIR_PULL):
            got = run_batch(g, n, srcs, gbx.desc_init(direction=direction, blocks_per_sm=bps))
            assert np.array_equal(got, want), (bps, direction)
        tr = gbx.bfs_batch_trace(g)
        assert len(tr) == want.max() + 1 and tr["n_new"].sum() == np.sum(want > 0)


def test_batch_rejects_bad_arguments():
    n, s, d, og, g = graph("rmat12")
    depth = torch.empty((2, n), dtype=torch.int32, device="cuda")
    with pytest.raises(gbx.GbxError) as e:
        gbx.bfs_batch(g, [0, n], depth)
    assert e.value.status == gbx.ERR_INVALID_INDEX
    with pytest.raises(gbx.GbxError) as e:
        gbx.bfs_batch(g, [0, 1], depth, gbx.desc_init(blocks_per_sm=-1))
    assert e.value.status == gbx.ERR_INVALID_VALUE


@pytest.mark.slow
@pytest.mark.parametrize("S,bps", [(64, 0), (64, 3), (1024, 0)])
def test_full_size_rmat21_batch_sampled_lanes(S, bps):
    """RMAT scale 21 (edge factor 16) with S sources in one batch, default and
    register-lean builds: sampled lanes bit-exact against the oracle."""
    n, s, d = synth.rmat_edges(21, 16, seed=1)
    og = oracle.graph(n, s, d)
    g = gbx.graph_build(n, s, d)
    srcs = synth.sources(n, s, d, S, seed=1)
    depth = torch.empty((S, n), dtype=torch.int16, device="cuda")
    gbx.bfs_batch(g, srcs, depth, gbx.desc_init(blocks_per_sm=bps))
    gbx.graph_sync(g)
    for b in sorted({0, 1, S // 2, S - 1}):
        assert np.array_equal(depth[b].cpu().numpy().astype(np.int32), oracle.bfs(og, srcs[b])[0])
    g.free()


@pytest.mark.slow
def test_full_size_grid2048_batch_sampled_lanes():
    n, s, d = synth.grid_edges(2048, 2048, p_delete=0.01, seed=1)
    og = oracle.graph(n, s, d)
    g = gbx.graph_build(n, s, d)
    srcs = synth.sources(n, s, d, 64, seed=1)
    depth = torch.empty((64, n), dtype=torch.int16, device="cuda")
    gbx.bfs_batch(g, srcs, depth)
    gbx.graph_sync(g)
    for b in (0, 33, 63):
        assert np.array_equal(depth[b].cpu().numpy().astype(np.int32), oracle.bfs(og, srcs[b])[0])
    g.free()
