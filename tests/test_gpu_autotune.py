"""Autotuner: the chosen descriptor gives the same depths as the oracle, and a
cached choice is returned without re-timing."""
import os

import numpy as np
import pytest

import oracle
import synth
from paper_1804_03327_gb300 import gbx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_autotune_bfs_and_cache(tmp_path):
    n, s, d = synth.rmat_edges(13, 16, seed=51)
    og = oracle.graph(n, s, d)
    g = gbx.graph_build(n, s, d)
    tune_src = synth.sources(n, s, d, 8, seed=52)
    cache = str(tmp_path / "tune.txt")
    desc, ms = gbx.autotune(g, gbx.TUNE_BFS, tune_src, cache)
    assert ms > 0 and desc.heuristic in (gbx.HEUR_RATIO, gbx.HEUR_BEAMER)
    assert os.path.exists(cache) and len(open(cache).read().splitlines()) == 1
    desc2, ms2 = gbx.autotune(g, gbx.TUNE_BFS, tune_src, cache)
    assert ms2 == pytest.approx(ms, rel=1e-6) and desc2.alpha == pytest.approx(desc.alpha)
    assert len(open(cache).read().splitlines()) == 1  # served from the cache
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    for src in synth.sources(n, s, d, 5, seed=53):
        gbx.bfs(g, int(src), depth, None, desc)
        gbx.graph_sync(g)
        assert np.array_equal(depth.cpu().numpy(), oracle.bfs(og, src)[0])


def test_autotune_batch():
    n, s, d = synth.grid_edges(80, 60, p_delete=0.01, seed=54)
    og = oracle.graph(n, s, d)
    g = gbx.graph_build(n, s, d)
    srcs = synth.sources(n, s, d, 64, seed=55)
    desc, ms = gbx.autotune(g, gbx.TUNE_BATCH, srcs)
    assert ms > 0
    depth = torch.empty((64, n), dtype=torch.int32, device="cuda")
    gbx.bfs_batch(g, srcs, depth, desc)
    gbx.graph_sync(g)
    assert np.array_equal(depth.cpu().numpy(), oracle.ms_bfs(og, srcs))


def test_autotune_sssp():
    n, s, d = synth.rmat_edges(12, 16, seed=56)
    w = (np.arange(len(s)) % 13 + 1).astype(np.float32)
    og = oracle.graph_weighted(n, s, d, w)
    g = gbx.graph_build(n, s, d)
    with pytest.raises(gbx.GbxError) as e:  # no weights yet
        gbx.autotune(g, gbx.TUNE_SSSP, synth.sources(n, s, d, 4, seed=57))
    assert e.value.status == gbx.ERR_INVALID_VALUE
    gbx.graph_set_weights(g, s, d, w)
    desc, ms = gbx.autotune(g, gbx.TUNE_SSSP, synth.sources(n, s, d, 4, seed=57))
    assert ms > 0 and desc.direction in (gbx.DIR_AUTO, gbx.DIR_PUSH, gbx.DIR_PULL)
    dist = torch.empty(n, dtype=torch.float32, device="cuda")
    for src in synth.sources(n, s, d, 3, seed=58):
        gbx.sssp(g, int(src), dist, desc)
        gbx.graph_sync(g)
        assert np.array_equal(dist.cpu().numpy(), oracle.sssp(og, int(src))[0])
