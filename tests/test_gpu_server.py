"""Continuous-batching BFS server: every query's depth row equals the oracle's,
and a query's result is the same when it runs alone and when it runs inside a
mix of concurrently batched queries on several graphs."""
import time

import numpy as np
import pytest

import oracle
import synth
from paper_1804_03327_gb300 import gbx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

_graphs = {}


def graphs():
    if not _graphs:
        for name, (n, s, d), sym in [("rmat12", synth.rmat_edges(12, 16, seed=41), True),
                                     ("rmat11-directed", synth.rmat_edges(11, 8, seed=42), False),
                                     ("grid", synth.grid_edges(60, 50, p_delete=0.01, seed=43), True)]:
            _graphs[name] = (n, s, d, oracle.graph(n, s, d, symmetrize=sym),
                             gbx.graph_build(n, s, d, symmetrize=sym))
    return _graphs


def filled_all(sizes, value, dtype=None):
    """Depth buffers pre-filled with a sentinel.  The fills run on torch's stream
    and the server's streams do not wait on it, so they must have finished before
    a buffer is submitted (one synchronisation, then the submissions back to back)."""
    outs = [torch.full((n,), value, dtype=dtype or torch.int32, device="cuda") for n in sizes]
    torch.cuda.synchronize()
    return outs


def filled(n, value, dtype=None):
    return filled_all([n], value, dtype)[0]


def drain(srv, want, timeout=60.0):
    got = {}
    t0 = time.time()
    while len(got) < want:
        for c in srv.poll():
            got[c.tag] = c
        assert time.time() - t0 < timeout, "server did not finish"
    return got


def test_server_results_alone_equal_results_in_the_mix():
    gs = graphs()
    names = list(gs)
    srv = gbx.Server(max_batch=64, slots=2)
    gid = {nm: srv.add_graph(gs[nm][4]) for nm in names}
    # alone
    n0, s0, d0, og0, g0 = gs["rmat12"]
    probe_src = int(synth.sources(n0, s0, d0, 1, seed=99)[0])
    alone = filled(n0, 555)
    assert srv.submit(gid["rmat12"], probe_src, alone, tag=10**9)
    c = drain(srv, 1)[10**9]
    assert c.status == 0 and c.batch_size == 1
    alone_np = alone.cpu().numpy().copy()
    assert np.array_equal(alone_np, oracle.bfs(og0, probe_src)[0])
    # in the mix: 360 queries over three graphs, the probe in the middle
    rng = np.random.default_rng(5)
    jobs = []
    for k in range(360):
        nm = names[k % 3]
        n, s, d, og, g = gs[nm]
        src = int(synth.sources(n, s, d, 40, seed=k % 7)[rng.integers(0, 40)])
        jobs.append((nm, src))
    jobs.insert(180, ("rmat12", probe_src))
    outs = filled_all([gs[nm][0] for nm, _ in jobs], 777)
    for tag, (nm, src) in enumerate(jobs):
        assert srv.submit(gid[nm], src, outs[tag], tag=tag)
    got = drain(srv, len(jobs))
    assert all(c.status == 0 for c in got.values())
    assert max(c.batch_size for c in got.values()) > 1  # queries were batched
    for tag, (nm, src) in enumerate(jobs):
        og = gs[nm][3]
        assert np.array_equal(outs[tag].cpu().numpy(), oracle.bfs(og, src)[0]), (nm, src)
    assert np.array_equal(outs[180].cpu().numpy(), alone_np)  # same alone and in the mix
    for c in got.values():
        assert c.t_submit <= c.t_launch <= c.t_done
    st = srv.stats()
    assert st["queued"] == 0 and st["in_flight"] == 0 and st["rejected"] == 0
    srv.destroy()


def test_server_int16_rows_and_admission():
    gs = graphs()
    n, s, d, og, g = gs["grid"]
    srv = gbx.Server(max_batch=64, slots=1, max_pending=5, depth_type=gbx.DEPTH_I16)
    gid = srv.add_graph(g)
    srcs = synth.sources(n, s, d, 40, seed=3)
    outs, accepted = [], 0
    refused = 0
    bufs = filled_all([n] * len(srcs), 9, torch.int16)
    for k, src in enumerate(srcs):
        out = bufs[k]
        if srv.submit(gid, int(src), out, tag=k):
            outs.append((k, src, out))
            accepted += 1
        else:
            refused += 1
    got = drain(srv, accepted)
    assert refused == srv.stats()["rejected"]
    for k, src, out in outs:
        assert got[k].status == 0
        assert np.array_equal(out.cpu().numpy().astype(np.int32), oracle.bfs(og, src)[0])
    srv.destroy()


def test_server_memory_budget_limits_lanes():
    gs = graphs()
    n, s, d, og, g = gs["rmat12"]
    # scratch of a 64-lane batch: V, three found-lane buffers, four depth planes, touched list
    one_word = 8 * 8 * n + 4 * (n + 1)
    srv = gbx.Server(max_batch=1024, slots=1, memory_budget=2 * one_word)
    gid = srv.add_graph(g)
    assert srv.lanes(gid) == 128
    srv.destroy()
    srv = gbx.Server(max_batch=64, memory_budget=100)
    with pytest.raises(gbx.GbxError) as e:
        srv.add_graph(g)
    assert e.value.status == gbx.ERR_OUT_OF_MEMORY
    srv.destroy()


def test_server_per_graph_descriptor():
    """Batches of a graph run with the descriptor set for it (here: pull only on the
    grid, push only on the RMAT graph); results stay equal to the oracle's."""
    gs = graphs()
    srv = gbx.Server(max_batch=64, slots=2)
    ids = {nm: srv.add_graph(gs[nm][4]) for nm in ("rmat12", "grid")}
    srv.set_graph_desc(ids["grid"], gbx.desc_init(direction=gbx.DIR_PULL, pull_probe=4))
    srv.set_graph_desc(ids["rmat12"], gbx.desc_init(direction=gbx.DIR_PUSH))
    with pytest.raises(gbx.GbxError) as e:
        srv.set_graph_desc(99, gbx.desc_init())
    assert e.value.status == gbx.ERR_INVALID_INDEX
    with pytest.raises(gbx.GbxError) as e:
        srv.set_graph_desc(ids["grid"], gbx.desc_init(pull_probe=2))
    assert e.value.status == gbx.ERR_INVALID_VALUE
    jobs = []
    for k in range(100):
        nm = ("rmat12", "grid")[k % 2]
        n, s, d, og, g = gs[nm]
        jobs.append((nm, int(synth.sources(n, s, d, 20, seed=11)[k % 20])))
    outs = filled_all([gs[nm][0] for nm, _ in jobs], 5)
    for k, (nm, src) in enumerate(jobs):
        assert srv.submit(ids[nm], src, outs[k], tag=k)
    got = drain(srv, len(jobs))
    assert all(c.status == 0 for c in got.values())
    for k, (nm, src) in enumerate(jobs):
        assert np.array_equal(outs[k].cpu().numpy(), oracle.bfs(gs[nm][3], src)[0])
    srv.destroy()
