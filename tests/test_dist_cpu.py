"""The multi-rank path of the benchmark on CPU (gloo, world size 2): each rank
takes its own seeded sources (weak scaling, no data-path collective), and the
whole-job numbers are the longest timed region over the ranks and the sum of
the edges every rank traversed."""
import os
import socket

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, s, d = synth.rmat_edges(10, 16, seed=1)
        mine = bench.rank_sources(n, s, d, rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, [int(x) for x in mine])
        # rank r times (r + 1) seconds over 100 * (r + 1) edges
        elapsed, edges = bench.aggregate_over_ranks(1.0 + rank, 100 * (rank + 1), dist, "cpu")
        out[rank] = (gathered, elapsed, edges)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_sources_and_aggregate():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    g0, e0, s0 = out[0]
    g1, e1, s1 = out[1]
    assert g0 == g1  # both ranks see the same assignment
    assert len(g0[0]) == len(g0[1]) == bench.SOURCES
    assert not set(g0[0]) & set(g0[1])  # disjoint sources: no rank repeats another's work
    assert e0 == e1 == 2.0 and s0 == s1 == 300  # max of the timed regions, sum of the edges


def test_rank_zero_takes_the_workload_sources():
    n, s, d = synth.rmat_edges(10, 16, seed=1)
    r0 = bench.rank_sources(n, s, d, 0)
    assert np.array_equal(r0, synth.sources(n, s, d, bench.SOURCES, seed=bench.SEED))
    assert np.array_equal(bench.rank_sources(n, s, d, 1), bench.rank_sources(n, s, d, 1))  # deterministic
    assert bench.aggregate_over_ranks(3.5, 42) == (3.5, 42)  # one rank: unchanged
