"""Host-side pieces of the benchmark that need no GPU: the SSSP byte model, the
measured-peak lookup and the rule that DRAM traffic from a committed ncu summary
is reported only for the kernel source it was taken on."""
import os
import shutil

import numpy as np

import bench


def _trace(rows):
    dt = np.dtype([("direction", np.int32), ("nf", np.int64), ("e_exam", np.int64), ("n_new", np.int64)])
    return np.array(rows, dtype=dt)


def test_sssp_bytes_counts_each_term_once():
    n = 64
    push = (1, 3, 10, 4)   # 3 queued vertices, 10 relaxed edges, 4 improved
    pull = (2, 0, 100, 5)  # every in-edge (100) relaxed, 5 improved
    # init: distances and stamps (8 B a vertex)
    # push: id, prefix, row start per queued vertex; column, weight, target distance per edge;
    #       distance, stamp, queue slot and prefix per improved vertex
    # pull: row list and row starts (8 B a vertex at most), column, weight and source distance
    #       per in-edge, distance and stamp per improved vertex
    # pull then push: the stamps read once to queue the improved vertices
    p_push = 12 * 3 + 12 * 10 + 16 * 4
    p_pull = 8 * 64 + 12 * 100 + 8 * 5
    assert bench.sssp_bytes(_trace([push, pull]), n) == 8 * 64 + p_push + p_pull
    assert bench.sssp_bytes(_trace([pull, push]), n) == 8 * 64 + p_pull + 4 * 64 + p_push
    assert bench.sssp_bytes(_trace([]), n) == 8 * n


def test_peak_is_the_measured_copy_bandwidth():
    peak, kind = bench.peaks()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        import json

        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert kind == "fallback" and peak == bench.FALLBACK_HBM_GBS


def test_committed_dram_summary_is_well_formed():
    kv = {}
    for line in open(os.path.join(bench.ROOT, "profiles", "bfs_kernel_rmat22_dram.txt")):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    assert len(kv["kernel_source_sha"]) == 16 and int(kv["kernel_source_sha"], 16) >= 0
    # DRAM moves whole sectors: at least the algorithmic bytes per launch of the same sources
    assert float(kv["dram_bytes_per_launch"]) >= float(kv["algorithmic_bytes_per_launch_64_sources"])


def test_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    csrc = root / "paper_1804_03327_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("bfs.cu", "frontier.cuh", "gbx_internal.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_1804_03327_gb300", "csrc", f), csrc / f)
    (root / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.ncu_traffic(22) is None  # no summary at all
    summary = root / "profiles" / "bfs_kernel_rmat22_dram.txt"
    summary.write_text(f"# comment = ignored\nkernel_source_sha = {bench.kernel_source_sha()}\n"
                       "dram_bytes_per_launch = 123456\n")
    assert bench.ncu_traffic(22) == 123456.0
    with open(csrc / "bfs.cu", "a") as fh:  # the kernel changed after the capture
        fh.write("\n// edited\n")
    assert bench.ncu_traffic(22) is None
