"""Input generators: determinism, counter-based independence and shape."""
import numpy as np

import synth


def test_splitmix64_published_vector():
    # SplitMix64 from state 0: the first output is 0xE220A8397B1DCDAF
    assert synth.draw(0, 0) == 0xE220A8397B1DCDAF


def test_rmat_deterministic_and_in_range():
    n, s1, d1 = synth.rmat_edges(10, 16, seed=1)
    _, s2, d2 = synth.rmat_edges(10, 16, seed=1)
    _, s3, _ = synth.rmat_edges(10, 16, seed=2)
    assert n == 1024 and len(s1) == 16 * 1024
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)
    assert not np.array_equal(s1, s3)
    assert s1.min() >= 0 and s1.max() < n and d1.min() >= 0 and d1.max() < n


def test_rmat_quadrant_skew_without_relabel():
    """With a = 0.57 the top-left quadrant is the most likely at each bit level."""
    n, s, d = synth.rmat_edges(12, 16, seed=3, relabel=False)
    top = (s < n // 2) & (d < n // 2)
    assert abs(top.mean() - 0.57) < 0.02


def test_permutation_is_a_bijection():
    p = synth.permutation(5000, seed=9)
    assert np.array_equal(np.sort(p), np.arange(5000))


def test_grid_edge_counts():
    n, s, d = synth.grid_edges(40, 30, p_delete=0.0)
    assert n == 1200 and len(s) == 30 * 39 + 29 * 40
    assert np.all(s < d)
    n, s1, _ = synth.grid_edges(2048, 2048, p_delete=0.01, seed=1)
    slots = 2 * 2048 * 2047
    assert abs(len(s1) - 0.99 * slots) < 5 * np.sqrt(0.01 * slots)


def test_sources_distinct_nonzero_degree():
    n, s, d = synth.rmat_edges(12, 4, seed=5)
    src = synth.sources(n, s, d, 64, seed=1)
    assert len(src) == 64 and len(set(src.tolist())) == 64
    touched = np.zeros(n, bool)
    keep = s != d
    touched[s[keep]] = True
    touched[d[keep]] = True
    assert touched[src].all()


def test_vertex_set_density():
    v = synth.vertex_set(100000, 0.25, seed=4)
    assert abs(v.mean() - 0.25) < 0.01
    assert np.array_equal(v, synth.vertex_set(100000, 0.25, seed=4))
