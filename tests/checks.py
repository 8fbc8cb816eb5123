"""Result checks shared by the parity tests (test code, not the oracle)."""
import numpy as np


def assert_valid_parents(out_ptr, out_col, depth, parent, source):
    """Any parent p of v with an edge p -> v and depth[p] = depth[v] - 1 is valid
    (early exit may pick any one); the source is its own parent; unreached -1."""
    depth = np.asarray(depth)
    parent = np.asarray(parent)
    n = len(depth)
    assert parent[source] == source
    reached = depth >= 0
    assert np.all(parent[~reached] == -1)
    v = np.flatnonzero(reached)
    v = v[v != source]
    p = parent[v]
    assert np.all((p >= 0) & (p < n)), "parent out of range"
    assert np.all(depth[p] == depth[v] - 1), "parent depth is not depth - 1"
    # edge p -> v exists: v must appear in row p of A (rows sorted ascending)
    starts = np.asarray(out_ptr)[p]
    ends = np.asarray(out_ptr)[p + 1]
    col = np.asarray(out_col)
    for a, b, pp, vv in zip(starts, ends, p, v):
        k = np.searchsorted(col[a:b], vv)
        assert k < b - a and col[a + k] == vv, f"no edge {pp} -> {vv}"
