"""Pins for the CPU oracle: each check comes from something other than the oracle
itself -- brute force on tiny graphs, closed forms, invariants, an outside
library (scipy), and the worked examples the paper states (tests/golden/)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- brute-force helpers (tests only)

def dense_adjacency(n, src, dst, symmetrize=True, drop_self_loops=True):
    a = np.zeros((n, n), dtype=bool)
    for u, v in zip(src.tolist(), dst.tolist()):
        if drop_self_loops and u == v:
            continue
        a[u, v] = True
        if symmetrize:
            a[v, u] = True
    return a


def brute_force_depth(adj, s):
    """Repeated dense Boolean matvec f <- (A^T f) AND NOT v (Algorithm 1)."""
    n = adj.shape[0]
    depth = np.full(n, -1, dtype=np.int64)
    f = np.zeros(n, dtype=bool)
    f[s] = True
    v = np.zeros(n, dtype=bool)
    d = 0
    while f.any():
        depth[f] = d
        v |= f
        f = (adj.T.astype(np.int64) @ f.astype(np.int64) > 0) & ~v
        d += 1
    return depth


def union_find_component(n, row_ptr, col, s):
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for u in range(n):
        for k in range(row_ptr[u], row_ptr[u + 1]):
            a, b = find(u), find(int(col[k]))
            if a != b:
                parent[a] = b
    root = find(s)
    return np.array([find(v) == root for v in range(n)])


def small_graphs():
    out = []
    for seed in range(40):
        n = 2 + (seed * 7) % 63
        p = [0.02, 0.05, 0.1, 0.3][seed % 4]
        out.append(("er", synth.er_edges(n, p, seed=seed, directed=False), True))
    for seed in range(20):
        n = 2 + (seed * 5) % 40
        out.append(("er-directed", synth.er_edges(n, 0.08, seed=100 + seed, directed=True), False))
    for n in (2, 5, 17, 64):
        out.append(("path", synth.path_edges(n), True))
        out.append(("tree", synth.tree_edges(n, seed=n), True))
    for k in (1, 3, 30):
        out.append(("star", synth.star_edges(k), True))
    for n in (2, 6, 20):
        out.append(("complete", synth.complete_edges(n), True))
    # two disjoint components plus isolated vertices
    n1, s1, d1 = synth.path_edges(10)
    out.append(("disconnected", (30, np.concatenate([s1, s1 + 15]), np.concatenate([d1, d1 + 15])), True))
    return out


# ---------------------------------------------------------------- CSR build

@pytest.mark.parametrize("symmetrize", [True, False])
def test_csr_build_matches_edge_sets(symmetrize):
    for seed in range(30):
        n = 1 + seed % 50
        rng = np.random.default_rng(seed)
        m = int(rng.integers(0, 200))
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        row_ptr, col = oracle.csr_build(n, src, dst, symmetrize=symmetrize)
        want = set()
        for u, v in zip(src.tolist(), dst.tolist()):
            if u != v:
                want.add((u, v))
                if symmetrize:
                    want.add((v, u))
        got = [(u, int(c)) for u in range(n) for c in col[row_ptr[u]:row_ptr[u + 1]]]
        assert len(got) == len(set(got)) == len(want)
        assert set(got) == want
        for u in range(n):
            row = col[row_ptr[u]:row_ptr[u + 1]]
            assert np.all(np.diff(row) > 0)


def test_csr_build_keeps_self_loops_when_asked():
    row_ptr, col = oracle.csr_build(3, [0, 1, 1], [0, 1, 2], symmetrize=False, drop_self_loops=False)
    assert row_ptr.tolist() == [0, 1, 3, 3]
    assert col.tolist() == [0, 1, 2]


def test_csr_build_rejects_bad_vertex():
    with pytest.raises(ValueError):
        oracle.csr_build(3, [0, 5], [1, 2])


def test_transpose_reverses_every_entry():
    n, src, dst = synth.er_edges(30, 0.1, seed=3, directed=True)
    row_ptr, col = oracle.csr_build(n, src, dst, symmetrize=False)
    t_ptr, t_col = oracle.transpose(n, row_ptr, col)
    fwd = {(u, int(c)) for u in range(n) for c in col[row_ptr[u]:row_ptr[u + 1]]}
    rev = {(int(c), u) for u in range(n) for c in t_col[t_ptr[u]:t_ptr[u + 1]]}
    assert fwd == rev
    for u in range(n):
        assert np.all(np.diff(t_col[t_ptr[u]:t_ptr[u + 1]]) > 0)


# ---------------------------------------------------------------- BFS: brute force, closed forms, library

def test_bfs_equals_brute_force_dense_matvec():
    count = 0
    for name, (n, src, dst), sym in small_graphs():
        g = oracle.graph(n, src, dst, symmetrize=sym)
        adj = dense_adjacency(n, src, dst, symmetrize=sym)
        for s in range(0, n, max(1, n // 5)):
            depth, parent, levels = oracle.bfs(g, s)
            assert np.array_equal(depth, brute_force_depth(adj, s)), (name, n, s)
            assert levels == depth.max() + 1
            count += 1
    assert count > 200


def test_bfs_grid_closed_form_manhattan():
    w, h = 37, 23
    n, src, dst = synth.grid_edges(w, h, p_delete=0.0)
    g = oracle.graph(n, src, dst)
    for (x0, y0) in [(0, 0), (36, 22), (17, 9)]:
        depth, _, levels = oracle.bfs(g, y0 * w + x0)
        ys, xs = np.divmod(np.arange(n), w)
        assert np.array_equal(depth, np.abs(xs - x0) + np.abs(ys - y0))
        assert levels == depth.max() + 1


def test_bfs_path_star_complete_closed_forms():
    n, s_, d_ = synth.path_edges(50)
    g = oracle.graph(n, s_, d_)
    depth, _, _ = oracle.bfs(g, 13)
    assert np.array_equal(depth, np.abs(np.arange(50) - 13))
    n, s_, d_ = synth.star_edges(40)
    g = oracle.graph(n, s_, d_)
    depth, _, _ = oracle.bfs(g, 0)
    assert depth[0] == 0 and np.all(depth[1:] == 1)
    depth, _, _ = oracle.bfs(g, 7)
    assert depth[7] == 0 and depth[0] == 1 and np.sum(depth == 2) == 39
    n, s_, d_ = synth.complete_edges(25)
    g = oracle.graph(n, s_, d_)
    depth, _, _ = oracle.bfs(g, 4)
    assert depth[4] == 0 and np.sum(depth == 1) == 24


def test_bfs_invariants_rmat():
    n, src, dst = synth.rmat_edges(12, 16, seed=7)
    g = oracle.graph(n, src, dst)
    for s in synth.sources(n, src, dst, 4, seed=7):
        depth, parent, _ = oracle.bfs(g, s)
        assert depth[s] == 0 and parent[s] == s
        comp = union_find_component(n, g.out_ptr, g.out_col, s)
        assert np.array_equal(depth >= 0, comp)
        assert np.all(parent[~comp] == -1)
        for v in np.flatnonzero(comp):
            if v == s:
                continue
            p = parent[v]
            assert depth[p] == depth[v] - 1
            assert v in g.out_col[g.out_ptr[p]:g.out_ptr[p + 1]]
        rows = np.repeat(np.arange(n), np.diff(g.out_ptr))
        both = (depth[rows] >= 0) & (depth[g.out_col] >= 0)
        assert np.all(np.abs(depth[rows][both] - depth[g.out_col][both]) <= 1)


def test_bfs_matches_scipy_shortest_path():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for sym, (n, src, dst) in [(True, synth.rmat_edges(11, 8, seed=3)), (False, synth.er_edges(60, 0.04, 9, True))]:
        g = oracle.graph(n, src, dst, symmetrize=sym)
        mat = sp.csr_matrix((np.ones(g.nnz), g.out_col, g.out_ptr), shape=(n, n))
        for s in synth.sources(n, src, dst, 3, seed=5):
            depth, _, _ = oracle.bfs(g, s)
            dist = csgraph.shortest_path(mat, directed=True, unweighted=True, indices=int(s))
            want = np.where(np.isinf(dist), -1, dist).astype(np.int64)
            assert np.array_equal(depth, want)


# ---------------------------------------------------------------- level trace: closed forms

def test_trace_path_closed_form():
    n = 12
    g = oracle.graph(*synth.path_edges(n))
    depth, _, levels = oracle.bfs(g, 0)
    tr = oracle.bfs_trace(g, depth, levels)
    deg = np.diff(g.out_ptr)
    assert len(tr) == n
    for L in range(n):
        assert tr[L]["nf"] == 1 and tr[L]["mf"] == deg[L]
        assert tr[L]["nu"] == n - 1 - L
        assert tr[L]["mu"] == deg[L + 1:].sum()
        want_exam = (1 if L + 1 <= n - 1 else 0) + deg[L + 2:].sum()
        assert tr[L]["e_exam"] == want_exam
        assert tr[L]["n_new"] == (1 if L + 1 <= n - 1 else 0)


def test_trace_star_closed_form():
    k = 9
    g = oracle.graph(*synth.star_edges(k))
    depth, _, levels = oracle.bfs(g, 1)
    tr = oracle.bfs_trace(g, depth, levels)
    assert levels == 3
    want = [
        dict(nf=1, mf=1, nu=k, nu_nz=k, mu=2 * k - 1, e_exam=k, n_new=1, mf_new=k),
        dict(nf=1, mf=k, nu=k - 1, nu_nz=k - 1, mu=k - 1, e_exam=k - 1, n_new=k - 1, mf_new=k - 1),
        dict(nf=k - 1, mf=k - 1, nu=0, nu_nz=0, mu=0, e_exam=0, n_new=0, mf_new=0),
    ]
    for L, w in enumerate(want):
        for key, val in w.items():
            assert tr[L][key] == val, (L, key)


def test_trace_conservation_rmat():
    n, src, dst = synth.rmat_edges(11, 16, seed=2)
    g = oracle.graph(n, src, dst)
    s = synth.sources(n, src, dst, 1, seed=2)[0]
    depth, _, levels = oracle.bfs(g, s)
    tr = oracle.bfs_trace(g, depth, levels)
    indeg = np.diff(g.in_ptr)
    assert tr["nf"].sum() == np.sum(depth >= 0)
    assert np.all(tr["n_new"][:-1] == tr["nf"][1:])
    assert np.all(tr["nu"][:-1] - tr["n_new"][:-1] == tr["nu"][1:])
    assert np.all(tr["mu"][:-1] - tr["mu"][1:] == [indeg[depth == L + 1].sum() for L in range(levels - 1)])
    # early exit never examines more than the full in-degree, and at least one edge per found row
    assert np.all(tr["e_exam"] <= tr["mu"])
    assert np.all(tr["e_exam"] >= tr["n_new"])


# ---------------------------------------------------------------- direction rule (Section 6.3)

def test_direction_rule_worked_example():
    ex = json.load(open(os.path.join(GOLDEN, "direction_rule_example.json")))
    sizes = ex["frontier_sizes"]
    tr = np.zeros(len(sizes) - 1, dtype=oracle.LEVEL_DTYPE)
    tr["nf"] = sizes[:-1]
    tr["n_new"] = sizes[1:]
    got = oracle.direction_schedule(tr, ex["n"], ex["alpha"], ex["beta"])
    assert got == ex["expected_directions"]
    assert oracle.direction_schedule(tr, ex["n"], mode="pull") == ["pull"] * len(tr)


def test_direction_rule_beamer_worked_example():
    """Beamer's edge test on a hand-worked graph: the trace fields the rule reads
    (mf_new, mu) and the schedule; a step where m_f/m_u crosses alpha while the
    frontier is still small, and pull levels that return to push although the
    frontier did not shrink."""
    ex = json.load(open(os.path.join(GOLDEN, "direction_rule_beamer_example.json")))
    n = ex["n"]
    e = np.array(ex["edges"], dtype=np.int32)
    g = oracle.graph(n, e[:, 0], e[:, 1])
    depth, _, levels = oracle.bfs(g, ex["source"])
    tr = oracle.bfs_trace(g, depth, levels)
    assert levels == len(ex["expected_directions_beamer"])
    for key, want in ex["expected_trace"].items():
        assert tr[key].tolist() == want, key
    got = oracle.direction_schedule(tr, n, ex["alpha"], ex["beta"], heuristic="beamer")
    assert got == ex["expected_directions_beamer"]
    assert oracle.direction_schedule(tr, n, ex["alpha"], ex["beta"], heuristic="ratio") == \
        ex["expected_directions_ratio"]


@pytest.mark.parametrize("n", [10, 17, 40])
def test_direction_rule_beamer_path_closed_form(n):
    """Path 0 - 1 - ... - n-1 from vertex 0: after step k the new frontier {k+1} has
    2 out-edges (1 for the last vertex) and the unvisited vertices {k+2 .. n-1}
    have 2(n-k-2) - 1 in-edges, so with alpha = 1/4 the first switch to pull
    follows step k = n - 6 (2/7 > 1/4 >= 2/9); each pull level finds one vertex,
    1/n < beta = 1/8 sends it back to push, and the last step stays in push
    because nothing is left unvisited (m_u = 0)."""
    g = oracle.graph(*synth.path_edges(n))
    depth, _, levels = oracle.bfs(g, 0)
    tr = oracle.bfs_trace(g, depth, levels)
    assert levels == n
    want = ["push"] * (n - 5) + ["pull", "push", "pull", "push", "push"]
    assert oracle.direction_schedule(tr, n, 0.25, 0.125, heuristic="beamer") == want


def test_direction_rule_mesh_stays_push():
    """Section 6.3: the mesh-like graphs' best schedule is push-only; with
    alpha = 0.01 a grid frontier (<= ~2*sqrt(n)) stays below it once n > 4e4."""
    n, src, dst = synth.grid_edges(512, 512, p_delete=0.0)
    g = oracle.graph(n, src, dst)
    depth, _, levels = oracle.bfs(g, 0)
    tr = oracle.bfs_trace(g, depth, levels)
    assert set(oracle.direction_schedule(tr, n)) == {"push"}


# ---------------------------------------------------------------- masked matvec (Eq 2-5)

def _random_csr(nr, nc, p, seed):
    rng = np.random.default_rng(seed)
    a = rng.random((nr, nc)) < p
    row_ptr = np.concatenate([[0], np.cumsum(a.sum(1))]).astype(np.int32)
    col = np.nonzero(a)[1].astype(np.int32)
    return a, row_ptr, col


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("masked", [False, True])
@pytest.mark.parametrize("complement", [False, True])
@pytest.mark.parametrize("accum", [False, True])
def test_mxv_equals_dense_product(transpose, masked, complement, accum):
    for seed in range(12):
        nr, nc = 5 + seed * 3, 7 + (seed * 5) % 31
        a, row_ptr, col = _random_csr(nr, nc, 0.15, seed)
        rng = np.random.default_rng(100 + seed)
        nin, nout = (nr, nc) if transpose else (nc, nr)
        u = (rng.random(nin) < 0.3).astype(np.uint8)
        mask = (rng.random(nout) < 0.5).astype(np.uint8) if masked else None
        w_old = (rng.random(nout) < 0.4).astype(np.uint8)
        got = oracle.mxv(nr, nc, row_ptr, col, u, mask, transpose, complement, accum, w_old)
        prod = ((a.T if transpose else a).astype(np.int64) @ u.astype(np.int64)) > 0
        keep = np.ones(nout, bool) if mask is None else mask.astype(bool)
        if complement:
            keep = ~keep
        base = w_old.astype(bool) if accum else np.zeros(nout, bool)
        want = np.where(keep, base | prod, base).astype(np.uint8)
        assert np.array_equal(got, want), seed


def test_mxv_single_nonzero_gives_a_column():
    """Eq 3: if only f(i) is nonzero, f' is column i of A."""
    a, row_ptr, col = _random_csr(30, 20, 0.2, 5)
    for i in range(20):
        u = np.zeros(20, np.uint8)
        u[i] = 1
        got = oracle.mxv(30, 20, row_ptr, col, u)
        assert np.array_equal(got.astype(bool), a[:, i])


def test_mxv_complement_identity_and_zero_outside_mask():
    a, row_ptr, col = _random_csr(40, 40, 0.1, 9)
    u = synth.vertex_set(40, 0.3, seed=4)
    m = synth.vertex_set(40, 0.5, seed=5)
    x = oracle.mxv(40, 40, row_ptr, col, u, mask=m, complement=True)
    y = oracle.mxv(40, 40, row_ptr, col, u, mask=(1 - m).astype(np.uint8))
    assert np.array_equal(x, y)
    z = oracle.mxv(40, 40, row_ptr, col, u, mask=m)
    assert np.all(z[m == 0] == 0)  # Eq 4: masked-out rows are 0
    full = oracle.mxv(40, 40, row_ptr, col, u)
    assert np.array_equal(z, full & m)
    # no mask + complement: the complement of the implicit all-ones mask passes nothing
    assert not oracle.mxv(40, 40, row_ptr, col, u, complement=True).any()


def test_mxv_figure3_example():
    ex = json.load(open(os.path.join(GOLDEN, "fig3_example.json")))
    names = ex["stated_by_the_paper"]["vertices"]
    idx = {c: i for i, c in enumerate(names)}
    edges = ex["chosen_by_this_test"]["edges"]
    src = np.array([idx[a] for a, _ in edges], np.int32)
    dst = np.array([idx[b] for _, b in edges], np.int32)
    g = oracle.graph(8, src, dst)
    f = oracle.to_dense([idx[c] for c in ex["stated_by_the_paper"]["frontier"]], 8)
    v = oracle.to_dense([idx[c] for c in ex["stated_by_the_paper"]["visited"]], 8)
    children = oracle.mxv(8, 8, g.out_ptr, g.out_col, f, transpose=True)
    assert [names[i] for i in oracle.to_sparse(children)] == ex["stated_by_the_paper"]["push_children_before_filter"]
    res = oracle.mxv(8, 8, g.out_ptr, g.out_col, f, mask=v, complement=True, transpose=True)
    assert [names[i] for i in oracle.to_sparse(res)] == ex["stated_by_the_paper"]["push_result_after_visited_filter"]
    # pull computes only the unvisited rows (Figure 4c) and gets the same result
    assert [names[i] for i in np.flatnonzero(v == 0)] == ex["stated_by_the_paper"]["pull_rows_examined"]
    depth, _, _ = oracle.bfs(g, idx[ex["chosen_by_this_test"]["bfs_source"]])
    assert {names[i]: int(d) for i, d in enumerate(depth)} == ex["chosen_by_this_test"]["bfs_depth"]


def test_ms_bfs_lanes_equal_single_sources_including_duplicates():
    n, src, dst = synth.rmat_edges(9, 8, seed=11)
    g = oracle.graph(n, src, dst)
    srcs = list(synth.sources(n, src, dst, 5, seed=1))
    srcs = srcs + [srcs[0]]
    d = oracle.ms_bfs(g, srcs)
    adj = None
    for k, s in enumerate(srcs):
        assert np.array_equal(d[k], oracle.bfs(g, s)[0])
    assert np.array_equal(d[0], d[-1])
    # one lane against brute force as an outside check
    adj = dense_adjacency(n, src, dst)
    assert np.array_equal(d[1], brute_force_depth(adj, srcs[1]))


# ---------------------------------------------------------------- (min, +) semiring (Section 5.6)

def _weights(m, seed, integer=True):
    """Seeded weights: integers 1..64 (sums exact in binary32) or floats in (0, 8)."""
    rng = np.random.default_rng(seed)
    if integer:
        return rng.integers(1, 65, size=m).astype(np.float32)
    return (rng.random(m) * 8.0 + 1e-3).astype(np.float32)


@pytest.mark.parametrize("symmetrize", [True, False])
def test_csr_weights_match_pair_dictionary(symmetrize):
    n, s, d = synth.er_edges(60, 0.08, seed=21, directed=True)
    s = np.concatenate([s, s[:40]])  # parallel pairs with other weights
    d = np.concatenate([d, d[:40]])
    w = _weights(len(s), 5, integer=False)
    want = {}
    for a, b, x in zip(s.tolist(), d.tolist(), w.tolist()):
        if a == b:
            continue
        for r, c in ([(a, b), (b, a)] if symmetrize else [(a, b)]):
            want[(r, c)] = min(want.get((r, c), np.inf), x)
    g = oracle.graph_weighted(n, s, d, w, symmetrize=symmetrize)
    got = {(r, int(g.out_col[k])): float(g.out_val[k]) for r in range(n) for k in range(g.out_ptr[r], g.out_ptr[r + 1])}
    assert got == want
    got_t = {(int(g.in_col[k]), r): float(g.in_val[k]) for r in range(n) for k in range(g.in_ptr[r], g.in_ptr[r + 1])}
    assert got_t == want


@pytest.mark.parametrize("transpose,masked,complement,accum",
                         [(t, m, c, a) for t in (0, 1) for m in (0, 1) for c in (0, 1) for a in (0, 1)])
def test_minplus_with_zero_weights_is_the_boolean_matvec(transpose, masked, complement, accum):
    """All weights 0 and u in {0, +inf}: (min, +) reduces to (OR, AND) with 0 = true."""
    n, s, d = synth.er_edges(50, 0.06, seed=3, directed=True)
    g = oracle.graph_weighted(n, s, d, np.zeros(len(s), np.float32), symmetrize=False)
    for k in range(4):
        ub = synth.vertex_set(n, 0.2, seed=7 + k)
        mb = synth.vertex_set(n, 0.5, seed=17 + k) if masked else None
        wb = synth.vertex_set(n, 0.3, seed=27 + k)
        want = oracle.mxv(n, n, g.out_ptr, g.out_col, ub, mb, transpose=bool(transpose),
                          complement=bool(complement), accum=bool(accum), w_old=wb)
        u = np.where(ub != 0, 0.0, np.inf)
        w_old = np.where(wb != 0, 0.0, np.inf)
        got = oracle.mxv_minplus(n, n, g.out_ptr, g.out_col, g.out_val, u, mb, transpose=bool(transpose),
                                 complement=bool(complement), accum=bool(accum), w_old=w_old)
        assert np.array_equal(got == 0.0, want.astype(bool))
        assert np.all((got == 0.0) | np.isinf(got))


def test_minplus_unit_vector_gives_a_row_of_weights():
    n, s, d = synth.er_edges(40, 0.1, seed=9, directed=True)
    g = oracle.graph_weighted(n, s, d, _weights(len(s), 2, integer=False), symmetrize=False)
    for j in range(n):
        u = np.full(n, np.inf)
        u[j] = 0.0
        got = oracle.mxv_minplus(n, n, g.out_ptr, g.out_col, g.out_val, u, transpose=True)
        want = np.full(n, np.inf)
        for k in range(g.out_ptr[j], g.out_ptr[j + 1]):
            want[g.out_col[k]] = g.out_val[k]  # (A^T e_j)(c) = A(j, c)
        assert np.array_equal(got, want)
        got_n = oracle.mxv_minplus(n, n, g.out_ptr, g.out_col, g.out_val, u, transpose=False)
        want_n = np.full(n, np.inf)
        for r in range(n):
            for k in range(g.out_ptr[r], g.out_ptr[r + 1]):
                if g.out_col[k] == j:
                    want_n[r] = g.out_val[k]  # (A e_j)(r) = A(r, j)
        assert np.array_equal(got_n, want_n)


def test_minplus_is_tropically_linear():
    """min-plus matvec distributes over min and commutes with adding a constant."""
    n, s, d = synth.rmat_edges(7, 8, seed=4)
    g = oracle.graph_weighted(n, s, d, _weights(len(s), 3))
    rng = np.random.default_rng(1)
    for _ in range(5):
        u1 = np.where(rng.random(n) < 0.3, rng.integers(0, 100, n).astype(np.float64), np.inf)
        u2 = np.where(rng.random(n) < 0.3, rng.integers(0, 100, n).astype(np.float64), np.inf)
        f = lambda u: oracle.mxv_minplus(n, n, g.out_ptr, g.out_col, g.out_val, u, transpose=True)
        assert np.array_equal(f(np.minimum(u1, u2)), np.minimum(f(u1), f(u2)))
        assert np.array_equal(f(u1 + 5.0), f(u1) + 5.0)


def test_sssp_matches_scipy_dijkstra():
    scipy_sparse = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for directed, (n, s, d) in [(False, synth.rmat_edges(9, 8, seed=12)),
                                (True, synth.er_edges(300, 0.01, seed=13, directed=True)),
                                (False, synth.grid_edges(20, 15, p_delete=0.05, seed=14))]:
        for integer in (True, False):
            w = _weights(len(s), 6, integer=integer)
            g = oracle.graph_weighted(n, s, d, w, symmetrize=not directed)
            a = scipy_sparse.csr_matrix((g.out_val, g.out_col, g.out_ptr), shape=(n, n))
            for src in synth.sources(n, s, d, 3, seed=15):
                got, _ = oracle.sssp(g, int(src))
                want = csgraph.dijkstra(a, directed=True, indices=int(src))
                assert np.array_equal(np.isinf(got), np.isinf(want))
                fin = np.isfinite(want)
                if integer:  # integer sums below 2^24 are exact in binary32
                    assert np.array_equal(got[fin].astype(np.float64), want[fin])
                else:  # each of at most n - 1 additions rounds by at most half an ulp
                    assert np.all(np.abs(got[fin] - want[fin]) <= want[fin] * (n * 2.0 ** -24) + 1e-30)


def test_sssp_unit_weights_give_bfs_depth():
    n, s, d = synth.rmat_edges(9, 8, seed=31)
    g = oracle.graph_weighted(n, s, d, np.ones(len(s), np.float32))
    for src in synth.sources(n, s, d, 4, seed=2):
        depth, _, _ = oracle.bfs(g, int(src))
        dist, _ = oracle.sssp(g, int(src))
        assert np.array_equal(np.where(depth >= 0, depth.astype(np.float32), np.float32(np.inf)), dist)


def test_sssp_bellman_optimality_conditions():
    """d(s) = 0; d(v) <= fl32(d(u) + w) on every edge; every reached v != s has a
    tight in-edge.  (Checks the float result itself, not how it was computed.)"""
    n, s, d = synth.rmat_edges(10, 8, seed=33)
    g = oracle.graph_weighted(n, s, d, _weights(len(s), 8, integer=False))
    val32 = g.out_val.astype(np.float32)
    for src in synth.sources(n, s, d, 2, seed=4):
        dist, _ = oracle.sssp(g, int(src))
        assert dist[src] == 0.0
        tight = np.zeros(n, dtype=bool)
        for u in range(n):
            if not np.isfinite(dist[u]):
                continue
            for k in range(g.out_ptr[u], g.out_ptr[u + 1]):
                v = g.out_col[k]
                x = np.float32(dist[u] + val32[k])
                assert dist[v] <= x
                tight[v] |= dist[v] == x
        reached = np.isfinite(dist)
        reached[src] = False
        assert np.all(tight[reached])
