"""CPU oracle for the push-pull BFS hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product path (the CUDA
library ``paper_1804_03327_gb300``) never imports it and shares no code with
it.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, compiled with
gcc on first use); this file marshals numpy arrays and adds two plain rules
written in Python:

* ``direction_schedule``: the per-level push/pull choice of Section 6.3
  (``r = nnz(f)/M``; push -> pull when r rises above alpha, pull -> push when
  it falls below beta; alpha = beta = 0.01), and Beamer's edge-ratio variant
  that Section 6.3 starts from.
* ``ms_bfs``: many sources as independent single-source BFS runs (one lane
  per source), the definition the bit-parallel batched form must reproduce.

The (min, +) semiring of Section 5.6 (weighted graphs, ``mxv_minplus`` in
double, ``sssp`` as Bellman-Ford with binary32 sums) is in ``oracle.c`` too.

Pins (tests/test_oracle_pins.py): brute-force dense Boolean matvec BFS on
n <= 64, closed forms (grid Manhattan distance, path, star, complete graph),
BFS invariants, scipy's BFS as an outside library, dense-matrix mxv for every
flag combination, the Figure 3 worked example and two hand-worked direction
schedules, one per rule, plus a closed form of Beamer's rule on a path
(tests/golden/).  The (min, +) functions: weights against a Python
dictionary of pairs; the matvec
against the Boolean oracle (zero weights), unit vectors (a column of weights)
and tropical linearity; SSSP against scipy's Dijkstra (exact on integer
weights), the BFS depth (unit weights) and the Bellman optimality conditions.
Parity unpinned: none of the functions below.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LEVEL_DTYPE = np.dtype([("nf", np.int64), ("mf", np.int64), ("nu", np.int64), ("nu_nz", np.int64),
                        ("mu", np.int64), ("e_exam", np.int64), ("n_new", np.int64), ("mf_new", np.int64)])


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2, single-threaded)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            lib.oracle_csr_build.restype = i64
            lib.oracle_csr_build.argtypes = [i32, i64, p, p, i32, i32, p, p]
            lib.oracle_transpose.restype = ctypes.c_int
            lib.oracle_transpose.argtypes = [i32, p, p, p, p]
            lib.oracle_bfs.restype = i32
            lib.oracle_bfs.argtypes = [i32, p, p, i32, p, p]
            lib.oracle_bfs_trace.restype = i32
            lib.oracle_bfs_trace.argtypes = [i32, p, p, p, p, i32, p, i32]
            lib.oracle_mxv.restype = ctypes.c_int
            lib.oracle_mxv.argtypes = [i32, i32, p, p, i32, p, p, i32, i32, p]
            lib.oracle_csr_weights.argtypes = [i32, i64, p, p, p, i32, i32, p, p, p]
            lib.oracle_transpose_weighted.argtypes = [i32, p, p, p, p, p, p]
            lib.oracle_mxv_minplus.argtypes = [i32, i32, p, p, p, i32, p, p, i32, i32, p]
            lib.oracle_sssp_bf.argtypes = [i32, p, p, p, i32, p]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Graph:
    """Oracle-side graph: CSR of A (out-edges) and CSR of A^T (in-edges)."""

    def __init__(self, n, out_ptr, out_col, in_ptr, in_col):
        self.n = int(n)
        self.out_ptr, self.out_col = out_ptr, out_col
        self.in_ptr, self.in_col = in_ptr, in_col

    @property
    def nnz(self) -> int:
        return int(self.out_ptr[-1])


def csr_build(n: int, src, dst, symmetrize: bool = True, drop_self_loops: bool = True):
    """CSR (row_ptr, col) of the edge list: optional symmetrisation, self-loop
    removal, duplicate removal, ascending rows (Section 7.1)."""
    src, dst = _i32(src), _i32(dst)
    m = len(src)
    row_ptr = np.empty(n + 1, dtype=np.int32)
    col = np.empty(max(1, (2 * m) if symmetrize else m), dtype=np.int32)
    nnz = _load().oracle_csr_build(n, m, _p(src), _p(dst), int(symmetrize), int(drop_self_loops),
                                   _p(row_ptr), _p(col))
    if nnz < 0:
        raise ValueError(f"oracle_csr_build failed ({nnz})")
    return row_ptr, col[:nnz].copy()


def transpose(n: int, row_ptr, col):
    t_ptr = np.empty(n + 1, dtype=np.int32)
    t_col = np.empty(max(1, len(col)), dtype=np.int32)
    if _load().oracle_transpose(n, _p(_i32(row_ptr)), _p(_i32(col)), _p(t_ptr), _p(t_col)) != 0:
        raise MemoryError("oracle_transpose failed")
    return t_ptr, t_col[:len(col)].copy()


def graph(n: int, src, dst, symmetrize: bool = True, drop_self_loops: bool = True) -> Graph:
    out_ptr, out_col = csr_build(n, src, dst, symmetrize, drop_self_loops)
    if symmetrize:
        return Graph(n, out_ptr, out_col, out_ptr, out_col)
    in_ptr, in_col = transpose(n, out_ptr, out_col)
    return Graph(n, out_ptr, out_col, in_ptr, in_col)


def bfs(g: Graph, source: int):
    """Queue BFS: (depth int32[n], parent int32[n], levels)."""
    depth = np.empty(g.n, dtype=np.int32)
    parent = np.empty(g.n, dtype=np.int32)
    levels = _load().oracle_bfs(g.n, _p(g.out_ptr), _p(g.out_col), int(source), _p(depth), _p(parent))
    if levels < 0:
        raise ValueError(f"bad source {source}")
    return depth, parent, int(levels)


def bfs_trace(g: Graph, depth, levels: int) -> np.ndarray:
    """Per-step statistics (LEVEL_DTYPE records) for the given depths."""
    depth = _i32(depth)
    out = np.zeros(max(levels, 1), dtype=LEVEL_DTYPE)
    k = _load().oracle_bfs_trace(g.n, _p(g.out_ptr), _p(g.in_ptr), _p(g.in_col), _p(depth), int(levels),
                                 _p(out), int(levels))
    return out[:k]


def direction_schedule(trace: np.ndarray, n: int, alpha: float = 0.01, beta: float = 0.01,
                       heuristic: str = "ratio", mode: str = "auto") -> list[str]:
    """Direction ('push' / 'pull') of each BFS step (Section 6.3).

    Starts in push.  After step L the new frontier F_{L+1} decides step L+1:
    ratio rule: r = |F|/n; push -> pull if r_{L+1} > alpha and |F_{L+1}| > |F_L|;
    pull -> push if r_{L+1} < beta and |F_{L+1}| < |F_L|.
    beamer rule (the test Section 6.3 starts from): push -> pull if
    m_f / m_u > alpha, with m_f the out-edges of F_{L+1} and m_u the in-edges of
    the vertices still unvisited after step L (no switch when m_u = 0);
    pull -> push if r_{L+1} < beta, with no condition on the frontier's trend
    (Section 6.3 states Beamer's way back as nnz(f)/M < beta alone).
    Thresholds are single precision, as the descriptor carries them;
    comparisons are in double precision.
    """
    if mode in ("push", "pull"):
        return [mode] * len(trace)
    a = float(np.float32(alpha))
    b = float(np.float32(beta))
    d = "push"
    dirs = []
    for L in range(len(trace)):
        rec = trace[L]
        dirs.append(d)
        nf, nn = int(rec["nf"]), int(rec["n_new"])
        r_new = float(nn) / float(n)
        if d == "push":
            if heuristic == "ratio":
                if r_new > a and nn > nf:
                    d = "pull"
            else:
                mf = int(rec["mf_new"])
                mu = int(trace[L + 1]["mu"]) if L + 1 < len(trace) else 0
                if mu > 0 and float(mf) / float(mu) > a:
                    d = "pull"
        else:
            if heuristic == "ratio":
                if r_new < b and nn < nf:
                    d = "push"
            elif r_new < b:
                d = "push"
    return dirs


def mxv(nrows: int, ncols: int, row_ptr, col, u, mask=None, transpose: bool = False,
        complement: bool = False, accum: bool = False, w_old=None) -> np.ndarray:
    """Dense 0/1 uint8 result of the masked Boolean matvec (Eq 2-5).

    ``u``/``mask`` may be 0/1 byte vectors or index lists (sparse, int32)."""
    nin = nrows if transpose else ncols
    nout = ncols if transpose else nrows
    u = to_dense(u, nin)
    m = None if mask is None else to_dense(mask, nout)
    w = np.zeros(nout, dtype=np.uint8) if w_old is None else to_dense(w_old, nout).copy()
    rc = _load().oracle_mxv(nrows, ncols, _p(_i32(row_ptr)), _p(_i32(col)), int(transpose), _p(u), _p(m),
                            int(complement), int(accum), _p(w))
    if rc != 0:
        raise MemoryError("oracle_mxv failed")
    return w


def to_dense(v, n: int) -> np.ndarray:
    v = np.asarray(v)
    if v.dtype == np.uint8 and v.shape == (n,):
        return np.ascontiguousarray((v != 0).astype(np.uint8))
    out = np.zeros(n, dtype=np.uint8)
    out[v.astype(np.int64)] = 1
    return out


def to_sparse(v) -> np.ndarray:
    """Sorted unique int32 indices of the nonzeros (Section 3: sorted lists)."""
    return np.flatnonzero(np.asarray(v)).astype(np.int32)


def ms_bfs(g: Graph, sources) -> np.ndarray:
    """Depth int32[S, n]: one independent single-source BFS per lane."""
    sources = list(sources)
    out = np.empty((len(sources), g.n), dtype=np.int32)
    for k, s in enumerate(sources):
        out[k], _, _ = bfs(g, s)
    return out


class WeightedGraph(Graph):
    """Graph with edge weights: out_val[k] belongs to out_col[k], in_val[k] to in_col[k]
    (double; every value is a binary32 input weight)."""

    def __init__(self, n, out_ptr, out_col, out_val, in_ptr, in_col, in_val):
        super().__init__(n, out_ptr, out_col, in_ptr, in_col)
        self.out_val, self.in_val = out_val, in_val


def graph_weighted(n: int, src, dst, w, symmetrize: bool = True, drop_self_loops: bool = True) -> WeightedGraph:
    """Weighted CSR of A and of A^T; parallel pairs keep the smallest weight."""
    src, dst = _i32(src), _i32(dst)
    w = np.ascontiguousarray(w, dtype=np.float32)
    out_ptr, out_col = csr_build(n, src, dst, symmetrize, drop_self_loops)
    out_val = np.empty(max(1, len(out_col)), dtype=np.float64)
    if _load().oracle_csr_weights(n, len(src), _p(src), _p(dst), _p(w), int(symmetrize), int(drop_self_loops),
                                  _p(out_ptr), _p(out_col), _p(out_val)) != 0:
        raise ValueError("oracle_csr_weights: the CSR does not match the edge list")
    out_val = out_val[:len(out_col)].copy()
    if symmetrize:
        return WeightedGraph(n, out_ptr, out_col, out_val, out_ptr, out_col, out_val)
    in_ptr = np.empty(n + 1, dtype=np.int32)
    in_col = np.empty(max(1, len(out_col)), dtype=np.int32)
    in_val = np.empty(max(1, len(out_col)), dtype=np.float64)
    if _load().oracle_transpose_weighted(n, _p(out_ptr), _p(out_col), _p(out_val), _p(in_ptr), _p(in_col),
                                         _p(in_val)) != 0:
        raise MemoryError("oracle_transpose_weighted failed")
    return WeightedGraph(n, out_ptr, out_col, out_val, in_ptr, in_col[:len(out_col)].copy(),
                         in_val[:len(out_col)].copy())


def mxv_minplus(nrows: int, ncols: int, row_ptr, col, val, u, mask=None, transpose: bool = False,
                complement: bool = False, accum: bool = False, w_old=None) -> np.ndarray:
    """float64 result of the masked (min, +) matvec; +inf marks an absent entry."""
    nin = nrows if transpose else ncols
    nout = ncols if transpose else nrows
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.shape == (nin,)
    m = None if mask is None else to_dense(mask, nout)
    w = np.full(nout, np.inf) if w_old is None else np.ascontiguousarray(w_old, dtype=np.float64).copy()
    rc = _load().oracle_mxv_minplus(nrows, ncols, _p(_i32(row_ptr)), _p(_i32(col)),
                                    _p(np.ascontiguousarray(val, dtype=np.float64)), int(transpose), _p(u), _p(m),
                                    int(complement), int(accum), _p(w))
    if rc != 0:
        raise MemoryError("oracle_mxv_minplus failed")
    return w


def sssp(g: WeightedGraph, source: int):
    """Bellman-Ford distances (float32, +inf unreached) over out-edges, and the
    number of iterations that changed them."""
    d = np.empty(g.n, dtype=np.float32)
    val32 = np.ascontiguousarray(g.out_val, dtype=np.float32)
    it = _load().oracle_sssp_bf(g.n, _p(g.out_ptr), _p(g.out_col), _p(val32), int(source), _p(d))
    if it < 0:
        raise MemoryError("oracle_sssp_bf failed")
    return d, int(it)
