"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module draws raw inputs only (edge samples, vertex subsets, sources); it
holds none of the method's arithmetic.  The heavy loops are in ``gen.c``
(SplitMix64, counter-based), compiled on first use with gcc.

Recipes (the paper names graph classes but gives no generator parameters):

* ``rmat_edges``: RMAT with a, b, c, d = 0.57, 0.19, 0.19, 0.05 and
  ``edge_factor * 2**scale`` directed samples, then a seeded relabelling.
  Stand-in for the paper's Kronecker / RMAT datasets (Section 7, Table 3).
* ``grid_edges``: 4-neighbour W x H mesh, each undirected edge deleted with
  probability ``p_delete``.  Stand-in for the mesh-like datasets of Table 3.
* ``sources``: distinct seeded vertices of nonzero degree.
* ``vertex_set``: Bernoulli(density) vertex membership, for random frontier
  and mask vectors as in the Section 3.2 microbenchmark.
* small deterministic shapes (path, star, complete, tree, Erdos-Renyi) for
  the oracle pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libsynth.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, u64, f64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
            lib.synth_draw.restype = u64
            lib.synth_draw.argtypes = [u64, u64]
            lib.synth_rmat.restype = ctypes.c_int
            lib.synth_rmat.argtypes = [i32, i32, f64, f64, f64, u64, i32, p, p]
            lib.synth_grid_edge_slots.restype = i64
            lib.synth_grid_edge_slots.argtypes = [i32, i32]
            lib.synth_grid.restype = i64
            lib.synth_grid.argtypes = [i32, i32, f64, u64, p, p]
            lib.synth_sources.restype = i32
            lib.synth_sources.argtypes = [i32, i64, p, p, i32, u64, p]
            lib.synth_vertex_set.restype = ctypes.c_int
            lib.synth_vertex_set.argtypes = [i32, f64, u64, u64, p]
            lib.synth_permutation.restype = ctypes.c_int
            lib.synth_permutation.argtypes = [i32, u64, p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def draw(seed: int, i: int) -> int:
    """i-th output of the SplitMix64 stream started at state ``seed``."""
    return int(_load().synth_draw(seed & (2**64 - 1), i))


def rmat_edges(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               seed: int = 1, relabel: bool = True):
    """Directed RMAT samples ``(src, dst)`` as int32 arrays; n = 2**scale."""
    m = edge_factor << scale
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = _load().synth_rmat(scale, edge_factor, a, b, c, seed, 1 if relabel else 0, _ptr(src), _ptr(dst))
    if rc != 0:
        raise ValueError(f"synth_rmat failed ({rc})")
    return 1 << scale, src, dst


def grid_edges(width: int, height: int, p_delete: float = 0.01, seed: int = 1):
    """Undirected mesh edges (each once, src < dst); n = width * height."""
    lib = _load()
    slots = lib.synth_grid_edge_slots(width, height)
    src = np.empty(max(slots, 1), dtype=np.int32)
    dst = np.empty(max(slots, 1), dtype=np.int32)
    k = lib.synth_grid(width, height, p_delete, seed, _ptr(src), _ptr(dst))
    if k < 0:
        raise ValueError("synth_grid failed")
    return width * height, src[:k].copy(), dst[:k].copy()


def sources(n: int, src: np.ndarray, dst: np.ndarray, k: int, seed: int = 1) -> np.ndarray:
    """Up to k distinct seeded sources among vertices with a non-self-loop edge."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    out = np.empty(max(k, 1), dtype=np.int32)
    got = _load().synth_sources(n, len(src), _ptr(src), _ptr(dst), k, seed, _ptr(out))
    if got < 0:
        raise MemoryError("synth_sources failed")
    return out[:got].copy()


def vertex_set(n: int, density: float, seed: int = 1, stream: int = 0) -> np.ndarray:
    """Seeded Bernoulli(density) membership: uint8[n] of 0/1."""
    out = np.empty(max(n, 1), dtype=np.uint8)
    _load().synth_vertex_set(n, float(density), seed, stream, _ptr(out))
    return out[:n]


def permutation(n: int, seed: int = 1) -> np.ndarray:
    """The relabelling ``rmat_edges`` applies: perm[v] = new label of v."""
    out = np.empty(max(n, 1), dtype=np.int32)
    _load().synth_permutation(n, seed, _ptr(out))
    return out[:n]


# ---- small deterministic shapes -----------------------------------------------------------

def path_edges(n: int):
    v = np.arange(n - 1, dtype=np.int32)
    return n, v, v + 1


def star_edges(k: int):
    """Centre 0, leaves 1..k."""
    leaves = np.arange(1, k + 1, dtype=np.int32)
    return k + 1, np.zeros(k, dtype=np.int32), leaves


def complete_edges(n: int):
    i, j = np.triu_indices(n, 1)
    return n, i.astype(np.int32), j.astype(np.int32)


def tree_edges(n: int, seed: int = 1):
    """Random recursive tree: vertex v > 0 attaches to a seeded earlier vertex."""
    par = np.array([draw(seed, v) % v for v in range(1, n)], dtype=np.int64)
    return n, par.astype(np.int32), np.arange(1, n, dtype=np.int32)


def er_edges(n: int, p: float, seed: int = 1, directed: bool = False):
    """Erdos-Renyi G(n, p) samples (ordered pairs if directed, else i < j)."""
    s = draw(seed, 12345)
    src, dst = [], []
    for i in range(n):
        for j in range(n):
            if i == j or (not directed and j <= i):
                continue
            if (draw(s, i * n + j) >> 11) * (1.0 / 9007199254740992.0) < p:
                src.append(i)
                dst.append(j)
    return n, np.array(src, dtype=np.int32), np.array(dst, dtype=np.int32)
