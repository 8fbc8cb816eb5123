"""Algorithmic bytes of a direction-optimized BFS, per level, from level counts.

These are the bytes the method must move (int32 = 4 B), not what a kernel
happened to read, so that achieved bandwidth = bytes / time never credits
redundant traffic:

* push level (Eq 5): read each frontier entry and its two row offsets
  (12 |f|), the frontier's neighbour ids (4 nnz(m_f^+)), write the next
  frontier list (4 |new|), depth and parent of new vertices (8 |new|), and
  stream the visited bitmap once (M/8).
* pull level (Eq 4 with masking and early exit): scan the mask bitmap and the
  nonempty-row bitmap (2 M/8), read two offsets per unvisited row that has
  in-edges (8 |U_nz|), the in-neighbours examined up to the first hit
  (4 e_exam), test them against the visited bitmap (M/8 streamed once),
  write depth and parent of new vertices (8 |new|) and the next bitmap (M/8).
  Without early exit e_exam is the full in-degree sum of the rows computed;
  without masking every nonempty row is computed.
* once per BFS: initialise depth and parent (8 M).

The counts come from the level trace (``gbx.bfs_trace``), whose fields are
checked against the CPU oracle's trace by the parity tests.
"""
from __future__ import annotations

import numpy as np

PUSH, PULL = 1, 2


def level_bytes(rec, n: int, with_parent: bool = True) -> int:
    bm = (n + 7) // 8
    out_per_new = 8 if with_parent else 4
    if int(rec["direction"]) == PUSH:
        return 12 * int(rec["nf"]) + 4 * int(rec["mf"]) + 4 * int(rec["n_new"]) + out_per_new * int(rec["n_new"]) + bm
    return 2 * bm + 8 * int(rec["nu_nz"]) + 4 * int(rec["e_exam"]) + bm + out_per_new * int(rec["n_new"]) + bm


def bfs_bytes(trace: np.ndarray, n: int, with_parent: bool = True) -> int:
    """Algorithmic bytes of one BFS with the given per-level trace."""
    init = (8 if with_parent else 4) * n
    return init + sum(level_bytes(r, n, with_parent) for r in trace)


def reached_edges(trace: np.ndarray) -> int:
    """Undirected edges in the reached component of a symmetric graph:
    half the degree sum over every reached vertex (sum of mf over levels)."""
    return int(np.sum(trace["mf"])) // 2


def summary(trace: np.ndarray) -> dict:
    dirs = ["push" if int(d) == PUSH else "pull" for d in trace["direction"]]
    return {"levels": len(trace), "directions": dirs,
            "frontier": [int(x) for x in trace["nf"]],
            "pull_examined": [int(x) for x, d in zip(trace["e_exam"], dirs) if d == "pull"]}
