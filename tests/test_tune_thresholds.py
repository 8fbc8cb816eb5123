"""Host checks of gbx_tune_thresholds (no device work): the ratio-rule
thresholds derived from a BFS traced both ways reproduce the per-level best
schedule, judged by the oracle's statement of the Section 6.3 rule."""
import numpy as np
import pytest

import oracle
from paper_1804_03327_gb300 import build as gbx_build
from paper_1804_03327_gb300 import gbx


@pytest.fixture(scope="module")
def lib():
    gbx_build.build()
    return gbx.load()


def _trace(sizes, times, direction):
    """Level records of one BFS: sizes[L] = (|F_L|, |F_{L+1}|), times[L] in ns."""
    dt = np.dtype([(f, np.int64) for f in gbx.LEVEL_FIELDS])
    out = np.zeros(len(sizes), dtype=dt)
    for L, ((nf, nn), t) in enumerate(zip(sizes, times)):
        out[L]["direction"] = direction
        out[L]["level"] = L
        out[L]["nf"] = nf
        out[L]["n_new"] = nn
        out[L]["time_ns"] = t
    return out


# a hand-made 7-level BFS on n = 1000 vertices
SIZES = [(1, 10), (10, 200), (200, 600), (600, 150), (150, 30), (30, 5), (5, 0)]
PUSH_NS = [5, 10, 50, 90, 30, 8, 5]
PULL_NS = [100, 40, 20, 25, 20, 12, 10]


def test_worked_example(lib):
    push = _trace(SIZES, PUSH_NS, gbx.DIR_PUSH)
    pull = _trace(SIZES, PULL_NS, gbx.DIR_PULL)
    a, b, sched = gbx.tune_thresholds(push, pull, 1000)
    # per level the faster direction (level 0 pushes): push push pull pull pull push push
    assert sched == [gbx.DIR_PUSH, gbx.DIR_PUSH, gbx.DIR_PULL, gbx.DIR_PULL, gbx.DIR_PULL, gbx.DIR_PUSH,
                     gbx.DIR_PUSH]
    # alpha between r after level 0 (0.01, grew) and r after level 1 (0.2): their geometric mean;
    # beta between r after level 4 (0.03, the switch back) and r after level 3 (0.15, shrank too early)
    assert a == pytest.approx(np.sqrt(0.01 * 0.2), rel=1e-6)
    assert b == pytest.approx(np.sqrt(0.03 * 0.15), rel=1e-6)
    want = ["pull" if d == gbx.DIR_PULL else "push" for d in sched]
    assert oracle.direction_schedule(push, 1000, alpha=a, beta=b, heuristic="ratio") == want


def test_push_throughout_never_switches(lib):
    push = _trace(SIZES, [1] * 7, gbx.DIR_PUSH)
    pull = _trace(SIZES, [9] * 7, gbx.DIR_PULL)
    a, b, sched = gbx.tune_thresholds(push, pull, 1000)
    assert sched == [gbx.DIR_PUSH] * 7 and a >= 1e29 and b == 0.0
    assert oracle.direction_schedule(push, 1000, alpha=a, beta=b) == ["push"] * 7


def test_pull_to_the_end_keeps_beta_zero(lib):
    push = _trace(SIZES, [5, 10, 50, 90, 30, 8, 5], gbx.DIR_PUSH)
    pull = _trace(SIZES, [100, 40, 20, 25, 20, 1, 1], gbx.DIR_PULL)
    a, b, sched = gbx.tune_thresholds(push, pull, 1000)
    assert sched[2:] == [gbx.DIR_PULL] * 5 and b == 0.0
    assert oracle.direction_schedule(push, 1000, alpha=a, beta=b) == ["push", "push"] + ["pull"] * 5


def test_traces_of_different_runs_are_refused(lib):
    push = _trace(SIZES, PUSH_NS, gbx.DIR_PUSH)
    other = list(SIZES)
    other[3] = (600, 151)
    pull = _trace(other, PULL_NS, gbx.DIR_PULL)
    with pytest.raises(gbx.GbxError) as e:
        gbx.tune_thresholds(push, pull, 1000)
    assert e.value.status == gbx.ERR_INVALID_VALUE
