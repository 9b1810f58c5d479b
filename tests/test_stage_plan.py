"""CPU checks of the stage test of the two-stage schedules (Sec. III-A: rows
per level, row density, relative position), exported as jv_stage_plan: the
library's split equals a restatement written here, on synthetic level
widths and on the level sets the oracle computes for the stencil workloads;
bad level pointers are refused.  No GPU: the function is host code."""
import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.fixture(scope="module")
def jv():
    from paper_1812_06160_gb300 import build
    build.build()
    from paper_1812_06160_gb300 import _jv
    return _jv


def restated(level_ptr, dep_sum, min_rows, dens, pos):
    """upper[l] and the tail start, from the three rules as stated."""
    lp = np.asarray(level_ptr, dtype=np.int64)
    n = int(lp[-1])
    w = np.diff(lp)
    up = w >= (min_rows if min_rows > 0 else 1024)
    if dens > 0:
        mean = float(np.sum(dep_sum)) / n
        up &= np.asarray(dep_sum, dtype=np.float64) / w <= dens * mean
    if 0 < pos < 1:
        up &= lp[:-1] < pos * n
    tail = len(w)
    while tail > 0 and not up[tail - 1]:
        tail -= 1
    return up.astype(np.uint8), tail


def hybrid_launches(upper):
    """One launch per upper-stage level, one per maximal run of the others."""
    runs = int(np.sum((upper[1:] == 0) & (upper[:-1] == 1))) + int(len(upper) > 0 and upper[0] == 0)
    return int(upper.sum()) + runs


@pytest.mark.parametrize("seed", range(6))
def test_random_widths_match_restatement(jv, seed):
    rng = np.random.default_rng(seed)
    nlev = int(rng.integers(1, 400))
    w = rng.integers(1, 3000, nlev)
    lp = np.concatenate([[0], np.cumsum(w)]).astype(np.int32)
    dep = rng.integers(0, 30, nlev) * w
    for min_rows, dens, pos in [(0, 0, 0), (1, 0, 0), (500, 0, 0), (1500, 1.0, 0), (200, 0, 0.6),
                                (100, 0.8, 0.3), (10 ** 9, 0, 0)]:
        up, tail = jv.jv_stage_plan(lp, dep if dens > 0 else None, min_rows, dens, pos)
        want_up, want_tail = restated(lp, dep, min_rows, dens, pos)
        assert np.array_equal(up, want_up) and tail == want_tail, (min_rows, dens, pos)
        if min_rows == 10 ** 9:
            assert tail == 0 and hybrid_launches(up) == 1          # one sync-free launch
        if min_rows == 1 and dens == 0 and pos == 0:
            assert tail == nlev and hybrid_launches(up) == nlev    # every level on its own


def test_thin_level_between_wide_ones_stays_in_place(jv):
    # Fig. 3: a narrow level between wide ones is second-stage material but
    # not part of the tail; the hybrid schedule runs it as a sync-free run of
    # its own between two per-level launches
    lp = np.cumsum([0, 2000, 5, 2000, 3, 2]).astype(np.int32)
    up, tail = jv.jv_stage_plan(lp)
    assert list(up) == [1, 0, 1, 0, 0] and tail == 3
    assert hybrid_launches(up) == 4


@pytest.mark.parametrize("name,rp_ci", [("lap5_64", lambda: W.lap5(64)[:2]),
                                        ("lap7_24", lambda: W.lap7(24)[:2]),
                                        ("aniso5_96", lambda: W.aniso5(96)[:2])])
def test_stencil_level_sets(jv, name, rp_ci):
    rp, ci = rp_ci()
    lev, nlev, ptr, _ = O.level_sets(rp, ci)
    n = len(rp) - 1
    dep = np.bincount(lev, weights=np.diff(rp) - 1, minlength=nlev).astype(np.int64)
    for min_rows in (0, 16, 48):
        up, tail = jv.jv_stage_plan(ptr, dep, min_rows, 1.2, 0.9)
        want_up, want_tail = restated(ptr, dep, min_rows, 1.2, 0.9)
        assert np.array_equal(up, want_up) and tail == want_tail
    # with the default 1,024 rows every level of these small grids is thin
    up, tail = jv.jv_stage_plan(ptr)
    assert tail == 0 and not up.any()
    # the levels of a d-dimensional stencil widen then narrow: with a
    # threshold below the widest level the upper stage is one run in the middle
    up, tail = jv.jv_stage_plan(ptr, stage_min_rows=int(np.diff(ptr).max()) // 2)
    first, last = int(np.argmax(up)), int(len(up) - np.argmax(up[::-1]) - 1)
    assert up[first:last + 1].all() and tail == last + 1


def test_bad_inputs_refused(jv):
    with pytest.raises(jv.JvError) as e:
        jv.jv_stage_plan(np.array([0, 3, 3, 5]))           # an empty level
    assert e.value.status == jv.JV_ERR_ARG
    with pytest.raises(jv.JvError):
        jv.jv_stage_plan(np.array([1, 3, 5]))               # does not start at 0
    with pytest.raises(jv.JvError):
        jv.jv_stage_plan(np.array([0, 3, 5]), None, 0, 1.5)  # density without sums
    with pytest.raises(jv.JvError):
        jv.jv_stage_plan(np.array([0, 3, 5]), None, 0, 0, 1.5)  # position above 1
