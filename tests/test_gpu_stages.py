"""Two-stage schedules (Sec. III-A, Fig. 2; Sec. III-B, Fig. 8) on the GPU.

Hybrid: the launch plan follows the stage test (rows per level, row density,
relative position) worked out here from the oracle's level sets, and the
factor and all solves stay bit-exact with the oracle.  Even-Rows corner: the
factor of the level-ordered matrix B = P A P^T is bit-exact with the oracle's
ILU(0) (and MILU(0)) of B in FP64 and FP32, under every upper-stage mode, on
the parity cases and at full size; a zero pivot inside the corner is reported
on its row; a tail that is not the last rows is refused."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from jvutil import small_matrices

jv = pytest.importorskip("paper_1812_06160_gb300")
pytestmark = pytest.mark.gpu

CASES = small_matrices()
IDS = [c[0] for c in CASES]


def T(a):
    return torch.tensor(np.asarray(a), device="cuda")


def dep_counts(rp, ci):
    """Dependencies of every row / column in the four structures L, U, Ut, Lt."""
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    lo, up = ci < rows, ci > rows
    return {"L": np.bincount(rows[lo], minlength=n), "U": np.bincount(rows[up], minlength=n),
            "Ut": np.bincount(ci[up], minlength=n), "Lt": np.bincount(ci[lo], minlength=n)}


def level_sets(rp, ci, which):
    if which in ("L", "U"):
        return O.level_sets(rp, ci, upper=(which == "U"))
    return O.transposed_level_sets(rp, ci, which)


def stage_plan(ptr, lev, dep, n, min_rows, dens, pos):
    """(launches of the hybrid schedule, first level of the second-stage tail)."""
    w = np.diff(ptr)
    up = w >= min_rows
    if dens > 0:
        mean = dep.sum() / n
        lsum = np.bincount(lev, weights=dep, minlength=len(w))
        up &= lsum / np.maximum(w, 1) <= dens * mean
    if 0 < pos < 1:
        up &= ptr[:-1] < pos * n
    runs = int(np.sum(~up[:1])) + int(np.sum(~up[1:] & up[:-1]))
    tail = len(w)
    while tail > 0 and not up[tail - 1]:
        tail -= 1
    return int(up.sum()) + runs, tail


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_hybrid_launch_plan_follows_stage_test(case):
    _, rp, ci, _ = case
    n = len(rp) - 1
    deps = dep_counts(rp, ci)
    for min_rows, dens, pos in [(1, 0, 0), (10 ** 9, 0, 0), (16, 0, 0), (8, 1.5, 0),
                                (4, 0, 0.5), (2, 1.0, 0.7)]:
        h = jv.jv_analyze(T(rp), T(ci), exact=True, mode="hybrid", stage_min_rows=min_rows,
                          stage_max_density=dens, stage_position=pos)
        info = jv.jv_get_info(h)
        for k, which in enumerate(("L", "U", "Ut", "Lt")):
            lev, nlev, ptr, _ = level_sets(rp, ci, which)
            want, _ = stage_plan(ptr, lev, deps[which], n, min_rows, dens, pos)
            assert info["hybrid_launches"][k] == want, (which, min_rows, dens, pos)
        if min_rows == 1 and dens == 0:
            assert info["hybrid_launches"] == info["nlev"]          # every level on its own
        if min_rows == 10 ** 9:
            assert info["hybrid_launches"] == [1, 1, 1, 1]           # one sync-free launch


@pytest.mark.parametrize("min_rows", [16, 3])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_hybrid_bit_exact(case, min_rows):
    _, rp, ci, v = case
    n = len(rp) - 1
    h = jv.jv_analyze(T(rp), T(ci), exact=True, mode="hybrid", stage_min_rows=min_rows)
    olu, st, bad = O.ilu0(rp, ci, v)
    if st != O.OK:
        with pytest.raises(jv.JvError) as e:
            jv.jv_ilu0_factor(h, T(v))
        assert e.value.status == jv.JV_ERR_ZERO_PIVOT and e.value.bad_row == bad
        return
    lu = jv.jv_ilu0_factor(h, T(v))
    assert np.array_equal(lu.cpu().numpy(), olu)
    o32, st32, _ = O.ilu0(rp, ci, v, dtype=np.float32)
    if st32 == O.OK:
        assert np.array_equal(jv.jv_ilu0_factor(h, T(v).float()).cpu().numpy(), o32)
    diag = O.diag_ptr(rp, ci)
    b = W.rhs(n, 1, seed=21)
    y = jv.jv_lsolve(h, lu, T(b))
    assert np.array_equal(y.cpu().numpy(), O.lsolve(rp, ci, diag, olu, b))
    z = jv.jv_usolve(h, lu, y)
    assert np.array_equal(z.cpu().numpy(), O.usolve(rp, ci, diag, olu, y.cpu().numpy()))
    gt = jv.jv_usolve_t(h, lu, T(b))
    assert np.array_equal(gt.cpu().numpy(), O.usolve_t(rp, ci, diag, olu, b))
    lt = jv.jv_lsolve_t(h, lu, gt)
    assert np.array_equal(lt.cpu().numpy(), O.lsolve_t(rp, ci, diag, olu, gt.cpu().numpy()))
    B3 = W.rhs(n, 3, seed=22)
    Y3 = jv.jv_lsolve(h, lu, T(B3))
    assert np.array_equal(Y3.cpu().numpy(), O.lsolve(rp, ci, diag, olu, B3))


def reordered(rp, ci, v):
    _, _, _, perm = O.level_sets(rp, ci)
    _, brp, bci, vmap = O.permute(rp, ci, perm)
    return brp, bci, v[vmap]


def check_corner_info(h, brp, bci, min_rows):
    info = jv.jv_get_info(h)
    n = len(brp) - 1
    lev, nlev, ptr, _ = O.level_sets(brp, bci)
    _, tail = stage_plan(ptr, lev, dep_counts(brp, bci)["L"], n, min_rows, 0, 0)
    for t in (0, 1):
        R, nl = info["corner_rows"][t], info["corner_levels"][t]
        assert 0 <= nl <= nlev - tail
        assert R == n - ptr[nlev - nl]
    return info


@pytest.mark.parametrize("mode", ["level", "syncfree", "hybrid"])
@pytest.mark.parametrize("min_rows", [0, 6])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_er_corner_bit_exact(case, min_rows, mode):
    _, rp, ci, v = case
    brp, bci, bv = reordered(rp, ci, v)
    h = jv.jv_analyze(T(rp), T(ci), exact=True, reorder=True, er_corner=True, mode=mode,
                      stage_min_rows=min_rows)
    info = check_corner_info(h, brp, bci, min_rows or 1024)
    assert info["corner_rows"][1] >= info["corner_rows"][0]
    if min_rows == 0 and case[0] != "powerlaw6000":
        assert info["corner_rows"][0] > 0          # every level thin: a corner fits
    vb = jv.jv_permute_values(h, T(v))
    assert np.array_equal(vb.cpu().numpy(), bv)
    olu, st, bad = O.ilu0(brp, bci, bv)
    if st != O.OK:
        with pytest.raises(jv.JvError) as e:
            jv.jv_ilu0_factor(h, vb)
        assert e.value.status == jv.JV_ERR_ZERO_PIVOT and e.value.bad_row == bad
        return
    assert np.array_equal(jv.jv_ilu0_factor(h, vb).cpu().numpy(), olu)
    o32, st32, bad32 = O.ilu0(brp, bci, bv, dtype=np.float32)
    if st32 == O.OK:
        assert np.array_equal(jv.jv_ilu0_factor(h, vb.float()).cpu().numpy(), o32)
        # FP64 values, FP32 factor: the cast is fused into the load
        assert np.array_equal(jv.jv_ilu0_factor(h, vb, lu_dtype=torch.float32).cpu().numpy(), o32)
    else:
        with pytest.raises(jv.JvError) as e:
            jv.jv_ilu0_factor(h, vb.float())
        assert e.value.bad_row == bad32


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_er_corner_milu_bit_exact(case):
    _, rp, ci, v = case
    brp, bci, bv = reordered(rp, ci, v)
    h = jv.jv_analyze(T(rp), T(ci), exact=True, reorder=True, er_corner=True, milu=True, stage_min_rows=6)
    olu, st, bad = O.ilu0(brp, bci, bv, milu=True)
    vb = jv.jv_permute_values(h, T(v))
    if st != O.OK:
        with pytest.raises(jv.JvError) as e:
            jv.jv_ilu0_factor(h, vb)
        assert e.value.status == jv.JV_ERR_ZERO_PIVOT and e.value.bad_row == bad
        return
    assert np.array_equal(jv.jv_ilu0_factor(h, vb).cpu().numpy(), olu)


def test_er_corner_zero_pivot_inside_corner():
    # an infinite diagonal on the corner's first row: its pivot is the first
    # non-finite one, and the rows after it inherit NaNs (the smallest
    # failing row is the one reported)
    rp, ci, v = W.lap5(12)
    brp, bci, bv = reordered(rp, ci, v)
    n = len(brp) - 1
    h = jv.jv_analyze(T(rp), T(ci), exact=True, reorder=True, er_corner=True, stage_min_rows=6)
    R = jv.jv_get_info(h)["corner_rows"][0]
    assert 1 < R < n
    r0 = n - R
    dpos = brp[r0] + int(np.nonzero(bci[brp[r0]:brp[r0 + 1]] == r0)[0][0])
    v2 = bv.copy()
    v2[dpos] = np.inf
    _, st2, bad2 = O.ilu0(brp, bci, v2)
    assert st2 == O.ERR_ZERO_PIVOT and bad2 == r0
    with pytest.raises(jv.JvError) as e:
        jv.jv_ilu0_factor(h, T(v2))
    assert e.value.status == jv.JV_ERR_ZERO_PIVOT and e.value.bad_row == r0


def test_er_corner_needs_trailing_rows():
    # natural order, levels i + j of an 8 x 8 grid: with at least 4 rows per
    # upper-stage level the tail is levels 12..14, rows {47, 54, 55, 61, 62,
    # 63} -- not the last six rows
    rp, ci, v = W.lap5(8)
    with pytest.raises(jv.JvError) as e:
        jv.jv_analyze(T(rp), T(ci), exact=True, er_corner=True, stage_min_rows=4)
    assert e.value.status == jv.JV_ERR_ARG
    # a corner that is the whole matrix fits any order (no row above it)
    h = jv.jv_analyze(T(rp), T(ci), exact=True, er_corner=True)
    assert jv.jv_get_info(h)["corner_rows"] == [64, 64]
    olu, _, _ = O.ilu0(rp, ci, v)
    assert np.array_equal(jv.jv_ilu0_factor(h, T(v)).cpu().numpy(), olu)
    with pytest.raises(jv.JvError) as e:
        jv.jv_analyze(T(rp), T(ci), exact=True, reorder=True, er_corner=True, band_rows=64)
    assert e.value.status == jv.JV_ERR_ARG
    # a tridiagonal matrix is level-ordered as it stands: no reordering needed
    rp, ci, v = W.stencil((50, 1, 1), [(-1, 0, 0), (1, 0, 0)], [-1.0, -1.0], 4.0)
    h = jv.jv_analyze(T(rp), T(ci), exact=True, er_corner=True)
    assert jv.jv_get_info(h)["corner_rows"][0] == 50
    olu, _, _ = O.ilu0(rp, ci, v)
    assert np.array_equal(jv.jv_ilu0_factor(h, T(v)).cpu().numpy(), olu)


@pytest.mark.parametrize("cfg,dtypes", [("c1", (np.float64, np.float32)),
                                        ("c2", (np.float64, np.float32)),
                                        ("c5", (np.float32,))])
def test_er_corner_full_size(cfg, dtypes):
    c = W.config(cfg)
    rp, ci, v = c["rowptr"], c["colidx"], c["vals"]
    brp, bci, bv = reordered(rp, ci, v)
    h = jv.jv_analyze(T(rp), T(ci), exact=True, reorder=True, er_corner=True)
    info = check_corner_info(h, brp, bci, 1024)
    vb = jv.jv_permute_values(h, T(v))
    for dt in dtypes:
        assert info["corner_rows"][0 if dt == np.float64 else 1] > 0
        olu, st, _ = O.ilu0(brp, bci, bv, dtype=dt)
        assert st == O.OK
        got = jv.jv_ilu0_factor(h, vb if dt == np.float64 else vb.float())
        assert np.array_equal(got.cpu().numpy(), olu)


def test_hybrid_full_size_c2():
    c = W.config("c2")
    rp, ci, v = c["rowptr"], c["colidx"], c["vals"]
    n = len(rp) - 1
    h = jv.jv_analyze(T(rp), T(ci), exact=True, mode="hybrid")
    info = jv.jv_get_info(h)
    assert 1 < info["hybrid_launches"][0] < info["nlev"][0]
    olu, st, _ = O.ilu0(rp, ci, v)
    lu = jv.jv_ilu0_factor(h, T(v))
    assert np.array_equal(lu.cpu().numpy(), olu)
    diag = O.diag_ptr(rp, ci)
    b = c["b"]
    y = jv.jv_lsolve(h, lu, T(b))
    assert np.array_equal(y.cpu().numpy(), O.lsolve(rp, ci, diag, olu, b))
    z = jv.jv_usolve(h, lu, y)
    assert np.array_equal(z.cpu().numpy(), O.usolve(rp, ci, diag, olu, y.cpu().numpy()))


SOLVES = (("L", 0, "jv_lsolve", O.lsolve), ("U", 1, "jv_usolve", O.usolve),
          ("Ut", 2, "jv_usolve_t", O.usolve_t), ("Lt", 3, "jv_lsolve_t", O.lsolve_t))


def check_solve_corners(rp, ci, v, brp, bci, olu, mode, min_rows, seed):
    """The four one-column solves with corners: FP64 bit-exact with the
    oracle; FP32 (every mix of b and x precisions) bit-exact with the
    sync-free path without corners."""
    n = len(brp) - 1
    h = jv.jv_analyze(T(rp), T(ci), exact=True, reorder=True, er_corner=True, mode=mode,
                      stage_min_rows=min_rows)
    h0 = jv.jv_analyze(T(rp), T(ci), exact=True, reorder=True)
    info = jv.jv_get_info(h)
    diag = O.diag_ptr(brp, bci)
    b = W.rhs(n, 1, seed=seed)
    lu = T(olu)
    for _, k, fn, ofn in SOLVES:
        got = getattr(jv, fn)(h, lu, T(b)).cpu().numpy()
        assert np.array_equal(got, ofn(brp, bci, diag, olu, b)), (fn, info["solve_corner_rows"][k])
    lu32 = lu.float()
    for bt in (torch.float32, torch.float64):
        for xt in (torch.float32, torch.float64):
            bb = T(b).to(bt)
            for _, _, fn, _ in SOLVES:
                x1 = getattr(jv, fn)(h, lu32, bb, x_dtype=xt)
                x0 = getattr(jv, fn)(h0, lu32, bb, x_dtype=xt)
                assert x1.dtype == xt and torch.equal(x1, x0), (fn, bt, xt)
    # several columns: no corner, the plain schedule
    B3 = W.rhs(n, 3, seed=seed + 1)
    assert np.array_equal(jv.jv_usolve(h, lu, T(B3)).cpu().numpy(),
                          O.usolve(brp, bci, diag, olu, B3))
    return info


@pytest.mark.parametrize("mode", ["syncfree", "level", "hybrid"])
@pytest.mark.parametrize("min_rows", [0, 6])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_er_solve_corners_bit_exact(case, min_rows, mode):
    name, rp, ci, v = case
    brp, bci, bv = reordered(rp, ci, v)
    olu, st, _ = O.ilu0(brp, bci, bv)
    if st != O.OK:
        pytest.skip("zero pivot case")
    info = check_solve_corners(rp, ci, v, brp, bci, olu, mode, min_rows, seed=31)
    if min_rows == 0 and name not in ("powerlaw6000", "rand1"):
        assert info["solve_corner_rows"][0][0] > 0 and info["solve_corner_rows"][0][1] > 0


@pytest.mark.parametrize("cfg", ["c1", "c5"])
def test_er_solve_corners_full_size(cfg):
    c = W.config(cfg)
    rp, ci, v = c["rowptr"], c["colidx"], c["vals"]
    brp, bci, bv = reordered(rp, ci, v)
    olu, st, _ = O.ilu0(brp, bci, bv)
    assert st == O.OK
    info = check_solve_corners(rp, ci, v, brp, bci, olu, "syncfree", 0, seed=41)
    # symmetric patterns in level order: every structure's tail is an end of the order
    assert all(r[0] > 0 and r[1] >= r[0] for r in info["solve_corner_rows"])
    if cfg == "c1":                                   # the whole FP32 solve fits one CTA
        assert all(r[1] == len(rp) - 1 for r in info["solve_corner_rows"])
