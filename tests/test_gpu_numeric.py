"""GPU factor / solves / spmv / masked outer product vs the oracle.

Bars: the FP64 and FP32 factors, the FP64 solves (all four), spmv and the
masked outer product are bit-exact -- the kernels perform the oracle's
operations in the oracle's order, each rounded separately, and only the
loads run in parallel; FP32 solves are reported against the FP64 oracle and
bounded."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from jvutil import SCHEDULES, analyze, close, close_scaled, max_rel, small_matrices, solve_scale

jv = pytest.importorskip("paper_1812_06160_gb300")
pytestmark = pytest.mark.gpu

CASES = small_matrices()
IDS = [c[0] for c in CASES]
MODES = list(SCHEDULES)


def T(a):
    return torch.tensor(np.asarray(a), device="cuda")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_factor_fp64_bit_exact(case, mode):
    _, rp, ci, v = case
    h = analyze(jv, rp, ci, mode)
    lu = jv.jv_ilu0_factor(h, T(v))
    olu, st, _ = O.ilu0(rp, ci, v)
    assert st == 0
    assert np.array_equal(lu.cpu().numpy(), olu)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_factor_fp64_reciprocal_pivots_within_1e12(case, mode):
    # the default FP64 factor multiplies by each pivot's reciprocal: every
    # entry within 1e-12 relative of the oracle's divisions
    _, rp, ci, v = case
    h = analyze(jv, rp, ci, mode, exact=False)
    lu = jv.jv_ilu0_factor(h, T(v)).cpu().numpy()
    olu, st, _ = O.ilu0(rp, ci, v)
    assert st == 0
    ok, err = close(lu, olu)
    assert ok, err


@pytest.mark.parametrize("mode", MODES)
def test_factor_nine_point_rows(mode):
    # a 9-point stencil: nearly every row needs 17..32 words (the wide
    # one-lane slot, no one-warp rows), while the band schedule's one-thread
    # rows over 16 words work in the global scratch area, which must exist
    m = 30
    offs = [(dx, dy, 0) for dx in (-1, 0, 1) for dy in (-1, 0, 1) if (dx, dy) != (0, 0)]
    rp, ci, v = W.stencil((m, m, 1), offs, [-0.1] * 8, 1.0)
    h = analyze(jv, rp, ci, mode)
    olu, st, _ = O.ilu0(rp, ci, v)
    assert st == 0
    assert np.array_equal(jv.jv_ilu0_factor(h, T(v)).cpu().numpy(), olu)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nrhs", [1, 3, 33])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_solves_fp64_default_mode(case, nrhs, mode):
    # default mode: the U and U^T solves form s / u_ii from 1/u_ii and one
    # correction step, which gives the division's own result, so a structure
    # of short rows solves bit-exactly; a structure with rows above long_row
    # sums those rows by lanes and a fixed tree (one column): within 1e-12 of
    # the magnitude of each entry's terms (jvutil.solve_scale)
    _, rp, ci, v = case
    n = len(rp) - 1
    h = analyze(jv, rp, ci, mode, exact=False)
    nlong = jv.jv_get_info(h)["nlong"]
    olu, _, _ = O.ilu0(rp, ci, v)
    diag = O.diag_ptr(rp, ci)
    b = W.rhs(n, nrhs, seed=17 + nrhs)
    lu, bt = T(olu), T(b)
    for k, (name, ofn) in enumerate((("jv_lsolve", O.lsolve), ("jv_usolve", O.usolve),
                                     ("jv_usolve_t", O.usolve_t), ("jv_lsolve_t", O.lsolve_t))):
        x = getattr(jv, name)(h, lu, bt).cpu().numpy()
        want = ofn(rp, ci, diag, olu, b)
        if nlong[k] == 0 or nrhs > 1:
            assert np.array_equal(x, want), (name, close(x, want)[1])
        else:
            ok, err = close_scaled(x, want, solve_scale(ofn, rp, ci, diag, olu, b))
            assert ok, (name, err)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_factor_fp32_bit_exact_to_fp32_twin(case, mode):
    _, rp, ci, v = case
    h = analyze(jv, rp, ci, mode)
    olu32, st, _ = O.ilu0(rp, ci, v.astype(np.float32), dtype=np.float32)
    lu = jv.jv_ilu0_factor(h, T(v), lu_dtype=torch.float32)        # fused down-cast
    assert np.array_equal(lu.cpu().numpy(), olu32)
    inplace = T(v.astype(np.float32))
    jv.jv_ilu0_factor(h, inplace, lu=inplace)                        # in place
    assert np.array_equal(inplace.cpu().numpy(), olu32)
    olu64, _, _ = O.ilu0(rp, ci, v)
    if len(v) > 1:
        assert max_rel(olu32, olu64) < 1e-4     # reported FP32-vs-FP64 error, bounded


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nrhs", [1, 3, 33])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_solves_fp64(case, nrhs, mode):
    _, rp, ci, v = case
    n = len(rp) - 1
    h = analyze(jv, rp, ci, mode)
    olu, _, _ = O.ilu0(rp, ci, v)
    diag = O.diag_ptr(rp, ci)
    b = W.rhs(n, nrhs, seed=7 + nrhs)
    lu = T(olu)
    bt = T(b)
    for name, ofn in (("jv_lsolve", O.lsolve), ("jv_usolve", O.usolve),
                      ("jv_lsolve_t", O.lsolve_t), ("jv_usolve_t", O.usolve_t)):
        x = getattr(jv, name)(h, lu, bt).cpu().numpy()
        want = ofn(rp, ci, diag, olu, b)
        assert np.array_equal(x, want), (name, close(x, want)[1])


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_solves_fp32_and_mixed(case, mode):
    _, rp, ci, v = case
    n = len(rp) - 1
    h = analyze(jv, rp, ci, mode)
    olu32, _, _ = O.ilu0(rp, ci, v.astype(np.float32), dtype=np.float32)
    diag = O.diag_ptr(rp, ci)
    lu64 = olu32.astype(np.float64)
    b = W.rhs(n, 1, seed=5)
    lu = T(olu32)
    want_y = O.lsolve(rp, ci, diag, lu64, b)
    want_z = O.usolve(rp, ci, diag, lu64, want_y)
    y32 = jv.jv_lsolve(h, lu, T(b.astype(np.float32)))
    assert y32.dtype == torch.float32 and max_rel(y32.cpu().numpy(), want_y) < 1e-4
    ym = jv.jv_lsolve(h, lu, T(b))                                   # FP64 in, FP32 out
    assert ym.dtype == torch.float32 and max_rel(ym.cpu().numpy(), want_y) < 1e-4
    zm = jv.jv_usolve(h, lu, ym, x_dtype=torch.float64)              # FP32 in, FP64 out
    assert zm.dtype == torch.float64 and max_rel(zm.cpu().numpy(), want_z) < 1e-4
    b3 = W.rhs(n, 5, seed=6)
    x3 = jv.jv_usolve_t(h, lu, T(b3.astype(np.float32))).cpu().numpy()
    assert max_rel(x3, O.usolve_t(rp, ci, diag, lu64, b3)) < 1e-4


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_spmv(case):
    _, rp, ci, v = case
    n = len(rp) - 1
    h = jv.jv_analyze(T(rp), T(ci), exact=True)
    x = W.rhs(n, 1, seed=3)
    y0 = W.rhs(n, 1, seed=4)
    scale = O.spmv(rp, ci, np.abs(v), np.abs(x)) + np.abs(y0)
    for alpha, beta in ((1.0, 0.0), (-2.0, 0.5), (-1.0, 1.0)):
        y = jv.jv_spmv(h, T(v), T(x), T(y0), alpha=alpha, beta=beta).cpu().numpy()
        want = O.spmv(rp, ci, v, x, y0, alpha=alpha, beta=beta)
        assert np.array_equal(y, want)
    y32 = jv.jv_spmv(h, T(v.astype(np.float32)), T(x.astype(np.float32))).cpu().numpy()
    assert np.all(np.abs(y32 - O.spmv(rp, ci, v, x)) <= 1e-5 * (scale + 1e-30))


@pytest.mark.parametrize("long_row", [0, 8])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_spmv_default_mode(case, long_row):
    # default mode: rows longer than spmv_long_row (128, or 8 here to reach
    # the warp path on small matrices) sum by lanes and a fixed tree, within
    # 1e-12 of the magnitude of their terms and identical run to run; the
    # other rows keep the serial order bit for bit
    _, rp, ci, v = case
    n = len(rp) - 1
    h = jv.jv_analyze(T(rp), T(ci), spmv_long_row=long_row)
    thr = long_row or 128
    lens = np.diff(rp)
    assert jv.jv_get_info(h)["spmv_wide_rows"] == int((lens > thr).sum())
    short = lens <= thr
    x = W.rhs(n, 1, seed=3)
    y0 = W.rhs(n, 1, seed=4)
    for alpha, beta in ((1.0, 0.0), (-2.0, 0.5), (-1.0, 1.0)):
        y = jv.jv_spmv(h, T(v), T(x), T(y0), alpha=alpha, beta=beta).cpu().numpy()
        y2 = jv.jv_spmv(h, T(v), T(x), T(y0), alpha=alpha, beta=beta).cpu().numpy()
        assert np.array_equal(y, y2)
        want = O.spmv(rp, ci, v, x, y0, alpha=alpha, beta=beta)
        assert np.array_equal(y[short], want[short])
        scale = abs(alpha) * O.spmv(rp, ci, np.abs(v), np.abs(x)) + abs(beta) * np.abs(y0)
        ok, err = close_scaled(y, want, scale)
        assert ok, err
        # values 8 bytes off a 16-byte boundary take the scalar-load kernel:
        # the same bits
        vu = T(np.concatenate([[0.0], v]))[1:]
        yu = jv.jv_spmv(h, vu, T(x), T(y0), alpha=alpha, beta=beta).cpu().numpy()
        assert np.array_equal(yu, y)
    x32 = x.astype(np.float32)
    y32 = jv.jv_spmv(h, T(v.astype(np.float32)), T(x32)).cpu().numpy()
    want32 = O.spmv(rp, ci, v.astype(np.float32).astype(np.float64), x32.astype(np.float64))
    assert np.all(np.abs(y32 - want32) <= 1e-5 * (O.spmv(rp, ci, np.abs(v), np.abs(x)) + 1e-30))


OUTER_CASES = [c for c in CASES if c[0] in ("rand37", "rand250", "rand600", "rand1500", "lap5_33",
                                            "aniso5_41", "powerlaw6000", "band20_800")]


@pytest.mark.parametrize("nrhs", [1, 7, 32])
@pytest.mark.parametrize("case", OUTER_CASES, ids=[c[0] for c in OUTER_CASES])
def test_masked_outer(case, nrhs):
    # rows of at most 64 entries take the thread-per-row kernel, longer
    # ones (powerlaw6000) the warp-per-row kernel
    _, rp, ci, _ = case
    n = len(rp) - 1
    h = jv.jv_analyze(T(rp), T(ci), exact=True)
    diag = O.diag_ptr(rp, ci)
    a, b = W.rhs(n, nrhs, seed=1), W.rhs(n, nrhs, seed=2)
    for which in (0, 1):
        g = jv.jv_masked_outer(h, which, T(a), T(b), alpha=-1.0).cpu().numpy()
        want = O.masked_outer(rp, ci, diag, which, a, b, alpha=-1.0)
        assert np.array_equal(g, want)
        # FP32, and the 16-byte vector loads (aligned rows of 32 columns)
        # against the scalar loads of the same data read from a copy that is
        # 4 bytes off the 16-byte boundary
        a32, b32 = T(a).float(), T(b).float()
        g32 = jv.jv_masked_outer(h, which, a32, b32, alpha=-1.0)
        buf_a = torch.empty(a32.numel() + 1, dtype=torch.float32, device="cuda")
        buf_b = torch.empty(b32.numel() + 1, dtype=torch.float32, device="cuda")
        ua, ub = buf_a[1:].view_as(a32), buf_b[1:].view_as(b32)
        ua.copy_(a32)
        ub.copy_(b32)
        assert ua.data_ptr() % 16 != 0
        assert torch.equal(jv.jv_masked_outer(h, which, ua, ub, alpha=-1.0), g32)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_reordered_factor_and_solve(case):
    """B = P A P^T: the factor of B is bit-exact to the oracle's factor of B;
    solving in B's order and permuting back matches the natural-order solve
    (the level order keeps lower(A) lower on these symmetric-pattern cases,
    up to summation order)."""
    _, rp, ci, v = case
    n = len(rp) - 1
    h = jv.jv_analyze(T(rp), T(ci), exact=True, reorder=True)
    _, _, _, perm = O.level_sets(rp, ci)
    iperm, brp, bci, vmap = O.permute(rp, ci, perm)
    vb = jv.jv_permute_values(h, T(v))
    assert np.array_equal(vb.cpu().numpy(), v[vmap])
    lu = jv.jv_ilu0_factor(h, vb)
    olu, _, _ = O.ilu0(brp, bci, v[vmap])
    assert np.array_equal(lu.cpu().numpy(), olu)
    b = W.rhs(n, 2, seed=9)
    bb = jv.jv_permute_vector(h, T(b))
    assert np.array_equal(bb.cpu().numpy(), b[perm])
    z = jv.jv_usolve(h, lu, jv.jv_lsolve(h, lu, bb))
    back = jv.jv_permute_vector(h, z, inverse=True).cpu().numpy()
    bdiag = O.diag_ptr(brp, bci)
    want_b = O.usolve(brp, bci, bdiag, olu, O.lsolve(brp, bci, bdiag, olu, b[perm]))
    assert np.array_equal(z.cpu().numpy(), want_b)
    sym = np.array_equal(O.transpose(rp, ci)[0], rp) and np.array_equal(O.transpose(rp, ci)[1], ci)
    if sym:
        olu_a, _, _ = O.ilu0(rp, ci, v)
        diag = O.diag_ptr(rp, ci)
        want = O.usolve(rp, ci, diag, olu_a, O.lsolve(rp, ci, diag, olu_a, b))
        assert close(back, want, rel=1e-10)[0]
