"""Scheduling on the levels of lower(A + A^T) / upper(A + A^T) (Sec. III's
option): the levels are bit-exact with the oracle's levels of the
symmetrised pattern, the factor and the four solves are unchanged (bit-exact
with the oracle on A), and with the level-order permutation the factors of
P A P^T are A's, permuted, for nonsymmetric patterns too."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from jvutil import analyze, close, small_matrices

jv = pytest.importorskip("paper_1812_06160_gb300")
pytestmark = pytest.mark.gpu

CASES = small_matrices()
IDS = [c[0] for c in CASES]


def T(a):
    return torch.tensor(np.asarray(a), device="cuda")


def symmetrised(rp, ci):
    """CSR pattern of A + A^T (plain numpy)."""
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    r = np.concatenate([rows, ci]).astype(np.int64)
    c = np.concatenate([ci, rows]).astype(np.int64)
    key = np.unique(r * n + c)
    r, c = key // n, key % n
    srp = np.zeros(n + 1, dtype=np.int32)
    np.add.at(srp, r + 1, 1)
    return np.cumsum(srp).astype(np.int32), c.astype(np.int32)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_sym_levels_match_oracle(case):
    _, rp, ci, _ = case
    srp, sci = symmetrised(rp, ci)
    h = jv.jv_analyze(T(rp), T(ci), exact=True, sym_levels=True)
    for which, upper in (("L", False), ("U", True), ("Ut", False), ("Lt", True)):
        nlev, ptr, rows, lev = jv.jv_get_levels(h, which)
        olev, onlev, optr, orows = O.level_sets(srp, sci, upper=upper)
        assert nlev == onlev
        assert np.array_equal(lev.cpu().numpy(), olev)
        assert np.array_equal(rows.cpu().numpy(), orows)
        assert np.array_equal(ptr.cpu().numpy(), optr)
    # never fewer levels than lower(A) alone
    assert jv.jv_get_info(h)["nlev"][0] >= O.levels(rp, ci)[1]


@pytest.mark.parametrize("mode", ["level", "syncfree"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_sym_levels_results_unchanged(case, mode):
    _, rp, ci, v = case
    olu, st, _ = O.ilu0(rp, ci, v)
    if st != O.OK:
        pytest.skip("zero pivot case")
    n = len(rp) - 1
    h = analyze(jv, rp, ci, mode, sym_levels=True)
    lu = jv.jv_ilu0_factor(h, T(v))
    assert np.array_equal(lu.cpu().numpy(), olu)
    diag = O.diag_ptr(rp, ci)
    b = W.rhs(n, 1, seed=5)
    y = jv.jv_lsolve(h, lu, T(b))
    assert np.array_equal(y.cpu().numpy(), O.lsolve(rp, ci, diag, olu, b))
    z = jv.jv_usolve(h, lu, y)
    assert np.array_equal(z.cpu().numpy(), O.usolve(rp, ci, diag, olu, y.cpu().numpy()))
    gt = jv.jv_usolve_t(h, lu, T(b))
    assert np.array_equal(gt.cpu().numpy(), O.usolve_t(rp, ci, diag, olu, b))
    lt = jv.jv_lsolve_t(h, lu, gt)
    assert np.array_equal(lt.cpu().numpy(), O.lsolve_t(rp, ci, diag, olu, gt.cpu().numpy()))


@pytest.mark.parametrize("case", [c for c in CASES if c[0] in ("rand37", "rand600", "rand1500")],
                         ids=["rand37", "rand600", "rand1500"])
def test_sym_levels_reorder_keeps_factors_of_nonsymmetric_patterns(case):
    _, rp, ci, v = case
    n = len(rp) - 1
    srp, sci = symmetrised(rp, ci)
    assert not (np.array_equal(srp, rp) and np.array_equal(sci, ci))   # really nonsymmetric
    h = jv.jv_analyze(T(rp), T(ci), exact=True, reorder=True, sym_levels=True)
    _, _, _, perm = O.level_sets(srp, sci)
    assert np.array_equal(jv.jv_get_perm(h)[0].cpu().numpy(), perm)
    iperm, brp, bci, vmap = O.permute(rp, ci, perm)
    vb = jv.jv_permute_values(h, T(v))
    lu = jv.jv_ilu0_factor(h, vb)
    olu_b, _, _ = O.ilu0(brp, bci, v[vmap])
    assert np.array_equal(lu.cpu().numpy(), olu_b)
    # the level order keeps every entry on its side of the diagonal, so B's
    # factors are A's factors permuted (up to the order of the updates)
    olu_a, st, _ = O.ilu0(rp, ci, v)
    assert st == O.OK
    assert close(olu_b, olu_a[vmap], rel=1e-10)[0]
    b = W.rhs(n, 1, seed=9)
    z = jv.jv_usolve(h, lu, jv.jv_lsolve(h, lu, jv.jv_permute_vector(h, T(b))))
    back = jv.jv_permute_vector(h, z, inverse=True).cpu().numpy()
    diag = O.diag_ptr(rp, ci)
    want = O.usolve(rp, ci, diag, olu_a, O.lsolve(rp, ci, diag, olu_a, b))
    assert close(back, want, rel=1e-10)[0]


def test_sym_levels_band_rejected():
    rp, ci, _ = W.lap5(8)
    with pytest.raises(jv.JvError) as e:
        jv.jv_analyze(T(rp), T(ci), exact=True, sym_levels=True, band_rows=64)
    assert e.value.status == jv.JV_ERR_ARG


@pytest.mark.slow
def test_nonsymmetric_powerlaw_level_statistics():
    # the C4 recipe without symmetrisation (structurally nonsymmetric, 1e6
    # rows): levels of lower(A) and of lower(A + A^T) both bit-exact with the
    # oracle's, their statistics reported (Sec. V's table of nonsymmetric
    # matrices compares the two choices), and the factor the same either way
    c = W.config("c4n")
    rp, ci, v = c["rowptr"], c["colidx"], c["vals"]
    srp, sci = symmetrised(rp, ci)
    olu, st, _ = O.ilu0(rp, ci, v)
    assert st == O.OK
    stats = {}
    for sym, (prp, pci) in ((False, (rp, ci)), (True, (srp, sci))):
        h = jv.jv_analyze(T(rp), T(ci), sym_levels=sym)
        for which, upper in (("L", False), ("U", True)):
            nlev, ptr, rows, lev = jv.jv_get_levels(h, which)
            olev, onlev, optr, orows = O.level_sets(prp, pci, upper=upper)
            assert nlev == onlev
            assert np.array_equal(ptr.cpu().numpy(), optr)
            assert np.array_equal(rows.cpu().numpy(), orows)
            w = np.diff(optr)
            stats[("lower(A+A^T)" if sym else "lower(A)", which)] = (
                onlev, int(w.min()), int(w.max()), float(np.median(w)))
        lu = jv.jv_ilu0_factor(h, T(v)).cpu().numpy()
        ok, err = close(lu, olu)
        assert ok, (sym, err)
    for k, (nl, mn, mx, med) in stats.items():
        print(f"{k[0]:>13} {k[1]}: {nl} levels, rows per level min {mn} max {mx} median {med:.0f}")
    assert stats[("lower(A+A^T)", "L")][0] >= stats[("lower(A)", "L")][0]
