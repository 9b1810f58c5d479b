"""GPU analysis vs the oracle, bit-exact: diag_ptr, CSC, the four level
structures (level of every row, level pointers, rows grouped by level) and
the level-order reordering, on small cases spanning several tiles and ragged
tails, long chains and degenerate shapes."""
import numpy as np
import pytest
import torch

import oracle as O
from jvutil import small_matrices

jv = pytest.importorskip("paper_1812_06160_gb300")
pytestmark = pytest.mark.gpu

CASES = small_matrices()
IDS = [c[0] for c in CASES]


def T(a):
    return torch.tensor(np.asarray(a), device="cuda")


def _oracle_levels(rp, ci):
    return {
        "L": O.level_sets(rp, ci, upper=False),
        "U": O.level_sets(rp, ci, upper=True),
        "Ut": O.transposed_level_sets(rp, ci, "Ut"),
        "Lt": O.transposed_level_sets(rp, ci, "Lt"),
    }


def _check_structures(h, rp, ci):
    diag = O.diag_ptr(rp, ci)
    grp, gci, gdiag = (t.cpu().numpy() for t in jv.jv_get_pattern(h))
    assert np.array_equal(grp, rp) and np.array_equal(gci, ci)
    assert np.array_equal(gdiag, diag)
    info = jv.jv_get_info(h)
    assert info["nnz_lower"] == int((diag - rp[:-1]).sum())
    assert info["nnz_upper"] == len(ci) - len(diag) - info["nnz_lower"]
    for which, (lev, nlev, ptr, rows) in _oracle_levels(rp, ci).items():
        gn, gptr, grows, glev = jv.jv_get_levels(h, which)
        assert gn == nlev, which
        assert np.array_equal(glev.cpu().numpy(), lev), which
        assert np.array_equal(gptr.cpu().numpy(), ptr), which
        assert np.array_equal(grows.cpu().numpy(), rows), which
    colptr, rowidx, c2c = O.transpose(rp, ci)
    gcp, gri, gc2c, gcd = (t.cpu().numpy() for t in jv.jv_get_csc(h))
    assert np.array_equal(gcp, colptr) and np.array_equal(gri, rowidx)
    assert np.array_equal(gc2c, c2c)
    n = len(rp) - 1
    for j in range(0, n, max(1, n // 50)):
        seg = rowidx[colptr[j]:colptr[j + 1]]
        assert gcd[j] == colptr[j] + int(np.searchsorted(seg, j))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_analysis_bit_exact(case):
    _, rp, ci, _ = case
    h = jv.jv_analyze(T(rp), T(ci))
    _check_structures(h, rp, ci)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_reorder_bit_exact(case):
    _, rp, ci, _ = case
    h = jv.jv_analyze(T(rp), T(ci), reorder=True)
    _, _, _, perm = O.level_sets(rp, ci)
    iperm, brp, bci, vmap = O.permute(rp, ci, perm)
    gperm, giperm, gvmap = (t.cpu().numpy() for t in jv.jv_get_perm(h))
    assert np.array_equal(gperm, perm) and np.array_equal(giperm, iperm)
    assert np.array_equal(gvmap, vmap)
    _check_structures(h, brp, bci)


def test_analysis_is_deterministic():
    _, rp, ci, _ = CASES[-1]
    a = [jv.jv_get_levels(jv.jv_analyze(T(rp), T(ci)), "L")[2].cpu().numpy() for _ in range(3)]
    assert all(np.array_equal(a[0], x) for x in a[1:])


@pytest.mark.parametrize("case", ["unsorted", "duplicate", "out_of_range", "negative", "no_diag",
                                  "bad_rowptr", "late_row"])
def test_pattern_errors_match_oracle(case):
    rp = np.array([0, 2, 4, 6], dtype=np.int32)
    ci = np.array([0, 1, 0, 1, 1, 2], dtype=np.int32)
    if case == "unsorted":
        ci = np.array([0, 1, 0, 1, 2, 1], dtype=np.int32)
    elif case == "duplicate":
        ci = np.array([0, 1, 0, 1, 2, 2], dtype=np.int32)
    elif case == "out_of_range":
        ci = np.array([0, 1, 0, 1, 2, 3], dtype=np.int32)
    elif case == "negative":
        ci = np.array([0, 1, -1, 1, 1, 2], dtype=np.int32)
    elif case == "no_diag":
        ci = np.array([0, 1, 0, 2, 1, 2], dtype=np.int32)
    elif case == "bad_rowptr":
        rp = np.array([0, 2, 1, 6], dtype=np.int32)
    elif case == "late_row":
        n = 5000
        rp = np.arange(n + 1, dtype=np.int32)
        ci = np.arange(n, dtype=np.int32)
        ci[4321] = 4320
    st, _, bad = O.validate(rp, ci)
    assert st != 0
    with pytest.raises(jv.JvError) as e:
        jv.jv_analyze(T(rp), T(ci))
    assert e.value.status == st and e.value.bad_row == bad
