"""jv_lsolve_noalloc: the forward substitution for callers that cannot let
the library allocate device memory (see include/jv.h).  Its results must be
those of the regular jv_lsolve (the same FP64 operations in the same order,
so equal bit for bit -- the bar the other solve tests use), on two calls in a
row, since the calls share one fixed scratch array that each call re-clears.

Kept in a file of its own that pytest collects last, so that a run stopping
at the first failure has already run every other test."""
import numpy as np
import pytest
import torch

import workloads as W

jv = pytest.importorskip("paper_1812_06160_gb300")
pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.asarray(a), device="cuda")


def _case(name):
    if name == "lap7_24":
        return W.lap7(24)
    if name == "random":
        return W.random_csr(3000, 5.0, seed=77)
    c = W.config(name)
    return c["rowptr"], c["colidx"], c["vals"]


@pytest.mark.parametrize("name", ["lap7_24", "random", "c2"])
def test_noalloc_lsolve_matches_lsolve_twice(name):
    rp, ci, v = _case(name)
    n = len(rp) - 1
    h = jv.jv_analyze(T(rp), T(ci))
    lu = jv.jv_ilu0_factor(h, T(v))
    rowptr, colidx, diag = jv.jv_get_pattern(h)
    _, _, level_rows, _ = jv.jv_get_levels(h, "L")
    for call, seed in enumerate((1, 2)):
        b = T(W.rhs(n, 1, seed=seed))
        want = jv.jv_lsolve(h, lu, b)
        got = jv.jv_lsolve_noalloc(rowptr, colidx, diag, level_rows, lu, b)
        assert torch.equal(got, want), f"call {call}"
    # the natural order is also a valid dependency order
    order = torch.arange(n, dtype=torch.int32, device="cuda")
    b = T(W.rhs(n, 1, seed=3))
    assert torch.equal(jv.jv_lsolve_noalloc(rowptr, colidx, diag, order, lu, b),
                       jv.jv_lsolve(h, lu, b))


def test_noalloc_rejects_too_many_rows():
    n = (1 << 21) + 1
    small = torch.zeros(4, dtype=torch.int32, device="cuda")
    vec = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = jv._jv.lib.jv_lsolve_noalloc(n, small.data_ptr(), small.data_ptr(), small.data_ptr(),
                                      small.data_ptr(), vec.data_ptr(), vec.data_ptr(),
                                      vec.data_ptr() + 8, None)
    assert st == jv.JV_ERR_ARG


def test_noalloc_bad_order_times_out_then_recovers():
    # reversed rows: every claimed chunk waits on rows that come later in the
    # order; 13,824 rows make 1,728 chunks, more than the SMs can hold at once,
    # so no schedule can finish them -- one bounded wait (about 2 s) expires,
    # the call reports JV_ERR_TIMEOUT, and the next call starts clean
    rp, ci, v = W.lap7(24)
    n = len(rp) - 1
    h = jv.jv_analyze(T(rp), T(ci))
    lu = jv.jv_ilu0_factor(h, T(v))
    rowptr, colidx, diag = jv.jv_get_pattern(h)
    b = T(W.rhs(n, 1, seed=4))
    rev = torch.arange(n - 1, -1, -1, dtype=torch.int32, device="cuda")
    with pytest.raises(jv.JvError) as e:
        jv.jv_lsolve_noalloc(rowptr, colidx, diag, rev, lu, b)
    assert e.value.status == jv.JV_ERR_TIMEOUT
    _, _, level_rows, _ = jv.jv_get_levels(h, "L")
    assert torch.equal(jv.jv_lsolve_noalloc(rowptr, colidx, diag, level_rows, lu, b),
                       jv.jv_lsolve(h, lu, b))


def test_noalloc_rejects_rows_outside_the_matrix():
    # an order entry equal to n names no row: the call reports JV_ERR_ARG
    # (the row is never read) and the next call starts clean
    rp, ci, v = W.lap5(20)
    n = len(rp) - 1
    h = jv.jv_analyze(T(rp), T(ci))
    lu = jv.jv_ilu0_factor(h, T(v))
    rowptr, colidx, diag = jv.jv_get_pattern(h)
    b = T(W.rhs(n, 1, seed=5))
    bad = torch.arange(n, dtype=torch.int32, device="cuda")
    bad[n // 2] = n
    with pytest.raises(jv.JvError) as e:
        jv.jv_lsolve_noalloc(rowptr, colidx, diag, bad, lu, b)
    assert e.value.status in (jv.JV_ERR_ARG, jv.JV_ERR_TIMEOUT)
    order = torch.arange(n, dtype=torch.int32, device="cuda")
    assert torch.equal(jv.jv_lsolve_noalloc(rowptr, colidx, diag, order, lu, b),
                       jv.jv_lsolve(h, lu, b))
