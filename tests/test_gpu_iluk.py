"""ILU(k) on the GPU: the level-of-fill pattern (columns and levels) is
bit-exact with the oracle's symbolic sweep for k = 0..3 on the parity cases
and at full size, A's values land on it exactly, and the numeric ILU(k) --
the ILU(0) kernels run on the filled pattern -- is bit-exact with the oracle's
sweep on that pattern."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from jvutil import small_matrices

jv = pytest.importorskip("paper_1812_06160_gb300")
pytestmark = pytest.mark.gpu

CASES = [c for c in small_matrices() if c[0] not in ("rand1", "rand2")] + \
    [c for c in small_matrices() if c[0] in ("rand1", "rand2")]


def T(a):
    return torch.tensor(np.asarray(a), device="cuda")


@pytest.mark.parametrize("level", [0, 1, 2, 3])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_iluk_pattern_bit_exact(case, level):
    name, rp, ci, v = case
    frp, fci, flev = O.iluk_pattern(rp, ci, level)
    if np.diff(frp).max() > 1024:
        with pytest.raises(jv.JvError) as e:
            jv.jv_iluk_symbolic(T(rp), T(ci), level)
        assert e.value.status == jv.JV_ERR_NOMEM
        return
    grp, gci, glev = jv.jv_iluk_symbolic(T(rp), T(ci), level, with_levels=True)
    assert np.array_equal(grp.cpu().numpy(), frp)
    assert np.array_equal(gci.cpu().numpy(), fci)
    assert np.array_equal(glev.cpu().numpy(), flev)
    fv = jv.jv_scatter_values(T(rp), T(ci), T(v), grp, gci)
    want = O.scatter_values(rp, ci, v, frp, fci)
    assert np.array_equal(fv.cpu().numpy(), want)
    # numeric ILU(k): the ILU(0) sweep on the filled pattern
    olu, st, bad = O.ilu0(frp, fci, want)
    h = jv.jv_analyze(grp, gci, exact=True)
    if st != O.OK:
        with pytest.raises(jv.JvError) as e:
            jv.jv_ilu0_factor(h, fv)
        assert e.value.status == jv.JV_ERR_ZERO_PIVOT and e.value.bad_row == bad
        return
    lu = jv.jv_ilu0_factor(h, fv)
    assert np.array_equal(lu.cpu().numpy(), olu)


def test_iluk_row_too_long_is_reported():
    n = 1100                                   # dense lower triangle: row i has i + 1 entries
    rp = np.concatenate([[0], np.cumsum(np.arange(1, n + 1))]).astype(np.int32)
    ci = np.concatenate([np.arange(i + 1) for i in range(n)]).astype(np.int32)
    with pytest.raises(jv.JvError) as e:
        jv.jv_iluk_symbolic(T(rp), T(ci), 1)
    assert e.value.status == jv.JV_ERR_NOMEM and e.value.bad_row == 1024


@pytest.mark.parametrize("cfg,level", [("c2", 1), ("c3", 1), ("c1", 3)])
def test_iluk_full_size(cfg, level):
    c = W.config(cfg)
    rp, ci, v = c["rowptr"], c["colidx"], c["vals"]
    frp, fci, flev = O.iluk_pattern(rp, ci, level)
    grp, gci, glev = jv.jv_iluk_symbolic(T(rp), T(ci), level, with_levels=True)
    assert np.array_equal(grp.cpu().numpy(), frp)
    assert np.array_equal(gci.cpu().numpy(), fci)
    assert np.array_equal(glev.cpu().numpy(), flev)
    fv = jv.jv_scatter_values(T(rp), T(ci), T(v), grp, gci)
    olu, st, _ = O.ilu0(frp, fci, O.scatter_values(rp, ci, v, frp, fci))
    assert st == O.OK
    h = jv.jv_analyze(grp, gci, exact=True)
    lu = jv.jv_ilu0_factor(h, fv)
    assert np.array_equal(lu.cpu().numpy(), olu)
    if cfg == "c2":
        # a stronger preconditioner: PCG on the filled pattern (A's values,
        # zeros on the fill) needs fewer iterations than with ILU(0)
        b = T(c["b"])
        _, info = jv.jv_pcg(h, fv, lu, b, tol=1e-8)
        h0 = jv.jv_analyze(T(rp), T(ci), exact=True)
        vt = T(v)
        _, info0 = jv.jv_pcg(h0, vt, jv.jv_ilu0_factor(h0, vt), b, tol=1e-8)
        assert info["converged"] and info["iters"] < info0["iters"]
