"""Full-size parity at the five workloads, in the launch configuration the
benchmark times (sync-free FP64 on the 7-point 128^3 Laplacian, plus the
level-scheduled path, the level-set-reordered matrix, FP32 factors and the
32-right-hand-side solves).  The oracle finishes every full-size factor and
solve in seconds, so every output entry is compared, not a sample."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from jvutil import analyze, max_rel

jv = pytest.importorskip("paper_1812_06160_gb300")
pytestmark = pytest.mark.gpu

_CACHE = {}


def cfg(name):
    if name not in _CACHE:
        _CACHE[name] = W.config(name)
    return _CACHE[name]


def T(a):
    return torch.tensor(np.asarray(a), device="cuda")


def _levels_match(h, rp, ci):
    for which, upper in (("L", False), ("U", True)):
        lev, nlev, ptr, rows = O.level_sets(rp, ci, upper=upper)
        gn, gptr, grows, glev = jv.jv_get_levels(h, which)
        assert gn == nlev
        assert np.array_equal(gptr.cpu().numpy(), ptr)
        assert np.array_equal(grows.cpu().numpy(), rows)


def _full_check(rp, ci, v, b, mode, dtype=np.float64, reorder=False):
    if mode == "auto":        # the benchmark's configuration: sync-free, schedule chosen by the analysis
        h = jv.jv_analyze(T(rp), T(ci), reorder=reorder)
    else:
        h = analyze(jv, rp, ci, mode, reorder=reorder)
    if reorder:
        _, _, _, perm = O.level_sets(rp, ci)
        _, rp, ci, vmap = O.permute(rp, ci, perm)
        v = v[vmap]
        b = b[perm]
    _levels_match(h, rp, ci)
    diag = O.diag_ptr(rp, ci)
    if dtype == np.float64:
        olu, st, _ = O.ilu0(rp, ci, v, diag)
        lu = jv.jv_ilu0_factor(h, T(v))
    else:
        olu, st, _ = O.ilu0(rp, ci, v.astype(np.float32), diag, dtype=np.float32)
        lu = jv.jv_ilu0_factor(h, T(v), lu_dtype=torch.float32)
    assert st == 0
    assert np.array_equal(lu.cpu().numpy(), olu)
    olu64 = olu.astype(np.float64)
    bb = b.astype(dtype)
    y = jv.jv_lsolve(h, lu, T(bb))
    z = jv.jv_usolve(h, lu, y)
    oy = O.lsolve(rp, ci, diag, olu64, bb.astype(np.float64))
    oz = O.usolve(rp, ci, diag, olu64, oy)
    if dtype == np.float64:
        assert np.array_equal(y.cpu().numpy(), oy)
        assert np.array_equal(z.cpu().numpy(), oz)
        x = W.rhs(len(rp) - 1, 1, seed=21)
        s = jv.jv_spmv(h, T(v), T(x)).cpu().numpy()
        assert np.array_equal(s, O.spmv(rp, ci, v, x))
    else:
        assert max_rel(y.cpu().numpy(), oy) < 1e-4
        assert max_rel(z.cpu().numpy(), oz) < 1e-3
    return h


@pytest.mark.parametrize("mode", ["auto", "syncfree", "level"])
def test_c2_lap7_128_fp64(mode):
    c = cfg("c2")
    _full_check(c["rowptr"], c["colidx"], c["vals"], c["b"], mode)


def test_c2_lap7_128_fp64_reordered():
    c = cfg("c2")
    _full_check(c["rowptr"], c["colidx"], c["vals"], c["b"], "auto", reorder=True)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_c3_cd27_96(dtype):
    c = cfg("c3")
    _full_check(c["rowptr"], c["colidx"], c["vals"], c["b"], "auto", dtype=dtype)


def test_c5_aniso_1024_32rhs():
    c = cfg("c5")
    rp, ci, v, B = c["rowptr"], c["colidx"], c["vals"], c["b"]
    diag = O.diag_ptr(rp, ci)
    olu32, _, _ = O.ilu0(rp, ci, v.astype(np.float32), diag, dtype=np.float32)
    h = jv.jv_analyze(T(rp), T(ci))
    lu = jv.jv_ilu0_factor(h, T(v), lu_dtype=torch.float32)
    assert np.array_equal(lu.cpu().numpy(), olu32)
    lu64 = olu32.astype(np.float64)
    b32 = B.astype(np.float32)
    y = jv.jv_lsolve(h, lu, T(b32))
    z = jv.jv_usolve(h, lu, y)
    oy = O.lsolve(rp, ci, diag, lu64, b32.astype(np.float64))
    oz = O.usolve(rp, ci, diag, lu64, oy)
    assert max_rel(y.cpu().numpy(), oy) < 1e-4 and max_rel(z.cpu().numpy(), oz) < 1e-3
    # FP64 32-RHS parity on the same factor
    y64 = jv.jv_lsolve(h, T(lu64), T(B))
    assert np.array_equal(y64.cpu().numpy(), O.lsolve(rp, ci, diag, lu64, B))
    g = c["g"]
    gy = jv.jv_usolve_t(h, T(lu64), T(g)).cpu().numpy()
    assert np.array_equal(gy, O.usolve_t(rp, ci, diag, lu64, g))


@pytest.mark.slow
def test_c4_powerlaw_1e6():
    c = cfg("c4")
    _full_check(c["rowptr"], c["colidx"], c["vals"], c["b"], "auto")
    _full_check(c["rowptr"], c["colidx"], c["vals"], c["b"], "auto", dtype=np.float32)
