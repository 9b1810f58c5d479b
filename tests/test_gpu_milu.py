"""Modified ILU(0) on the GPU: bit-exact with the oracle's MILU (FP64 and
FP32 twins) on the small parity cases in both schedules, at full size on the
7-point 128^3 and 27-point 96^3 workloads, and the row-sum property of the
factors."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from jvutil import analyze, small_matrices

jv = pytest.importorskip("paper_1812_06160_gb300")
pytestmark = pytest.mark.gpu

CASES = small_matrices()


def T(a):
    return torch.tensor(np.asarray(a), device="cuda")


@pytest.mark.parametrize("mode", ["level", "syncfree"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_milu_factor_bit_exact(case, mode):
    name, rp, ci, v = case
    olu, st, bad = O.ilu0(rp, ci, v, milu=True)
    h = analyze(jv, rp, ci, mode, milu=True)
    if st != O.OK:
        with pytest.raises(jv.JvError) as e:
            jv.jv_ilu0_factor(h, T(v))
        assert e.value.status == jv.JV_ERR_ZERO_PIVOT and e.value.bad_row == bad
        return
    lu = jv.jv_ilu0_factor(h, T(v)).cpu().numpy()
    assert np.array_equal(lu, olu), f"{name}: {np.abs(lu - olu).max()}"
    o32, st32, _ = O.ilu0(rp, ci, v, dtype=np.float32, milu=True)
    if st32 == O.OK:
        lu32 = jv.jv_ilu0_factor(h, T(v).float()).cpu().numpy()
        assert np.array_equal(lu32, o32)


def test_milu_band_schedule_rejected():
    rp, ci, v = W.lap5(8)
    with pytest.raises(jv.JvError) as e:
        jv.jv_analyze(T(rp), T(ci), exact=True, milu=True, band_rows=64)
    assert e.value.status == jv.JV_ERR_ARG


@pytest.mark.parametrize("cfg", ["c2", "c3"])
def test_milu_full_size_bit_exact_and_row_sums(cfg):
    c = W.config(cfg)
    rp, ci, v = c["rowptr"], c["colidx"], c["vals"]
    olu, st, _ = O.ilu0(rp, ci, v, milu=True)
    assert st == O.OK
    h = jv.jv_analyze(T(rp), T(ci), exact=True, milu=True)
    lu = jv.jv_ilu0_factor(h, T(v))
    assert np.array_equal(lu.cpu().numpy(), olu)
    # row sums: L U e == A e (to rounding), through the library's own solves:
    # A e = L U e  <=>  U^-1 L^-1 (A e) == e
    n = len(rp) - 1
    e = torch.ones(n, dtype=torch.float64, device="cuda")
    ae = jv.jv_spmv(h, T(v), e)
    z = jv.jv_usolve(h, lu, jv.jv_lsolve(h, lu, ae))
    assert (z - e).abs().max().item() <= 1e-9
    # plain ILU(0) does not keep them (there is dropped fill on these patterns)
    h0 = jv.jv_analyze(T(rp), T(ci), exact=True)
    lu0 = jv.jv_ilu0_factor(h0, T(v))
    z0 = jv.jv_usolve(h0, lu0, jv.jv_lsolve(h0, lu0, ae))
    assert (z0 - e).abs().max().item() > 1e-6
