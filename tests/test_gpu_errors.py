"""Failure paths on the GPU, none of which faults, traps or hangs it:
zero pivots are reported with the oracle's row; a row that never publishes
(test-only fault_row option) makes its dependants' bounded waits expire with
JV_ERR_TIMEOUT, the launch completes and the context stays usable; argument
errors are caught on the host before any launch."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from jvutil import SCHEDULES, analyze

jv = pytest.importorskip("paper_1812_06160_gb300")
pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.asarray(a), device="cuda")


@pytest.mark.parametrize("mode", SCHEDULES)
def test_zero_pivot_row_matches_oracle(mode):
    rp = np.array([0, 2, 5, 7], dtype=np.int32)
    ci = np.array([0, 1, 0, 1, 2, 1, 2], dtype=np.int32)
    v = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 3.0])
    _, st, bad = O.ilu0(rp, ci, v)
    assert st == O.ERR_ZERO_PIVOT and bad == 1
    h = analyze(jv, rp, ci, mode)
    with pytest.raises(jv.JvError) as e:
        jv.jv_ilu0_factor(h, T(v))
    assert e.value.status == jv.JV_ERR_ZERO_PIVOT and e.value.bad_row == 1


def test_zero_pivot_in_large_matrix():
    rp, ci, v = W.lap5(40)
    diag = O.diag_ptr(rp, ci)
    v2 = v.copy()
    v2[rp[777]:diag[777] + 1] = 0.0          # no multipliers and a zero diagonal: u_777 == 0
    _, st2, bad2 = O.ilu0(rp, ci, v2)
    assert st2 == O.ERR_ZERO_PIVOT and bad2 == 777
    for mode in SCHEDULES:
        h = analyze(jv, rp, ci, mode)
        with pytest.raises(jv.JvError) as e:
            jv.jv_ilu0_factor(h, T(v2))
        assert e.value.status == jv.JV_ERR_ZERO_PIVOT and e.value.bad_row == bad2


@pytest.mark.parametrize("mode", ["syncfree", "band"])
def test_syncfree_timeout_is_reported_and_context_survives(mode):
    rp, ci, v = W.lap5(24)
    n = len(rp) - 1
    # the last row of a 64-row band: every row that depends on it lies in the
    # next band, so in both sync-free schedules its dependants await it
    fault = 127
    h = analyze(jv, rp, ci, mode, fault_row=fault, spin_timeout_cycles=2_000_000)
    with pytest.raises(jv.JvError) as e:
        jv.jv_ilu0_factor(h, T(v))
    assert e.value.status == jv.JV_ERR_TIMEOUT and e.value.bad_row > fault
    olu, _, _ = O.ilu0(rp, ci, v)
    with pytest.raises(jv.JvError) as e:
        jv.jv_lsolve(h, T(olu), T(W.rhs(n, 1, seed=1)))
    assert e.value.status == jv.JV_ERR_TIMEOUT
    with pytest.raises(jv.JvError) as e:
        jv.jv_lsolve(h, T(olu), T(W.rhs(n, 4, seed=1)))
    assert e.value.status == jv.JV_ERR_TIMEOUT
    # the device is still healthy: a clean handle factors bit-exactly
    h2 = analyze(jv, rp, ci, mode)
    assert np.array_equal(jv.jv_ilu0_factor(h2, T(v)).cpu().numpy(), olu)
    torch.cuda.synchronize()


def test_timeout_in_power_law_rows():
    # a power-law row (the one-warp pull form) never publishes: the rows
    # awaiting its pivot time out, report, and the context survives
    rp, ci, v = W.powerlaw(3000, kmax=200, mean=12, seed_pattern=33, seed_values=34)
    lens = np.diff(rp)
    lower = [int((ci[rp[r]:rp[r + 1]] < r).sum()) for r in range(len(lens))]
    # a mid-length row early in the order: many later rows depend on it
    fault = next(r for r in range(len(lens)) if 20 <= lens[r] <= 40 and lower[r] >= 2)
    h = analyze(jv, rp, ci, "syncfree", fault_row=fault, spin_timeout_cycles=2_000_000)
    with pytest.raises(jv.JvError) as e:
        jv.jv_ilu0_factor(h, T(v))
    assert e.value.status == jv.JV_ERR_TIMEOUT and e.value.bad_row > fault
    olu, _, _ = O.ilu0(rp, ci, v)
    h2 = analyze(jv, rp, ci, "syncfree")
    assert np.array_equal(jv.jv_ilu0_factor(h2, T(v)).cpu().numpy(), olu)
    torch.cuda.synchronize()


def test_async_status_accumulates_until_sync():
    rp = np.array([0, 2, 5, 7], dtype=np.int32)
    ci = np.array([0, 1, 0, 1, 2, 1, 2], dtype=np.int32)
    v = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 3.0])
    h = jv.jv_analyze(T(rp), T(ci), check=False)
    jv.jv_ilu0_factor(h, T(v))               # enqueued, not checked
    st, row = jv.jv_status_sync(h)
    assert st == jv.JV_ERR_ZERO_PIVOT and row == 1
    assert jv.jv_status_sync(h) == (0, -1)


def test_host_argument_errors():
    rp, ci, v = W.lap5(8)
    h = jv.jv_analyze(T(rp), T(ci))
    lu = jv.jv_ilu0_factor(h, T(v))
    b = T(W.rhs(64, 1))
    with pytest.raises(ValueError):
        jv.jv_lsolve(h, lu, b[:10])
    with pytest.raises(jv.JvError) as e:
        jv.jv_lsolve(h, lu, b, x=b)          # x aliases b
    assert e.value.status == jv.JV_ERR_ARG
    with pytest.raises(TypeError):
        jv.jv_ilu0_factor(h, T(v).to(torch.int64))


def test_hop_latency_probe():
    # one publication seen by another SM: well under 10 us on any GPU this
    # library targets, and never zero
    hop = jv.jv_hop_latency(rounds=200, npartners=4)
    assert 0.05 < hop < 10.0
