"""CUDA-graph replay of the per-level launch sequences (modes level and
hybrid): a replay is bit-exact with the oracle, reads the buffers' contents
at replay time, is recaptured when buffers or mode change, counts its
launches like the plain sequence, and a capture of the caller's own takes the
launches directly."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

jv = pytest.importorskip("paper_1812_06160_gb300")
pytestmark = pytest.mark.gpu


def T(a):
    return torch.tensor(np.asarray(a), device="cuda")


@pytest.mark.parametrize("mode", ["level", "hybrid"])
def test_replay_bit_exact_and_reads_current_buffers(mode):
    rp, ci, v = W.lap7(11)
    n = len(rp) - 1
    diag = O.diag_ptr(rp, ci)
    olu, st, _ = O.ilu0(rp, ci, v)
    assert st == O.OK
    h = jv.jv_analyze(T(rp), T(ci), exact=True, mode=mode, stage_min_rows=20)
    vals = T(v)
    lu = torch.empty_like(vals)
    counts = []
    for _ in range(3):                              # capture, then two replays
        c0 = jv.jv_launch_count()
        jv.jv_ilu0_factor(h, vals, lu)
        counts.append(jv.jv_launch_count() - c0)
        assert np.array_equal(lu.cpu().numpy(), olu)
    assert counts[0] == counts[1] == counts[2] > 2
    b = T(W.rhs(n, 1, seed=3))
    y = torch.empty_like(b)
    for seed in (3, 4, 5):                          # same buffers, new contents
        hb = W.rhs(n, 1, seed=seed)
        b.copy_(T(hb))
        jv.jv_lsolve(h, lu, b, y)
        assert np.array_equal(y.cpu().numpy(), O.lsolve(rp, ci, diag, olu, hb))
    # new output buffer: a new capture; the old graph still serves the old one
    y2 = torch.empty_like(b)
    jv.jv_lsolve(h, lu, b, y2)
    assert torch.equal(y2, y)
    # mode switch: sync-free runs plainly, then the level graphs replay again
    jv.jv_set_mode(h, "syncfree")
    z = jv.jv_usolve(h, lu, y)
    jv.jv_set_mode(h, mode)
    z2 = jv.jv_usolve(h, lu, y)
    assert torch.equal(z, z2)
    assert np.array_equal(z.cpu().numpy(), O.usolve(rp, ci, diag, olu, y.cpu().numpy()))


def test_graphs_off_matches():
    rp, ci, v = W.aniso5(40)
    h1 = jv.jv_analyze(T(rp), T(ci), exact=True, mode="level")
    h0 = jv.jv_analyze(T(rp), T(ci), exact=True, mode="level", graphs=False)
    vals = T(v)
    for _ in range(2):
        lu1 = jv.jv_ilu0_factor(h1, vals)
        lu0 = jv.jv_ilu0_factor(h0, vals)
        assert torch.equal(lu1, lu0)
    b = T(W.rhs(len(rp) - 1, 2, seed=8))
    assert torch.equal(jv.jv_lsolve(h1, lu1, b), jv.jv_lsolve(h0, lu0, b))


def test_caller_capture_takes_the_launches():
    rp, ci, v = W.lap5(30)
    n = len(rp) - 1
    diag = O.diag_ptr(rp, ci)
    olu, _, _ = O.ilu0(rp, ci, v)
    h = jv.jv_analyze(T(rp), T(ci), exact=True, mode="level", check=False)
    lu = T(olu)
    b = T(W.rhs(n, 1, seed=1))
    y = torch.empty_like(b)
    z = torch.empty_like(b)
    jv.jv_lsolve(h, lu, b, y)                        # warm up outside the capture
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            jv.jv_lsolve(h, lu, b, y)
            jv.jv_usolve(h, lu, y, z)
    torch.cuda.current_stream().wait_stream(s)
    for seed in (11, 12):
        hb = W.rhs(n, 1, seed=seed)
        b.copy_(T(hb))
        g.replay()
        torch.cuda.synchronize()
        yy = O.lsolve(rp, ci, diag, olu, hb)
        assert np.array_equal(y.cpu().numpy(), yy)
        assert np.array_equal(z.cpu().numpy(), O.usolve(rp, ci, diag, olu, yy))
    st, _ = jv.jv_status_sync(h)
    assert st == 0
