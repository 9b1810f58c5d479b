"""GPU Krylov drivers vs the oracle's: same algorithm (flexible PCG,
right-preconditioned FGMRES(m) with modified Gram-Schmidt), so the iteration
counts agree within one and the solutions agree with the oracle's to the
requested tolerance; FP32 factors inside the FP64 iteration still converge
to 1e-8."""
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
def test_pcg_matches_oracle(mode):
    c = W.config("c1")
    rp, ci, v, b = c["rowptr"], c["colidx"], c["vals"], c["b"]
    olu, _, _ = O.ilu0(rp, ci, v)
    ox, oit, orel = O.pcg(rp, ci, v, olu, b, tol=1e-8)
    h = analyze(jv, rp, ci, mode)
    vt = T(v)
    lu = jv.jv_ilu0_factor(h, vt)
    x, info = jv.jv_pcg(h, vt, lu, T(b), tol=1e-8)
    assert info["converged"] and info["true_relres"] <= 1e-8
    assert abs(info["iters"] - oit) <= 1
    assert np.abs(x.cpu().numpy() - ox).max() <= 1e-6 * np.abs(ox).max()
    lu32 = jv.jv_ilu0_factor(h, vt, lu_dtype=torch.float32)
    x32, info32 = jv.jv_pcg(h, vt, lu32, T(b), tol=1e-8)
    assert info32["converged"] and info32["true_relres"] <= 1e-8
    assert abs(info32["iters"] - oit) <= 3


@pytest.mark.parametrize("mode", SCHEDULES)
def test_fgmres_matches_oracle(mode):
    rp, ci, v, _ = W.cd27(10)
    n = len(rp) - 1
    b = W.rhs(n, 1, seed=4)
    olu, _, _ = O.ilu0(rp, ci, v)
    ox, oit, orel = O.fgmres(rp, ci, v, olu, b, m=30, tol=1e-8)
    assert oit > 0
    h = analyze(jv, rp, ci, mode)
    vt = T(v)
    lu = jv.jv_ilu0_factor(h, vt)
    x, info = jv.jv_fgmres(h, vt, lu, T(b), tol=1e-8, restart=30)
    assert info["converged"] and info["true_relres"] <= 1e-8
    assert abs(info["iters"] - oit) <= 1
    assert np.abs(x.cpu().numpy() - ox).max() <= 1e-6 * np.abs(ox).max()
    lu32 = jv.jv_ilu0_factor(h, vt, lu_dtype=torch.float32)
    _, info32 = jv.jv_fgmres(h, vt, lu32, T(b), tol=1e-8, restart=30)
    assert info32["converged"] and info32["true_relres"] <= 1e-8


def test_fgmres_restarts():
    rp, ci, v = W.aniso5(40)
    n = len(rp) - 1
    b = W.rhs(n, 1, seed=11)
    olu, _, _ = O.ilu0(rp, ci, v)
    _, oit, _ = O.fgmres(rp, ci, v, olu, b, m=5, tol=1e-9, max_restarts=500)
    h = jv.jv_analyze(T(rp), T(ci))
    vt = T(v)
    lu = jv.jv_ilu0_factor(h, vt)
    _, info = jv.jv_fgmres(h, vt, lu, T(b), tol=1e-9, restart=5, max_restarts=500)
    assert info["converged"] and info["iters"] > 5
    assert abs(info["iters"] - oit) <= 2
