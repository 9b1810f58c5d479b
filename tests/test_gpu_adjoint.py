"""Differentiable preconditioner apply z = U^-1 L^-1 r: the GPU backward
(transposed solves + masked outer products, recomputing y = L^-1 r) against
the oracle's adjoint and against central finite differences."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from jvutil import SCHEDULES, analyze, max_rel

jv = pytest.importorskip("paper_1812_06160_gb300")
pytestmark = pytest.mark.gpu


def T(a, **kw):
    return torch.tensor(np.asarray(a), device="cuda", **kw)


def _oracle_adjoint(rp, ci, lu, r, gz):
    diag = O.diag_ptr(rp, ci)
    y = O.lsolve(rp, ci, diag, lu, r)
    z = O.usolve(rp, ci, diag, lu, y)
    gy = O.usolve_t(rp, ci, diag, lu, gz)
    gr = O.lsolve_t(rp, ci, diag, lu, gy)
    g = O.masked_outer(rp, ci, diag, 0, gr, y, -1.0) + O.masked_outer(rp, ci, diag, 1, gy, z, -1.0)
    return z, gr, g


@pytest.mark.parametrize("mode", SCHEDULES)
def test_backward_matches_oracle_adjoint(mode):
    rp, ci, v = W.aniso5(20)
    n = len(rp) - 1
    olu, _, _ = O.ilu0(rp, ci, v)
    r, gz = W.rhs(n, 6, seed=1), W.rhs(n, 6, seed=2)
    h = analyze(jv, rp, ci, mode)
    rt = T(r, requires_grad=True)
    lut = T(olu, requires_grad=True)
    z = jv.ilu_apply(rt, lut, h)
    (z * T(gz)).sum().backward()
    oz, ogr, og = _oracle_adjoint(rp, ci, olu, r, gz)
    assert max_rel(z.detach().cpu().numpy(), oz) < 1e-12
    assert max_rel(rt.grad.cpu().numpy(), ogr) < 1e-12
    assert max_rel(lut.grad.cpu().numpy(), og) < 1e-12


def test_finite_differences_fp64():
    rp, ci, v = W.aniso5(12, eps=0.01)
    n = len(rp) - 1
    olu, _, _ = O.ilu0(rp, ci, v)
    r, gz = W.rhs(n, 4, seed=3), W.rhs(n, 4, seed=4)
    h = jv.jv_analyze(T(rp), T(ci))
    rt = T(r, requires_grad=True)
    lut = T(olu, requires_grad=True)
    gzt = T(gz)
    loss = lambda rr, ll: float((jv.ilu_apply(rr, ll, h) * gzt).sum())
    (jv.ilu_apply(rt, lut, h) * gzt).sum().backward()
    rng = np.random.default_rng(5)
    for idx in rng.choice(n * 4, 6, replace=False):
        e = torch.zeros(n * 4, dtype=torch.float64, device="cuda")
        e[idx] = 1.0
        e = e.view(n, 4)
        hstep = 1e-6
        fd = (loss(rt.detach() + hstep * e, lut.detach()) - loss(rt.detach() - hstep * e, lut.detach())) / (2 * hstep)
        g = float(rt.grad.view(-1)[idx])
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(g))
    for p in rng.choice(len(olu), 8, replace=False):
        e = torch.zeros(len(olu), dtype=torch.float64, device="cuda")
        e[p] = 1.0
        hstep = 1e-6 * max(1.0, abs(olu[p]))
        fd = (loss(rt.detach(), lut.detach() + hstep * e) - loss(rt.detach(), lut.detach() - hstep * e)) / (2 * hstep)
        g = float(lut.grad[p])
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(g))


def test_fp32_adjoint_32_rhs_close_to_fp64():
    rp, ci, v = W.aniso5(64)
    n = len(rp) - 1
    olu32, _, _ = O.ilu0(rp, ci, v.astype(np.float32), dtype=np.float32)
    r, gz = W.rhs(n, 32, seed=7), W.rhs(n, 32, seed=8)
    h = jv.jv_analyze(T(rp), T(ci))
    rt = T(r.astype(np.float32), requires_grad=True)
    lut = T(olu32, requires_grad=True)
    z = jv.ilu_apply(rt, lut, h)
    (z * T(gz.astype(np.float32))).sum().backward()
    oz, ogr, og = _oracle_adjoint(rp, ci, olu32.astype(np.float64), r.astype(np.float32).astype(np.float64), gz.astype(np.float32).astype(np.float64))
    assert max_rel(z.detach().cpu().numpy(), oz) < 1e-4
    assert max_rel(rt.grad.cpu().numpy(), ogr) < 1e-4
    assert max_rel(lut.grad.cpu().numpy(), og) < 1e-4
