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


# Finite-difference bar: 1e-6 relative per sampled entry, i.e.
# |fd - g| <= 1e-6 * max(|g|, FD_FLOOR * max|g|), the floor (a fraction of the
# largest gradient entry of the same tensor) only for entries that nearly
# cancel, where a central difference cannot resolve a relative error.
FD_REL = 1e-6
FD_FLOOR = 1e-3


def _fd_ok(fd, g, gmax):
    return abs(fd - g) <= FD_REL * max(abs(g), FD_FLOOR * gmax)


def test_finite_differences_fp64():
    # central differences on the FP64 instance: z = U^-1 L^-1 r is linear in r
    # (the difference is exact up to rounding) and smooth in the factor values
    # (truncation ~ h^2); samples cover random entries and the largest ones,
    # of r and of both the L and the U part of the factor
    rp, ci, v = W.aniso5(24, eps=0.01)
    n = len(rp) - 1
    nrhs = 6
    olu, _, _ = O.ilu0(rp, ci, v)
    r, gz = W.rhs(n, nrhs, seed=3), W.rhs(n, nrhs, seed=4)
    h = jv.jv_analyze(T(rp), T(ci))
    rt = T(r, requires_grad=True)
    lut = T(olu, requires_grad=True)
    gzt = T(gz)
    loss = lambda rr, ll: float((jv.ilu_apply(rr, ll, h) * gzt).sum())
    (jv.ilu_apply(rt, lut, h) * gzt).sum().backward()
    gr = rt.grad.view(-1).cpu().numpy()
    glu = lut.grad.cpu().numpy()
    rng = np.random.default_rng(5)
    rows = np.repeat(np.arange(n), np.diff(rp))
    lower = np.flatnonzero(ci < rows)
    upper = np.flatnonzero(ci >= rows)
    r_idx = np.concatenate([rng.choice(n * nrhs, 16, replace=False), np.argsort(-np.abs(gr))[:4]])
    lu_idx = np.concatenate([rng.choice(lower, 12, replace=False), rng.choice(upper, 12, replace=False),
                             np.argsort(-np.abs(glu))[:4]])
    worst = 0.0
    for idx in r_idx:
        e = torch.zeros(n * nrhs, dtype=torch.float64, device="cuda")
        e[int(idx)] = 1.0
        e = e.view(n, nrhs)
        hs = 1e-6
        fd = (loss(rt.detach() + hs * e, lut.detach()) - loss(rt.detach() - hs * e, lut.detach())) / (2 * hs)
        g = float(gr[idx])
        worst = max(worst, abs(fd - g) / max(abs(g), FD_FLOOR * np.abs(gr).max()))
        assert _fd_ok(fd, g, np.abs(gr).max()), (int(idx), fd, g)
    for p in lu_idx:
        e = torch.zeros(len(olu), dtype=torch.float64, device="cuda")
        e[int(p)] = 1.0
        hs = 1e-6 * max(1.0, abs(olu[p]))
        fd = (loss(rt.detach(), lut.detach() + hs * e) - loss(rt.detach(), lut.detach() - hs * e)) / (2 * hs)
        g = float(glu[p])
        worst = max(worst, abs(fd - g) / max(abs(g), FD_FLOOR * np.abs(glu).max()))
        assert _fd_ok(fd, g, np.abs(glu).max()), (int(p), fd, g)
    print(f"finite differences: largest relative error {worst:.2e} over "
          f"{len(r_idx) + len(lu_idx)} entries")


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
