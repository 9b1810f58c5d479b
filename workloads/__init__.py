"""Seeded synthetic workloads shaped like the paper's test matrices.

This module only *builds inputs*: CSR patterns, values and right-hand sides.
It contains none of the method's arithmetic (no factorisation, no solve, no
level computation), and it is the one module shared by the oracle side and
the CUDA side of the tests, by ``bench.py`` and by ``smoke()``.

The paper measures on 18 SuiteSparse matrices (Sec. IV, Table I), which are
not available here; these generators stand in for them:

* ``lap5`` / ``lap7`` -- 5- and 7-point Laplacians in natural order (PDE
  group A of Table I: parabolic_fem, thermal2, ecology2, apache2, RD 5-7);
* ``cd27`` -- 27-point convection-diffusion (RD ~26, like af_shell3 /
  fem_filter density), nonsymmetric values;
* ``powerlaw`` -- random, power-law row lengths, structurally symmetrised
  (circuit matrices: scircuit, ASIC_*, G3_circuit); with
  ``symmetrize=False`` the pattern stays structurally nonsymmetric (the
  case where the levels of lower(A) and of lower(A + A^T) differ, Sec. III
  and Sec. V's table of nonsymmetric matrices);
* ``aniso5`` -- 2-D anisotropic diffusion (long level chains);
* ``random_csr`` -- small random patterns for exhaustive tests.

All patterns are 0-based CSR with int32 indices, strictly ascending columns
and a stored diagonal.  Values are float64.
"""
from __future__ import annotations

import numpy as np

__all__ = ["stencil", "lap5", "lap7", "cd27", "powerlaw", "aniso5", "random_csr",
           "rhs", "config", "CONFIG_NAMES"]


def stencil(dims, offsets, weights, diag_value):
    """Assemble a constant-coefficient stencil on a Dirichlet grid.

    dims = (mx, my, mz); offsets = list of (dx, dy, dz) excluding (0,0,0);
    weights = matching off-diagonal values; the diagonal is ``diag_value``
    for every row (neighbours outside the grid are simply dropped).
    Natural ordering p = x + mx*(y + my*z).
    """
    mx, my, mz = dims
    n = mx * my * mz
    offs = [(0, 0, 0)] + list(offsets)
    wts = [float(diag_value)] + [float(w) for w in weights]
    lin = [dx + mx * (dy + my * dz) for dx, dy, dz in offs]
    order = np.argsort(lin, kind="stable")
    idx = np.arange(n, dtype=np.int64)
    x = idx % mx
    y = (idx // mx) % my
    z = idx // (mx * my)
    cols = np.empty((n, len(offs)), dtype=np.int64)
    mask = np.empty((n, len(offs)), dtype=bool)
    vals = np.empty((n, len(offs)), dtype=np.float64)
    for slot, o in enumerate(order):
        dx, dy, dz = offs[o]
        ok = (x + dx >= 0) & (x + dx < mx) & (y + dy >= 0) & (y + dy < my) & \
             (z + dz >= 0) & (z + dz < mz)
        mask[:, slot] = ok
        cols[:, slot] = idx + lin[o]
        vals[:, slot] = wts[o]
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = cols[mask].astype(np.int32)
    v = vals[mask]
    return rowptr.astype(np.int32), colidx, v


def lap5(m, diag=4.0, off=-1.0):
    """2-D 5-point Laplacian on an m x m grid."""
    offs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0)]
    return stencil((m, m, 1), offs, [off] * 4, diag)


def lap7(m, diag=6.0 + 1e-3, off=-1.0):
    """3-D 7-point Laplacian on an m^3 grid, diagonal 6 + shift."""
    offs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    return stencil((m, m, m), offs, [off] * 6, diag)


def aniso5(m, eps=0.01):
    """2-D anisotropic diffusion: x-coupling -eps, y-coupling -1, diagonal 2+2 eps."""
    offs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0)]
    return stencil((m, m, 1), offs, [-eps, -eps, -1.0, -1.0], 2.0 + 2.0 * eps)


def cd27(m, peclet=10.0, seed=3):
    """3-D convection-diffusion, 27-point diffusion stencil (diagonal 26, all
    26 neighbours -1) plus first-order upwind convection with cell Peclet
    number ``peclet`` along a seeded random unit direction b: for every axis d
    the diagonal gains peclet*|b_d| and the upwind neighbour (offset
    -sign(b_d) along d) gains -peclet*|b_d|.  Nonsymmetric values, weakly
    diagonally dominant M-matrix.  Returns (rowptr, colidx, vals, b_dir)."""
    rng = np.random.default_rng(seed)
    bdir = rng.standard_normal(3)
    bdir /= np.linalg.norm(bdir)
    offs, wts = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx == dy == dz == 0:
                    continue
                w = -1.0
                d = (dx, dy, dz)
                for axis in range(3):
                    unit = [0, 0, 0]
                    unit[axis] = -int(np.sign(bdir[axis])) if bdir[axis] != 0 else 0
                    if tuple(unit) == d and bdir[axis] != 0:
                        w -= peclet * abs(bdir[axis])
                offs.append(d)
                wts.append(w)
    diag = 26.0 + peclet * float(np.abs(bdir).sum())
    rp, ci, v = stencil((m, m, m), offs, wts, diag)
    return rp, ci, v, bdir


def _powerlaw_pmf(kmin, kmax, mean):
    ks = np.arange(kmin, kmax + 1, dtype=np.float64)

    def mean_of(alpha):
        w = ks ** (-alpha)
        return float((ks * w).sum() / w.sum())

    lo, hi = 1.01, 6.0           # mean_of is decreasing in alpha
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mean_of(mid) > mean:
            lo = mid
        else:
            hi = mid
    alpha = 0.5 * (lo + hi)
    w = ks ** (-alpha)
    return ks.astype(np.int64), w / w.sum(), alpha


def powerlaw(n, kmin=4, kmax=2000, mean=16, seed_pattern=5, seed_values=6, symmetrize=True):
    """Random sparse matrix with power-law row lengths, symmetrised pattern.

    Every row draws an off-diagonal count k from P(k) ~ k^-alpha on
    [kmin, kmax] with alpha chosen so the mean is ``mean``, then k distinct
    uniform columns != i (duplicates merged).  The pattern is symmetrised
    (A + A^T; skipped with ``symmetrize=False``, which keeps the drawn
    entries only) and the diagonal added; every off-diagonal value is drawn
    independently uniform[-1, 1] (mirror entries independent, so the values
    are nonsymmetric) and the diagonal is 1 + sum |off-diagonal| of its row.
    """
    rng = np.random.default_rng(seed_pattern)
    ks, pmf, _ = _powerlaw_pmf(kmin, min(kmax, n - 1), mean)
    k = rng.choice(ks, size=n, p=pmf)
    rows = np.repeat(np.arange(n, dtype=np.int64), k)
    cols = rng.integers(0, n - 1, size=rows.size, dtype=np.int64)
    cols += (cols >= rows)
    parts = [rows * n + cols, np.arange(n, dtype=np.int64) * (n + 1)]
    if symmetrize:
        parts.append(cols * n + rows)
    keys = np.concatenate(parts)
    keys = np.unique(keys)
    r = keys // n
    c = keys - r * n
    counts = np.bincount(r, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    vrng = np.random.default_rng(seed_values)
    vals = vrng.uniform(-1.0, 1.0, size=keys.size)
    ondiag = r == c
    vals[ondiag] = 0.0
    rowabs = np.bincount(r, weights=np.abs(vals), minlength=n)
    vals[ondiag] = 1.0 + rowabs
    return rowptr.astype(np.int32), c.astype(np.int32), vals


def random_csr(n, avg_offdiag=3.0, seed=0, symmetric_pattern=False, dominant=True,
               lower_only=False, upper_only=False, max_row=None):
    """Small random CSR with a stored diagonal, for exhaustive tests."""
    rng = np.random.default_rng(seed)
    dense = rng.random((n, n)) < (avg_offdiag / max(n - 1, 1))
    if max_row is not None:
        for i in range(n):
            nz = np.flatnonzero(dense[i])
            if nz.size > max_row:
                dense[i, rng.choice(nz, nz.size - max_row, replace=False)] = False
    if symmetric_pattern:
        dense |= dense.T
    if lower_only:
        dense = np.tril(dense)
    if upper_only:
        dense = np.triu(dense)
    np.fill_diagonal(dense, True)
    vals = np.where(dense, rng.uniform(-1.0, 1.0, size=(n, n)), 0.0)
    if dominant:
        off = np.abs(vals).sum(axis=1) - np.abs(np.diag(vals))
        np.fill_diagonal(vals, 1.0 + off)
    else:
        np.fill_diagonal(vals, np.where(np.abs(np.diag(vals)) < 0.1, 1.0, np.diag(vals)))
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum(dense.sum(axis=1))
    r, c = np.nonzero(dense)
    return rowptr, c.astype(np.int32), vals[r, c].astype(np.float64)


def rhs(n, nrhs=1, seed=1):
    """Uniform[-1, 1] right-hand side(s), row-major n x nrhs (1-D if nrhs == 1)."""
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, size=(n, nrhs))
    return b[:, 0].copy() if nrhs == 1 else b


CONFIG_NAMES = ("c1", "c2", "c3", "c4", "c5", "c4n")


def config(name, scale=None):
    """The five workloads.  ``scale`` shrinks the grid / n for quick runs
    (None = full size).  Returns a dict with rowptr, colidx, vals, b, meta."""
    if name == "c1":
        m = scale or 64
        rp, ci, v = lap5(m)
        return dict(name="lap5_64x64" if m == 64 else f"lap5_{m}x{m}", rowptr=rp, colidx=ci,
                    vals=v, b=rhs(m * m, 1, seed=1), dtype="f64", grid=(m, m, 1))
    if name == "c2":
        m = scale or 128
        rp, ci, v = lap7(m)
        return dict(name=f"lap7_{m}^3_shift1e-3", rowptr=rp, colidx=ci, vals=v,
                    b=rhs(m ** 3, 1, seed=2), dtype="f64", grid=(m, m, m))
    if name == "c3":
        m = scale or 96
        rp, ci, v, bdir = cd27(m, 10.0, seed=3)
        return dict(name=f"cd27_{m}^3_pe10", rowptr=rp, colidx=ci, vals=v,
                    b=rhs(m ** 3, 1, seed=4), dtype="f32", grid=(m, m, m), bdir=bdir)
    if name == "c4":
        n = scale or 1_000_000
        rp, ci, v = powerlaw(n, seed_pattern=5, seed_values=6)
        return dict(name=f"powerlaw_n{n}", rowptr=rp, colidx=ci, vals=v,
                    b=rhs(n, 1, seed=9), dtype="f32")
    if name == "c4n":
        # the C4 recipe without the symmetrisation: a structurally
        # nonsymmetric pattern (about 17 entries per row)
        n = scale or 1_000_000
        rp, ci, v = powerlaw(n, seed_pattern=5, seed_values=6, symmetrize=False)
        return dict(name=f"powerlaw_nonsym_n{n}", rowptr=rp, colidx=ci, vals=v,
                    b=rhs(n, 1, seed=9), dtype="f64")
    if name == "c5":
        m = scale or 1024
        rp, ci, v = aniso5(m, 0.01)
        return dict(name=f"aniso5_{m}x{m}_eps0.01", rowptr=rp, colidx=ci, vals=v,
                    b=rhs(m * m, 32, seed=7), g=rhs(m * m, 32, seed=8), dtype="f32",
                    grid=(m, m, 1))
    raise KeyError(name)
