"""Shared helpers for the GPU parity tests (no arithmetic of the method here)."""
import numpy as np

import workloads as W


SCHEDULES = ("level", "syncfree", "band")


def analyze(jv, rowptr, colidx, schedule, **kw):
    """Handle for one schedule: 'level' (one launch per level), 'syncfree'
    (one persistent launch over level-ordered tasks), 'band' (sync-free band
    schedule, forced with a small band so it meets every pattern).  The
    handle divides by every pivot as the serial algorithm does
    (exact) unless the caller asks otherwise: the bit-exact tests
    compare that mode with the oracle, the tests of the default mode pass
    exact=False and compare within tolerance."""
    import torch
    kw.setdefault("exact", True)
    rp = torch.tensor(np.asarray(rowptr), device="cuda")
    ci = torch.tensor(np.asarray(colidx), device="cuda")
    if schedule == "level":
        return jv.jv_analyze(rp, ci, mode="level", **kw)
    if schedule == "syncfree":
        return jv.jv_analyze(rp, ci, mode="syncfree", band_rows=-1, **kw)
    return jv.jv_analyze(rp, ci, mode="syncfree", band_rows=kw.pop("band_rows", 64), **kw)


def close(got, want, rel=1e-12, floor_frac=1e-6):
    """Per-entry bound |g - o| <= rel * max(|o|, floor_frac * max|o|): relative
    error per entry, with a floor for entries that cancelled to near zero
    (the floor scale is the largest magnitude of the reference)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.maximum(np.abs(want), floor_frac * (np.abs(want).max() if want.size else 0.0))
    err = np.abs(got - want)
    bad = err > rel * scale
    return not bad.any(), float((err / np.where(scale > 0, scale, 1.0)).max() if want.size else 0.0)


def abs_factor(lu, diag):
    """|L| and |U| for the absolute-value recurrences of solve_scale:
    off-diagonal entries -|t|, diagonal |u_ii| (plain numpy)."""
    out = -np.abs(np.asarray(lu, dtype=np.float64))
    out[diag] = np.abs(np.asarray(lu, dtype=np.float64)[diag])
    return out


def solve_scale(solve, rowptr, colidx, diag, lu, b):
    """Per-entry magnitude of a triangular solve's terms: the same solve
    run on |b| with every off-diagonal entry -|t| and the diagonal |u_ii|, i.e.
    s_r = (|b_r| + sum_j |t_rj| s_j) [/ |u_rr|].  A solve that adds its rows'
    terms in another order (long rows summed by lanes and a tree) differs from
    the serial one by rounding relative to s_r, and by that much only: the
    componentwise bound of a triangular solve.  `solve` is the oracle's."""
    return solve(rowptr, colidx, diag, abs_factor(lu, diag), np.abs(np.asarray(b, dtype=np.float64)))


def close_scaled(got, want, scale, rel=1e-12):
    """|g - o| <= rel * max(|o|, s) per entry, s from solve_scale."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    ref = np.maximum(np.abs(want), np.asarray(scale, dtype=np.float64))
    err = np.abs(got - want)
    worst = float((err / np.where(ref > 0, ref, 1.0)).max()) if want.size else 0.0
    return not (err > rel * ref).any(), worst


def max_rel(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def tridiag(n, d=4.0, o=-1.0):
    rp = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        for j, v in ((i - 1, o), (i, d), (i + 1, o)):
            if 0 <= j < n:
                cols.append(j)
                vals.append(v)
        rp[i + 1] = len(cols)
    return rp, np.array(cols, dtype=np.int32), np.array(vals)


def dense_lower(n, seed=0):
    """Full lower triangle + diagonal + a superdiagonal: every row depends on all before it."""
    rng = np.random.default_rng(seed)
    rp = [0]
    cols, vals = [], []
    for i in range(n):
        for j in range(0, min(i + 2, n)):
            cols.append(j)
            vals.append(rng.uniform(-1, 1) if j != i else float(n + 1))
        rp.append(len(cols))
    return np.array(rp, dtype=np.int32), np.array(cols, dtype=np.int32), np.array(vals)


def small_matrices():
    """(name, rowptr, colidx, vals): small cases that span several tiles,
    ragged tails, long chains and degenerate shapes."""
    out = []
    for seed, (n, k, sym) in enumerate([(1, 0, False), (2, 1, False), (37, 3.0, False),
                                        (250, 4.0, True), (600, 6.0, False), (1500, 2.5, False)]):
        rp, ci, v = W.random_csr(n, k, seed=40 + seed, symmetric_pattern=sym)
        out.append((f"rand{n}", rp, ci, v))
    rp, ci, v = tridiag(3000)
    out.append(("tridiag3000", rp, ci, v))
    rp, ci, v = dense_lower(90, seed=3)
    out.append(("denselower90", rp, ci, v))
    n = 700
    out.append(("diagonal700", np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                np.linspace(1.0, 2.0, n)))
    rp, ci, v = W.lap5(33)
    out.append(("lap5_33", rp, ci, v))
    rp, ci, v = W.lap7(13)
    out.append(("lap7_13", rp, ci, v))
    rp, ci, v, _ = W.cd27(7)
    out.append(("cd27_7", rp, ci, v))
    rp, ci, v = W.aniso5(41)
    out.append(("aniso5_41", rp, ci, v))
    rp, ci, v = W.powerlaw(6000, kmax=400, seed_pattern=11, seed_values=12)
    out.append(("powerlaw6000", rp, ci, v))
    # 20 dependencies per row: one-lane rows that span several poll windows
    rp, ci, v = W.stencil((800, 1, 1), [(-d, 0, 0) for d in range(20, 0, -1)] +
                          [(d, 0, 0) for d in range(1, 21)], [-0.02] * 40, 1.0)
    out.append(("band20_800", rp, ci, v))
    return out
