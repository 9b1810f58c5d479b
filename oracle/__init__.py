"""Serial FP64 CPU oracle for the Javelin hot path (arXiv 1812.06160).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product path (``paper_1812_06160_gb300``) never imports it and shares no code
with it.

The arithmetic lives in ``jv_oracle.c`` (plain C).  Every update
``s <- s -/+ a*b`` there is one explicit fused multiply-add (C99 ``fma`` /
``fmaf``: the product is not rounded on its own); every division and every
other operation rounds separately, and the file is compiled with
``-ffp-contract=off`` so that the compiler fuses nothing else.  This
module compiles it on first use with the system C compiler and exposes numpy
wrappers.  Each wrapper names the paper passage its C function follows.

Every function here is pinned by ``tests/test_oracle_pins.py`` against
closed forms, library routines, exact rational arithmetic or brute force.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jv_oracle.c")
_LIB = os.path.join(_HERE, f"libjv_oracle_{platform.machine()}.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_PATTERN, ERR_NO_DIAG, ERR_ZERO_PIVOT = 0, -1, -2, -3, -4

_I = ctypes.c_int
_P = ctypes.c_void_p
_D = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, no GPU)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                   "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        sigs = {
            "jvo_validate": [_I, _I, _P, _P, _P, _P],
            "jvo_levels_longest_path": [_I, _P, _P, _I, _P],
            "jvo_levels_peel": [_I, _P, _P, _I, _P],
            "jvo_bucket_levels": [_I, _P, _I, _P, _P],
            "jvo_transpose": [_I, _P, _P, _P, _P, _P],
            "jvo_permute": [_I, _P, _P, _P, _P, _P, _P, _P],
            "jvo_ilu0": [_I, _P, _P, _P, _P, _P],
            "jvo_ilu0_f32": [_I, _P, _P, _P, _P, _P],
            "jvo_milu0": [_I, _P, _P, _P, _P, _P],
            "jvo_milu0_f32": [_I, _P, _P, _P, _P, _P],
            "jvo_iluk_symbolic": [_I, _P, _P, _I, ctypes.c_longlong, _P, _P, _P],
            "jvo_lsolve": [_I, _P, _P, _P, _P, _P, _P, _I],
            "jvo_usolve": [_I, _P, _P, _P, _P, _P, _P, _I],
            "jvo_lsolve_t": [_I, _P, _P, _P, _P, _P, _P, _I],
            "jvo_usolve_t": [_I, _P, _P, _P, _P, _P, _P, _I],
            "jvo_masked_outer": [_I, _P, _P, _P, _I, _P, _P, _I, _D, _P],
            "jvo_spmv": [_I, _P, _P, _P, _P, _P, _D, _D],
            "jvo_pcg": [_I, _P, _P, _P, _P, _P, _P, _P, _D, _I, _P],
            "jvo_fgmres": [_I, _P, _P, _P, _P, _P, _P, _P, _I, _D, _I, _P],
        }
        for name, args in sigs.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = None if name in ("jvo_bucket_levels", "jvo_transpose", "jvo_permute",
                                         "jvo_lsolve", "jvo_usolve", "jvo_lsolve_t",
                                         "jvo_usolve_t", "jvo_masked_outer", "jvo_spmv") else _I
        lib.jvo_iluk_symbolic.restype = ctypes.c_longlong
        _lib = lib
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, status, row):
        super().__init__(f"oracle status {status} at row {row}")
        self.status = status
        self.row = row


# --------------------------------------------------------------------------
# Analysis (Sec. II level scheduling, Sec. III-A upper stage)
# --------------------------------------------------------------------------
def validate(rowptr, colidx):
    """Return (status, diag, bad_row).  Sec. III, Fig. 1 needs ascending
    columns and a stored diagonal."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    n = len(rowptr) - 1
    diag = np.full(max(n, 1), -1, dtype=np.int32)
    bad = np.zeros(1, dtype=np.int32)
    st = _load().jvo_validate(n, len(colidx), _ptr(rowptr), _ptr(colidx), _ptr(diag), _ptr(bad))
    return st, diag[:n], int(bad[0])


def diag_ptr(rowptr, colidx):
    st, diag, bad = validate(rowptr, colidx)
    if st != OK:
        raise OracleError(st, bad)
    return diag


def levels(rowptr, colidx, upper=False, route="longest_path"):
    """Level of every row: longest dependency path (route='longest_path') or
    peeling of dependency-free vertices (route='peel').  Returns (lev, nlev)."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    n = len(rowptr) - 1
    lev = np.zeros(n, dtype=np.int32)
    fn = _load().jvo_levels_longest_path if route == "longest_path" else _load().jvo_levels_peel
    nlev = fn(n, _ptr(rowptr), _ptr(colidx), int(bool(upper)), _ptr(lev))
    if nlev < 0:
        raise OracleError(nlev, -1)
    return lev, int(nlev)


def bucket_levels(lev, nlev):
    """(level_ptr, level_rows): rows grouped by level, ascending inside."""
    lev = _i32(lev)
    n = len(lev)
    level_ptr = np.zeros(nlev + 1, dtype=np.int32)
    level_rows = np.zeros(n, dtype=np.int32)
    _load().jvo_bucket_levels(n, _ptr(lev), int(nlev), _ptr(level_ptr), _ptr(level_rows))
    return level_ptr, level_rows


def level_sets(rowptr, colidx, upper=False):
    lev, nlev = levels(rowptr, colidx, upper)
    ptr, rows = bucket_levels(lev, nlev)
    return lev, nlev, ptr, rows


def transpose(rowptr, colidx):
    """(colptr, rowidx, csc2csr) of the pattern, rows ascending per column."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    n = len(rowptr) - 1
    nnz = len(colidx)
    colptr = np.zeros(n + 1, dtype=np.int32)
    rowidx = np.zeros(max(nnz, 1), dtype=np.int32)
    c2c = np.zeros(max(nnz, 1), dtype=np.int32)
    _load().jvo_transpose(n, _ptr(rowptr), _ptr(colidx), _ptr(colptr), _ptr(rowidx), _ptr(c2c))
    return colptr, rowidx[:nnz], c2c[:nnz]


def transposed_level_sets(rowptr, colidx, which):
    """Level sets of the transposed solves: which='Ut' (forward over the
    columns of U) or 'Lt' (backward over the columns of L).  Their dependency
    DAGs are those of lower(A^T) and upper(A^T)."""
    colptr, rowidx, _ = transpose(rowptr, colidx)
    return level_sets(colptr, rowidx, upper=(which == "Lt"))


def permute(rowptr, colidx, perm):
    """B = P A P^T: (iperm, browptr, bcolidx, vmap)."""
    rowptr, colidx, perm = _i32(rowptr), _i32(colidx), _i32(perm)
    n = len(rowptr) - 1
    nnz = len(colidx)
    iperm = np.zeros(n, dtype=np.int32)
    browptr = np.zeros(n + 1, dtype=np.int32)
    bcol = np.zeros(max(nnz, 1), dtype=np.int32)
    vmap = np.zeros(max(nnz, 1), dtype=np.int32)
    _load().jvo_permute(n, _ptr(rowptr), _ptr(colidx), _ptr(perm), _ptr(iperm),
                        _ptr(browptr), _ptr(bcol), _ptr(vmap))
    return iperm, browptr, bcol[:nnz], vmap[:nnz]


# --------------------------------------------------------------------------
# Numeric factorisation (Sec. III, Fig. 1) and applies (Sec. VI)
# --------------------------------------------------------------------------
def ilu0(rowptr, colidx, vals, diag=None, dtype=np.float64, milu=False):
    """ILU(0) in place on a copy of vals; returns (lu, status, bad_row).
    milu=True: modified ILU(0), dropped fill-in applied to the diagonal."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    n = len(rowptr) - 1
    if diag is None:
        diag = diag_ptr(rowptr, colidx)
    diag = _i32(diag)
    bad = np.zeros(1, dtype=np.int32)
    if dtype == np.float32:
        a = np.array(vals, dtype=np.float32, copy=True)
        fn = _load().jvo_milu0_f32 if milu else _load().jvo_ilu0_f32
        st = fn(n, _ptr(rowptr), _ptr(colidx), _ptr(diag), _ptr(a), _ptr(bad))
    else:
        a = np.array(vals, dtype=np.float64, copy=True)
        fn = _load().jvo_milu0 if milu else _load().jvo_ilu0
        st = fn(n, _ptr(rowptr), _ptr(colidx), _ptr(diag), _ptr(a), _ptr(bad))
    return a, st, int(bad[0])


def iluk_pattern(rowptr, colidx, level):
    """ILU(k) level-of-fill pattern: (rowptr, colidx, lev) of the filled
    pattern, columns ascending, lev[p] the level of fill of every entry."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    n = len(rowptr) - 1
    cap = max(2 * len(colidx), 16)
    while True:
        frp = np.zeros(n + 1, dtype=np.int32)
        fci = np.zeros(cap, dtype=np.int32)
        flev = np.zeros(cap, dtype=np.int32)
        nz = _load().jvo_iluk_symbolic(n, _ptr(rowptr), _ptr(colidx), int(level), cap, _ptr(frp),
                                       _ptr(fci), _ptr(flev))
        if nz >= 0:
            return frp, fci[:nz].copy(), flev[:nz].copy()
        cap *= 2


def scatter_values(rowptr, colidx, vals, frowptr, fcolidx):
    """A's values placed on a pattern that contains A's (zeros elsewhere)."""
    n = len(rowptr) - 1
    out = np.zeros(len(fcolidx), dtype=np.asarray(vals).dtype)
    for i in range(n):
        f0, f1 = frowptr[i], frowptr[i + 1]
        pos = np.searchsorted(fcolidx[f0:f1], colidx[rowptr[i]:rowptr[i + 1]])
        out[f0 + pos] = vals[rowptr[i]:rowptr[i + 1]]
    return out


def _solve(name, rowptr, colidx, diag, lu, b):
    rowptr, colidx, diag, lu = _i32(rowptr), _i32(colidx), _i32(diag), _f64(lu)
    b = _f64(b)
    n = len(rowptr) - 1
    nrhs = 1 if b.ndim == 1 else b.shape[1]
    x = np.zeros_like(b)
    getattr(_load(), name)(n, _ptr(rowptr), _ptr(colidx), _ptr(diag), _ptr(lu), _ptr(b), _ptr(x), nrhs)
    return x


def lsolve(rowptr, colidx, diag, lu, b):
    """x = L^-1 b (unit lower; forward substitution)."""
    return _solve("jvo_lsolve", rowptr, colidx, diag, lu, b)


def usolve(rowptr, colidx, diag, lu, b):
    """x = U^-1 b (backward substitution)."""
    return _solve("jvo_usolve", rowptr, colidx, diag, lu, b)


def lsolve_t(rowptr, colidx, diag, lu, b):
    """x = L^-T b."""
    return _solve("jvo_lsolve_t", rowptr, colidx, diag, lu, b)


def usolve_t(rowptr, colidx, diag, lu, b):
    """x = U^-T b."""
    return _solve("jvo_usolve_t", rowptr, colidx, diag, lu, b)


def masked_outer(rowptr, colidx, diag, which, a, b, alpha=1.0):
    """g_p = alpha * sum_c a[i,c] b[j,c] on the strict lower (which=0) or
    upper-with-diagonal (which=1) part; zeros elsewhere."""
    rowptr, colidx, diag = _i32(rowptr), _i32(colidx), _i32(diag)
    a, b = _f64(a), _f64(b)
    n = len(rowptr) - 1
    nrhs = 1 if a.ndim == 1 else a.shape[1]
    g = np.zeros(len(colidx), dtype=np.float64)
    _load().jvo_masked_outer(n, _ptr(rowptr), _ptr(colidx), _ptr(diag), int(which),
                             _ptr(a), _ptr(b), nrhs, float(alpha), _ptr(g))
    return g


def spmv(rowptr, colidx, vals, x, y=None, alpha=1.0, beta=0.0):
    rowptr, colidx, vals, x = _i32(rowptr), _i32(colidx), _f64(vals), _f64(x)
    n = len(rowptr) - 1
    out = np.zeros(n, dtype=np.float64) if y is None else np.array(y, dtype=np.float64, copy=True)
    _load().jvo_spmv(n, _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(x), _ptr(out),
                     float(alpha), float(beta))
    return out


def pcg(rowptr, colidx, vals, lu, b, tol=1e-8, maxit=10000, x0=None, diag=None):
    """Flexible ILU(0)-preconditioned CG.  Returns (x, iters, relres)."""
    rowptr, colidx, vals, lu, b = _i32(rowptr), _i32(colidx), _f64(vals), _f64(lu), _f64(b)
    n = len(rowptr) - 1
    diag = _i32(diag_ptr(rowptr, colidx) if diag is None else diag)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    rel = np.zeros(1)
    it = _load().jvo_pcg(n, _ptr(rowptr), _ptr(colidx), _ptr(diag), _ptr(vals), _ptr(lu),
                         _ptr(b), _ptr(x), float(tol), int(maxit), _ptr(rel))
    return x, int(it), float(rel[0])


def fgmres(rowptr, colidx, vals, lu, b, m=30, tol=1e-8, max_restarts=200, x0=None, diag=None):
    """Right-preconditioned flexible GMRES(m).  Returns (x, iters, relres)."""
    rowptr, colidx, vals, lu, b = _i32(rowptr), _i32(colidx), _f64(vals), _f64(lu), _f64(b)
    n = len(rowptr) - 1
    diag = _i32(diag_ptr(rowptr, colidx) if diag is None else diag)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    rel = np.zeros(1)
    it = _load().jvo_fgmres(n, _ptr(rowptr), _ptr(colidx), _ptr(diag), _ptr(vals), _ptr(lu),
                            _ptr(b), _ptr(x), int(m), float(tol), int(max_restarts), _ptr(rel))
    return x, int(it), float(rel[0])
