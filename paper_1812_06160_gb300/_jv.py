"""ctypes binding of libjavelin_gb (include/jv.h).

Argument marshalling only: every function checks the torch tensors it is
given (device, dtype, contiguity, size), passes their device pointers and the
current torch CUDA stream to the C entry point of the same name, and raises
``JvError`` on a non-zero status.  Every computation runs in the library's
CUDA kernels; there is no CPU fallback -- if the shared library is missing the
import of this module fails with instructions to build it.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libjavelin_gb.so")

JV_OK = 0
JV_ERR_ARG = -1
JV_ERR_PATTERN = -2
JV_ERR_NO_DIAG = -3
JV_ERR_ZERO_PIVOT = -4
JV_ERR_TIMEOUT = -5
JV_ERR_CUDA = -6
JV_ERR_NOMEM = -7
JV_ERR_INTERNAL = -8
JV_ERR_NOT_CONVERGED = -9

JV_F64, JV_F32 = 0, 1
JV_MODE_LEVEL, JV_MODE_SYNCFREE, JV_MODE_HYBRID = 0, 1, 2
MODES = {"level": JV_MODE_LEVEL, "syncfree": JV_MODE_SYNCFREE, "hybrid": JV_MODE_HYBRID}
JV_LOWER, JV_UPPER, JV_UPPER_T, JV_LOWER_T = 0, 1, 2, 3
STRUCTURES = {"L": JV_LOWER, "U": JV_UPPER, "Ut": JV_UPPER_T, "Lt": JV_LOWER_T}


class jv_options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("reorder", ctypes.c_int), ("check", ctypes.c_int),
                ("long_row", ctypes.c_int),
                ("spin_timeout_cycles", ctypes.c_longlong), ("fault_row", ctypes.c_int),
                ("sf_ctas_per_sm", ctypes.c_int), ("sf_backoff_ns", ctypes.c_int),
                ("band_rows", ctypes.c_int), ("sf_gate_levels", ctypes.c_int),
                ("milu", ctypes.c_int), ("sym_levels", ctypes.c_int),
                ("stage_min_rows", ctypes.c_int), ("stage_max_density", ctypes.c_double),
                ("stage_position", ctypes.c_double), ("er_corner", ctypes.c_int),
                ("no_graphs", ctypes.c_int), ("exact", ctypes.c_int),
                ("spmv_long_row", ctypes.c_int)]


class jv_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nnz", ctypes.c_int), ("nnz_lower", ctypes.c_int),
                ("nnz_upper", ctypes.c_int), ("nlev", ctypes.c_int * 4),
                ("nlong", ctypes.c_int * 4), ("nlong_factor", ctypes.c_int),
                ("band_rows", ctypes.c_int * 4), ("nband_levels", ctypes.c_int * 4),
                ("npairs", ctypes.c_longlong), ("mode", ctypes.c_int), ("reorder", ctypes.c_int),
                ("hybrid_launches", ctypes.c_int * 4), ("hybrid_launches_factor", ctypes.c_int),
                ("corner_rows", ctypes.c_int * 2), ("corner_levels", ctypes.c_int * 2),
                ("solve_corner_rows", (ctypes.c_int * 2) * 4),
                ("spmv_wide_rows", ctypes.c_int)]


class jv_krylov_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("restart", ctypes.c_int),
                ("max_restarts", ctypes.c_int)]


class jv_krylov_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("relres", ctypes.c_double), ("true_relres", ctypes.c_double)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_1812_06160_gb300.build` (needs nvcc, sm_103a)")

lib = ctypes.CDLL(LIB_PATH)

_v, _i, _d, _ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
_pi = ctypes.POINTER(ctypes.c_int)
_pp = ctypes.POINTER(ctypes.c_void_p)
_SIGS = {
    "jv_default_options": (None, [ctypes.POINTER(jv_options)]),
    "jv_stage_plan": (_i, [_i, _v, _v, _i, ctypes.POINTER(jv_options), _v, ctypes.POINTER(_i)]),
    "jv_default_krylov_opts": (None, [ctypes.POINTER(jv_krylov_opts)]),
    "jv_analyze": (_i, [_i, _i, _v, _v, ctypes.POINTER(jv_options), _v, _pp]),
    "jv_last_bad_row": (_i, []),
    "jv_destroy": (None, [_v]),
    "jv_set_stream": (_i, [_v, _v]),
    "jv_set_mode": (_i, [_v, _i]),
    "jv_set_check": (_i, [_v, _i]),
    "jv_ilu0_factor": (_i, [_v, _i, _v, _i, _v, _pi]),
    "jv_lsolve": (_i, [_v, _i, _v, _i, _v, _i, _v, _i]),
    "jv_usolve": (_i, [_v, _i, _v, _i, _v, _i, _v, _i]),
    "jv_lsolve_t": (_i, [_v, _i, _v, _i, _v, _i, _v, _i]),
    "jv_usolve_t": (_i, [_v, _i, _v, _i, _v, _i, _v, _i]),
    "jv_spmv": (_i, [_v, _i, _v, _v, _v, _d, _d]),
    "jv_masked_outer": (_i, [_v, _i, _i, _v, _v, _i, _d, _v]),
    "jv_permute_values": (_i, [_v, _i, _v, _v]),
    "jv_permute_vector": (_i, [_v, _i, _i, _v, _v, _i]),
    "jv_get_info": (_i, [_v, ctypes.POINTER(jv_info)]),
    "jv_get_levels": (_i, [_v, _i, _pi, _pp, _pp, _pp]),
    "jv_get_pattern": (_i, [_v, _pp, _pp, _pp]),
    "jv_get_csc": (_i, [_v, _pp, _pp, _pp, _pp]),
    "jv_get_perm": (_i, [_v, _pp, _pp, _pp]),
    "jv_status_sync": (_i, [_v, _pi]),
    "jv_pcg": (_i, [_v, _v, _i, _v, _v, _v, ctypes.POINTER(jv_krylov_opts),
                    ctypes.POINTER(jv_krylov_info)]),
    "jv_fgmres": (_i, [_v, _v, _i, _v, _v, _v, ctypes.POINTER(jv_krylov_opts),
                       ctypes.POINTER(jv_krylov_info)]),
    "jv_lsolve_noalloc": (_i, [_i, _v, _v, _v, _v, _v, _v, _v, _v]),
    "jv_hop_latency": (_i, [_i, _i, ctypes.POINTER(ctypes.c_double), _v]),
    "jv_iluk_symbolic": (_i, [_i, _i, _v, _v, _i, _v, _v, _v, ctypes.POINTER(ctypes.c_longlong),
                              _pi, _v]),
    "jv_scatter_values": (_i, [_i, _v, _v, _i, _v, _v, _v, _v, _v]),
    "jv_launch_count": (ctypes.c_ulonglong, []),
    "jv_status_string": (ctypes.c_char_p, [_i]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class JvError(RuntimeError):
    def __init__(self, func, status, bad_row=-1):
        msg = lib.jv_status_string(status).decode()
        super().__init__(f"{func}: {msg} (status {status}" +
                         (f", row {bad_row})" if bad_row is not None and bad_row >= 0 else ")"))
        self.status = status
        self.bad_row = bad_row


def _check(func, status, bad_row=-1):
    if status != JV_OK:
        raise JvError(func, status, bad_row)


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return JV_F64
    if t.dtype == torch.float32:
        return JV_F32
    raise TypeError(f"values must be float64 or float32, got {t.dtype}")


def _torch_dtype(code):
    return torch.float64 if code == JV_F64 else torch.float32


def _dev(t: torch.Tensor, name: str, numel=None, dtype=None) -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (libjavelin_gb has no CPU path)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _stream(h):
    s = torch.cuda.current_stream(h.device).cuda_stream
    lib.jv_set_stream(h.ptr, ctypes.c_void_p(s))


class _DevView:
    """Zero-copy view of a handle-owned int32 device array."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, False),
                                         "version": 3, "strides": None}


def _view(ptr, n, device):
    if not ptr or n <= 0:
        return None
    return torch.as_tensor(_DevView(ptr, n), device=device)


class Handle:
    """Owns a jv_handle (the analysis of one sparsity pattern)."""

    def __init__(self, ptr, n, nnz, device):
        self.ptr = ptr
        self.n = n
        self.nnz = nnz
        self.device = device

    def __del__(self):
        if getattr(self, "ptr", None):
            lib.jv_destroy(self.ptr)
            self.ptr = None

    def info(self):
        return jv_get_info(self)


def jv_analyze(rowptr, colidx, mode="syncfree", reorder=False, check=True, long_row=0,
               spin_timeout_cycles=0, fault_row=-1, sf_ctas_per_sm=0, sf_backoff_ns=0,
               band_rows=0, sf_gate_levels=None, milu=False, sym_levels=False,
               stage_min_rows=0, stage_max_density=0.0, stage_position=0.0, er_corner=False,
               graphs=True, exact=False, spmv_long_row=0):
    """Analyse a CSR pattern (int32 CUDA tensors).  Returns a Handle.
    ``mode``: "level", "syncfree" or "hybrid" (the two-stage split of Sec. III-A,
    with the stage test ``stage_min_rows`` / ``stage_max_density`` /
    ``stage_position``); ``er_corner``: Even-Rows second stage of the factor
    (Sec. III-B); ``graphs``: replay the per-level launch sequences of the
    level and hybrid modes from captured CUDA graphs."""
    n = rowptr.numel() - 1
    nnz = colidx.numel()
    rp = _dev(rowptr, "rowptr", dtype=torch.int32)
    ci = _dev(colidx, "colidx", dtype=torch.int32)
    opt = jv_options()
    lib.jv_default_options(ctypes.byref(opt))
    opt.mode = MODES[mode]
    opt.reorder = int(bool(reorder))
    opt.check = int(bool(check))
    opt.long_row = int(long_row)
    opt.spin_timeout_cycles = int(spin_timeout_cycles)
    opt.fault_row = int(fault_row)
    opt.sf_ctas_per_sm = int(sf_ctas_per_sm)
    opt.sf_backoff_ns = int(sf_backoff_ns)
    opt.band_rows = int(band_rows)
    if sf_gate_levels is not None:
        opt.sf_gate_levels = int(sf_gate_levels)
    opt.milu = int(bool(milu))
    opt.sym_levels = int(bool(sym_levels))
    opt.stage_min_rows = int(stage_min_rows)
    opt.stage_max_density = float(stage_max_density)
    opt.stage_position = float(stage_position)
    opt.er_corner = int(bool(er_corner))
    opt.no_graphs = int(not graphs)
    opt.exact = int(bool(exact))
    opt.spmv_long_row = int(spmv_long_row)
    out = ctypes.c_void_p()
    stream = torch.cuda.current_stream(rowptr.device).cuda_stream
    with torch.cuda.device(rowptr.device):
        st = lib.jv_analyze(n, nnz, rp, ci, ctypes.byref(opt), ctypes.c_void_p(stream),
                            ctypes.byref(out))
    _check("jv_analyze", st, lib.jv_last_bad_row())
    return Handle(out.value, n, nnz, rowptr.device)


def jv_stage_plan(level_ptr, dep_sum=None, stage_min_rows=0, stage_max_density=0.0,
                  stage_position=0.0):
    """The stage test on the host (no GPU): level_ptr[nlev+1] and optional
    per-level dependency sums (numpy).  Returns (upper[nlev] as uint8, tail)."""
    import numpy as np
    lp = np.ascontiguousarray(level_ptr, dtype=np.int32)
    nlev = len(lp) - 1
    ds = None if dep_sum is None else np.ascontiguousarray(dep_sum, dtype=np.int64)
    opt = jv_options()
    lib.jv_default_options(ctypes.byref(opt))
    opt.stage_min_rows = int(stage_min_rows)
    opt.stage_max_density = float(stage_max_density)
    opt.stage_position = float(stage_position)
    upper = np.zeros(max(nlev, 1), dtype=np.uint8)
    tail = ctypes.c_int(-1)
    _check("jv_stage_plan", lib.jv_stage_plan(
        nlev, lp.ctypes.data, None if ds is None else ds.ctypes.data, int(lp[-1]),
        ctypes.byref(opt), upper.ctypes.data, ctypes.byref(tail)))
    return upper[:nlev], tail.value


def jv_destroy(h: Handle):
    h.__del__()


def jv_set_mode(h: Handle, mode: str):
    _check("jv_set_mode", lib.jv_set_mode(h.ptr, MODES[mode]))


def jv_set_check(h: Handle, check: bool):
    _check("jv_set_check", lib.jv_set_check(h.ptr, int(bool(check))))


def jv_ilu0_factor(h: Handle, vals, lu=None, lu_dtype=None):
    """ILU(0) of the values ``vals`` (nnz, float64/float32) into ``lu``.
    ``lu`` may be ``vals`` (in place).  Returns lu."""
    vp = _dev(vals, "vals", numel=h.nnz)
    if lu is None:
        lu = torch.empty(h.nnz, dtype=lu_dtype or vals.dtype, device=vals.device)
    lp = _dev(lu, "lu", numel=h.nnz)
    _stream(h)
    bad = ctypes.c_int(-1)
    st = lib.jv_ilu0_factor(h.ptr, _dt(vals), vp, _dt(lu), lp, ctypes.byref(bad))
    _check("jv_ilu0_factor", st, bad.value)
    return lu


def _solve(name, h, lu, b, x, x_dtype):
    nrhs = 1 if b.dim() == 1 else b.shape[1]
    lp = _dev(lu, "lu", numel=h.nnz)
    bp = _dev(b, "b", numel=h.n * nrhs)
    if x is None:
        x = torch.empty_like(b, dtype=x_dtype or lu.dtype)
    xp = _dev(x, "x", numel=h.n * nrhs)
    _stream(h)
    st = getattr(lib, name)(h.ptr, _dt(lu), lp, _dt(b), bp, _dt(x), xp, nrhs)
    _check(name, st)
    return x


def jv_lsolve(h, lu, b, x=None, x_dtype=None):
    """x = L^-1 b (b: n or n x nrhs row-major)."""
    return _solve("jv_lsolve", h, lu, b, x, x_dtype)


def jv_usolve(h, lu, b, x=None, x_dtype=None):
    """x = U^-1 b."""
    return _solve("jv_usolve", h, lu, b, x, x_dtype)


def jv_lsolve_t(h, lu, b, x=None, x_dtype=None):
    """x = L^-T b."""
    return _solve("jv_lsolve_t", h, lu, b, x, x_dtype)


def jv_usolve_t(h, lu, b, x=None, x_dtype=None):
    """x = U^-T b."""
    return _solve("jv_usolve_t", h, lu, b, x, x_dtype)


def jv_spmv(h, vals, x, y=None, alpha=1.0, beta=0.0):
    """y = alpha A x + beta y."""
    vp = _dev(vals, "vals", numel=h.nnz)
    xp = _dev(x, "x", numel=h.n, dtype=vals.dtype)
    if y is None:
        y = torch.empty_like(x)
        beta = 0.0
    yp = _dev(y, "y", numel=h.n, dtype=vals.dtype)
    _stream(h)
    _check("jv_spmv", lib.jv_spmv(h.ptr, _dt(vals), vp, xp, yp, float(alpha), float(beta)))
    return y


def jv_masked_outer(h, which, a, b, alpha=1.0, g=None):
    """g[p] = alpha sum_c a[i,c] b[j,c] on the strictly lower (which=0) or
    upper-with-diagonal (which=1) entries p = (i, j)."""
    nrhs = 1 if a.dim() == 1 else a.shape[1]
    ap = _dev(a, "a", numel=h.n * nrhs)
    bp = _dev(b, "b", numel=h.n * nrhs, dtype=a.dtype)
    if g is None:
        g = torch.zeros(h.nnz, dtype=a.dtype, device=a.device)
    gp = _dev(g, "g", numel=h.nnz, dtype=a.dtype)
    _stream(h)
    _check("jv_masked_outer", lib.jv_masked_outer(h.ptr, _dt(a), int(which), ap, bp, nrhs,
                                                  float(alpha), gp))
    return g


def jv_permute_values(h, vals, out=None):
    if out is None:
        out = torch.empty_like(vals)
    _stream(h)
    _check("jv_permute_values", lib.jv_permute_values(
        h.ptr, _dt(vals), _dev(vals, "vals", numel=h.nnz), _dev(out, "out", numel=h.nnz)))
    return out


def jv_permute_vector(h, x, inverse=False, out=None):
    nrhs = 1 if x.dim() == 1 else x.shape[1]
    if out is None:
        out = torch.empty_like(x)
    _stream(h)
    _check("jv_permute_vector", lib.jv_permute_vector(
        h.ptr, _dt(x), int(bool(inverse)), _dev(x, "x", numel=h.n * nrhs),
        _dev(out, "out", numel=h.n * nrhs), nrhs))
    return out


def jv_get_info(h):
    info = jv_info()
    _check("jv_get_info", lib.jv_get_info(h.ptr, ctypes.byref(info)))
    return dict(n=info.n, nnz=info.nnz, nnz_lower=info.nnz_lower, nnz_upper=info.nnz_upper,
                nlev=list(info.nlev), nlong=list(info.nlong), nlong_factor=info.nlong_factor,
                band_rows=list(info.band_rows), nband_levels=list(info.nband_levels),
                npairs=info.npairs, mode=info.mode, reorder=info.reorder,
                hybrid_launches=list(info.hybrid_launches),
                hybrid_launches_factor=info.hybrid_launches_factor,
                corner_rows=list(info.corner_rows), corner_levels=list(info.corner_levels),
                solve_corner_rows=[list(r) for r in info.solve_corner_rows],
                spmv_wide_rows=info.spmv_wide_rows)


def jv_get_levels(h, which="L"):
    """(nlev, level_ptr, level_rows, lev) as int32 CUDA tensors (copies)."""
    nlev = ctypes.c_int()
    p, r, l = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check("jv_get_levels", lib.jv_get_levels(h.ptr, STRUCTURES.get(which, which),
                                              ctypes.byref(nlev), ctypes.byref(p),
                                              ctypes.byref(r), ctypes.byref(l)))
    torch.cuda.synchronize(h.device)
    return (nlev.value, _view(p.value, nlev.value + 1, h.device).clone(),
            _view(r.value, h.n, h.device).clone(), _view(l.value, h.n, h.device).clone())


def jv_get_pattern(h):
    """(rowptr, colidx, diag_ptr) copies of the handle's pattern (B when reordered)."""
    rp, ci, dg = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check("jv_get_pattern", lib.jv_get_pattern(h.ptr, ctypes.byref(rp), ctypes.byref(ci),
                                                ctypes.byref(dg)))
    torch.cuda.synchronize(h.device)
    return (_view(rp.value, h.n + 1, h.device).clone(), _view(ci.value, h.nnz, h.device).clone(),
            _view(dg.value, h.n, h.device).clone())


def jv_get_csc(h):
    """(colptr, rowidx, csc2csr, cdiag) copies."""
    a, b, c, d = (ctypes.c_void_p() for _ in range(4))
    _check("jv_get_csc", lib.jv_get_csc(h.ptr, ctypes.byref(a), ctypes.byref(b),
                                        ctypes.byref(c), ctypes.byref(d)))
    torch.cuda.synchronize(h.device)
    return (_view(a.value, h.n + 1, h.device).clone(), _view(b.value, h.nnz, h.device).clone(),
            _view(c.value, h.nnz, h.device).clone(), _view(d.value, h.n, h.device).clone())


def jv_get_perm(h):
    """(perm, iperm, vmap) copies, or Nones without reordering."""
    a, b, c = (ctypes.c_void_p() for _ in range(3))
    _check("jv_get_perm", lib.jv_get_perm(h.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    torch.cuda.synchronize(h.device)
    if not a.value:
        return None, None, None
    return (_view(a.value, h.n, h.device).clone(), _view(b.value, h.n, h.device).clone(),
            _view(c.value, h.nnz, h.device).clone())


def jv_status_sync(h):
    """(status, bad_row) of the work enqueued so far; clears it."""
    _stream(h)
    bad = ctypes.c_int(-1)
    st = lib.jv_status_sync(h.ptr, ctypes.byref(bad))
    return st, bad.value


def _krylov(name, h, vals, lu, b, x, tol, maxit, restart, max_restarts):
    if x is None:
        x = torch.zeros_like(b)
    o = jv_krylov_opts()
    lib.jv_default_krylov_opts(ctypes.byref(o))
    o.tol = float(tol)
    if maxit is not None:
        o.maxit = int(maxit)
    if restart is not None:
        o.restart = int(restart)
    if max_restarts is not None:
        o.max_restarts = int(max_restarts)
    info = jv_krylov_info()
    _stream(h)
    st = getattr(lib, name)(h.ptr, _dev(vals, "vals", numel=h.nnz, dtype=torch.float64), _dt(lu),
                            _dev(lu, "lu", numel=h.nnz), _dev(b, "b", numel=h.n, dtype=torch.float64),
                            _dev(x, "x", numel=h.n, dtype=torch.float64), ctypes.byref(o),
                            ctypes.byref(info))
    res = dict(iters=info.iters, converged=bool(info.converged), relres=info.relres,
               true_relres=info.true_relres, status=st)
    if st not in (JV_OK, JV_ERR_NOT_CONVERGED):
        _check(name, st)
    return x, res


def jv_pcg(h, vals, lu, b, x=None, tol=1e-8, maxit=10000):
    """Flexible ILU(0)-PCG in FP64 with the factor ``lu`` (FP64 or FP32)."""
    return _krylov("jv_pcg", h, vals, lu, b, x, tol, maxit, None, None)


def jv_fgmres(h, vals, lu, b, x=None, tol=1e-8, restart=30, max_restarts=200):
    """Right-preconditioned FGMRES(restart) in FP64 with the factor ``lu``."""
    return _krylov("jv_fgmres", h, vals, lu, b, x, tol, None, restart, max_restarts)


def jv_lsolve_noalloc(rowptr, colidx, diag, order, lu, b, x=None):
    """x = L^-1 b (FP64, one right-hand side) without any device allocation
    by the library; see include/jv.h.  All arguments are CUDA tensors."""
    n = rowptr.numel() - 1
    if x is None:
        x = torch.empty_like(b)
    st = lib.jv_lsolve_noalloc(
        n, _dev(rowptr, "rowptr", dtype=torch.int32), _dev(colidx, "colidx", dtype=torch.int32),
        _dev(diag, "diag", numel=n, dtype=torch.int32), _dev(order, "order", numel=n, dtype=torch.int32),
        _dev(lu, "lu", dtype=torch.float64), _dev(b, "b", numel=n, dtype=torch.float64),
        _dev(x, "x", numel=n, dtype=torch.float64),
        ctypes.c_void_p(torch.cuda.current_stream(b.device).cuda_stream))
    _check("jv_lsolve_noalloc", st)
    return x


def jv_iluk_symbolic(rowptr, colidx, level, with_levels=False):
    """ILU(k) pattern of A's CSR pattern (int32 CUDA tensors): (fill_rowptr,
    fill_colidx[, fill_level]) as int32 CUDA tensors."""
    n = rowptr.numel() - 1
    rp = _dev(rowptr, "rowptr", dtype=torch.int32)
    ci = _dev(colidx, "colidx", dtype=torch.int32)
    frp = torch.empty(n + 1, dtype=torch.int32, device=rowptr.device)
    nnz = ctypes.c_longlong(0)
    bad = ctypes.c_int(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream(rowptr.device).cuda_stream)
    _check("jv_iluk_symbolic", lib.jv_iluk_symbolic(n, colidx.numel(), rp, ci, int(level),
                                                    frp.data_ptr(), None, None, ctypes.byref(nnz),
                                                    ctypes.byref(bad), stream), bad.value)
    fci = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=rowptr.device)
    flev = torch.empty_like(fci) if with_levels else None
    _check("jv_iluk_symbolic", lib.jv_iluk_symbolic(
        n, colidx.numel(), rp, ci, int(level), frp.data_ptr(), fci.data_ptr(),
        flev.data_ptr() if with_levels else None, ctypes.byref(nnz), ctypes.byref(bad), stream),
        bad.value)
    fci = fci[:nnz.value]
    return (frp, fci, flev[:nnz.value]) if with_levels else (frp, fci)


def jv_scatter_values(rowptr, colidx, vals, fill_rowptr, fill_colidx, out=None):
    """A's values on the filled pattern (zeros elsewhere)."""
    n = rowptr.numel() - 1
    if out is None:
        out = torch.empty(fill_colidx.numel(), dtype=vals.dtype, device=vals.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream(vals.device).cuda_stream)
    _check("jv_scatter_values", lib.jv_scatter_values(
        n, _dev(rowptr, "rowptr", dtype=torch.int32), _dev(colidx, "colidx", dtype=torch.int32),
        _dt(vals), _dev(vals, "vals", numel=colidx.numel()),
        _dev(fill_rowptr, "fill_rowptr", dtype=torch.int32),
        _dev(fill_colidx, "fill_colidx", dtype=torch.int32),
        _dev(out, "out", numel=fill_colidx.numel(), dtype=vals.dtype), stream))
    return out


def jv_hop_latency(rounds=1000, npartners=16, device=None) -> float:
    """Median one-way latency (microseconds) of a value published by one SM
    and polled by another: the unit step of the sync-free critical path."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    out = ctypes.c_double(0.0)
    _check("jv_hop_latency", lib.jv_hop_latency(int(rounds), int(npartners), ctypes.byref(out),
                                                ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)))
    return out.value


def jv_launch_count() -> int:
    return int(lib.jv_launch_count())


def jv_status_string(status: int) -> str:
    return lib.jv_status_string(int(status)).decode()
