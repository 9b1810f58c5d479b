"""GB300 (sm_103a) implementation of the Javelin hot path (arXiv 1812.06160):
level-scheduled / sync-free ILU(0), sparse triangular solves, CSR spmv and the
GPU dependency analysis, behind the C ABI of ``include/jv.h``.

The Python layer is a thin ctypes binding (``_jv``) plus a
``torch.autograd.Function`` for the differentiable preconditioner apply
(``autograd``).  Build the shared library with
``python -m paper_1812_06160_gb300.build``; importing any binding name before
that raises ImportError (there is no CPU fallback).
"""
import importlib

_BINDING = ("JV_OK", "JV_ERR_ARG", "JV_ERR_PATTERN", "JV_ERR_NO_DIAG", "JV_ERR_ZERO_PIVOT",
            "JV_ERR_TIMEOUT", "JV_ERR_CUDA", "JV_ERR_NOMEM", "JV_ERR_INTERNAL",
            "JV_ERR_NOT_CONVERGED", "LIB_PATH", "Handle", "JvError", "jv_analyze", "jv_destroy",
            "jv_set_mode", "jv_set_check", "jv_ilu0_factor", "jv_lsolve", "jv_usolve",
            "jv_lsolve_t", "jv_usolve_t", "jv_spmv", "jv_masked_outer", "jv_permute_values",
            "jv_permute_vector", "jv_get_info", "jv_get_levels", "jv_get_pattern", "jv_get_csc",
            "jv_get_perm", "jv_status_sync", "jv_pcg", "jv_fgmres", "jv_launch_count",
            "jv_status_string", "jv_lsolve_noalloc", "jv_hop_latency",
            "jv_iluk_symbolic", "jv_scatter_values", "jv_stage_plan")
__all__ = list(_BINDING) + ["IluApply", "ilu_apply"]


def __getattr__(name):
    if name in _BINDING:
        return getattr(importlib.import_module("._jv", __name__), name)
    if name in ("IluApply", "ilu_apply"):
        return getattr(importlib.import_module(".autograd", __name__), name)
    raise AttributeError(name)
