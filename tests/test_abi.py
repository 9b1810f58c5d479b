"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports
every entry point declared in include/jv.h, and the binding rejects host
tensors before any call reaches the library (no compute without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "jv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jv_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_06160_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path():
    names = _declared()
    for must in ("jv_analyze", "jv_ilu0_factor", "jv_lsolve", "jv_usolve", "jv_spmv",
                 "jv_lsolve_t", "jv_usolve_t", "jv_masked_outer", "jv_pcg", "jv_fgmres",
                 "jv_destroy", "jv_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_pure_host_entry_points(lib):
    lib.jv_status_string.restype = ctypes.c_char_p
    assert lib.jv_status_string(0) == b"ok"
    assert b"pivot" in lib.jv_status_string(-4)
    lib.jv_launch_count.restype = ctypes.c_ulonglong
    assert lib.jv_launch_count() == 0


def test_binding_rejects_host_tensors(lib):
    import paper_1812_06160_gb300 as jv
    rp = torch.tensor([0, 1], dtype=torch.int32)
    ci = torch.tensor([0], dtype=torch.int32)
    with pytest.raises(ValueError, match="CUDA tensor"):
        jv.jv_analyze(rp, ci)


def test_binding_option_struct_layout(lib):
    from paper_1812_06160_gb300 import _jv
    opt = _jv.jv_options()
    lib.jv_default_options(ctypes.byref(opt))
    assert (opt.mode, opt.reorder, opt.check, opt.fault_row) == (1, 0, 1, -1)
    ko = _jv.jv_krylov_opts()
    lib.jv_default_krylov_opts(ctypes.byref(ko))
    assert (ko.tol, ko.maxit, ko.restart, ko.max_restarts) == (1e-8, 10000, 30, 200)
    assert np.dtype(np.int32).itemsize == ctypes.sizeof(ctypes.c_int)
    assert (opt.sf_gate_levels, opt.stage_min_rows, opt.stage_max_density,
            opt.stage_position, opt.er_corner) == (-1, 0, 0.0, 0.0, 0)
    # the C struct is no larger than the binding's: jv_default_options writes
    # nothing past ctypes.sizeof (a canary after the struct survives)
    size = ctypes.sizeof(_jv.jv_options)
    buf = (ctypes.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    lib.jv_default_options(ctypes.byref(buf))
    assert bytes(buf[size:]) == b"\xab" * 64
