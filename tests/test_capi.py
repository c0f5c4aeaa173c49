"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (CPU only)."""
import ctypes
import os
import re

import paper_2006_15367_gb300 as mf
from paper_2006_15367_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mlfma.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mlfma_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    lib_path = _build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert "mlfma_plan_create" in names and "mlfma_apply" in names and "mlfma_apply_adjoint" in names
    assert "mlfma_destroy" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_options_defaults_without_gpu():
    o = mf.mlfma_options_init()
    assert o.struct_size == ctypes.sizeof(mf.Options)
    assert o.precision == mf.PREC_FP32 and o.max_depth == 12 and o.digit_margin == -1


def test_invalid_arguments_rejected_before_any_device_work():
    lib = mf.load()
    h = ctypes.c_void_p()
    pts = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    assert lib.mlfma_plan_create(None, 1, 1.0, 3, 0, None, ctypes.byref(h)) == 1
    assert lib.mlfma_plan_create(pts, 0, 1.0, 3, 0, None, ctypes.byref(h)) == 1
    assert lib.mlfma_plan_create(pts, 1, -1.0, 3, 0, None, ctypes.byref(h)) == 1
    assert lib.mlfma_plan_create(pts, 1, float("nan"), 3, 0, None, ctypes.byref(h)) == 1
    assert lib.mlfma_plan_create(pts, 1, 1.0, 0, 0, None, ctypes.byref(h)) == 1
    assert lib.mlfma_plan_create(pts, 1, 1.0, 13, 0, None, ctypes.byref(h)) == 1
    assert lib.mlfma_plan_create(pts, 1, 1.0, 3, -1, None, ctypes.byref(h)) == 1
    assert h.value is None
    assert "digits" in mf.mlfma_last_error() or "leaf_max" in mf.mlfma_last_error()
    assert lib.mlfma_apply(None, None, None, 1) == 1
    lib.mlfma_destroy(None)
