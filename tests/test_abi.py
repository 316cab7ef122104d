"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/fmm_gb300.h declares (no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "fmm_gb300.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_13218_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fmm_plan_create", "fmm_energy", "fmm_forces", "fmm_solute_solvent_energy", "fmm_plan_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings_and_null_handling(lib):
    lib.fmm_status_string.restype = ctypes.c_char_p
    lib.fmm_status_string.argtypes = [ctypes.c_int]
    assert lib.fmm_status_string(0) == b"ok"
    assert b"invalid" in lib.fmm_status_string(1)
    lib.fmm_plan_destroy.argtypes = [ctypes.c_void_p]
    lib.fmm_plan_destroy(None)  # accepts NULL
    lib.fmm_plan_last_launch_count.argtypes = [ctypes.c_void_p]
    lib.fmm_plan_last_launch_count.restype = ctypes.c_int64
    assert lib.fmm_plan_last_launch_count(None) == -1
    lib.fmm_plan_create.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    lib.fmm_plan_create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    # argument validation happens before any CUDA call
    assert lib.fmm_plan_create(-1.0, 10, 3, 4, ctypes.byref(h)) == 1
    assert lib.fmm_plan_create(1.0, 10, 3, 99, ctypes.byref(h)) == 1
    assert lib.fmm_plan_create(1.0, 10, 3, 4, None) == 1
    lib.fmm_batch_set_option.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double]
    lib.fmm_batch_set_option.restype = ctypes.c_int
    assert lib.fmm_batch_set_option(None, 1, 1, 0.0) == 1
    lib.fmm_batch_sweep_info.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.fmm_batch_sweep_info.restype = ctypes.c_int
    assert lib.fmm_batch_sweep_info(None, None, None) == 1


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2003_13218_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
