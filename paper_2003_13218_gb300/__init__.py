"""GB300-native periodic fast multipole method for net-charged boxes neutralised
by a uniform background charge (arXiv:2003.13218).

The compute path is the CUDA library ``libfmm_gb300.so`` (C ABI in
``include/fmm_gb300.h``); ``fmm`` is its ctypes binding and ``boxes`` the
seeded input generator.  Submodules are imported on first use so that the
input generator can be loaded without torch or the CUDA library.
"""
import importlib

__all__ = ["fmm", "boxes", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    if name in ("FMMPlan", "FmmEnergy", "FMMError", "load_library"):
        return getattr(importlib.import_module(".fmm", __name__), name)
    raise AttributeError(name)
