"""GB300-native VL2 ideal-MHD stepper (arXiv:2005.06651, Sec. 3): CUDA kernels behind a C ABI.

Submodules are loaded lazily so that importing the seeded input generators (``.inputs``) never
loads the CUDA library.
"""
import importlib

__all__ = ["inputs", "vl2"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
