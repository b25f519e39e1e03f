"""GB300-native IB-LBM hot path (arXiv 2102.01305) behind a C ABI.

* ``include/ibl.h``    the C ABI (the boundary);
* ``csrc/``            CUDA kernels for sm_103a and the ABI implementation;
* ``ibl``              thin ctypes binding with the ABI's names (loaded lazily);
* ``build``            in-tree nvcc build of ``libibl.so``.
"""
import importlib

__all__ = ["ibl", "build"]


def __getattr__(name):
    if name in ("ibl", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
