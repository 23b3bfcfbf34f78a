"""GB300-native hot path of Scalable Laplacian K-modes (SLK-BO).

The compute lives in a CUDA library (``csrc/``, sm_103a) behind the C-ABI of
``include/slk.h``; :mod:`.slk` is the thin ctypes binding with the same names.
The binding is imported lazily so that :mod:`.inputs` (seeded synthetic data)
imports without a GPU.
"""
import importlib

__all__ = ["inputs", "slk"]


def __getattr__(name):
    if name in ("slk", "inputs", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
