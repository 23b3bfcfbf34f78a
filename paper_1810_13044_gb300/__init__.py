"""GB300-native hot path of Scalable Laplacian K-modes (SLK-BO).

The compute lives in a CUDA library (``csrc/``, sm_103a) behind the C-ABI of
``include/slk.h``; :mod:`.slk` is the thin ctypes binding with the same names.
The binding is loaded lazily so that :mod:`.inputs` (seeded synthetic data)
imports without a GPU.
"""
__all__ = ["inputs", "slk"]


def __getattr__(name):
    if name == "slk":
        from . import slk
        return slk
    if name == "inputs":
        from . import inputs
        return inputs
    raise AttributeError(name)
