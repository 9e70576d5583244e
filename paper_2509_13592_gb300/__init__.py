"""GB300 BCCB sparse-recovery solver: Python side of the C ABI in include/bccb.h.

The binding (``binding.py``) is loaded on first use, so ``build`` can run before
the library exists.  Any use of the binding raises ImportError when
``libbccb.so`` has not been built: there is no CPU fallback.
"""
import importlib

_SUBMODULES = {"binding", "build", "learned", "shard"}


def __getattr__(name):
    if name in _SUBMODULES:
        return importlib.import_module("." + name, __name__)
    if name.startswith("__"):
        raise AttributeError(name)
    return getattr(importlib.import_module(".binding", __name__), name)
