"""GB300-native neighbourhood graph: exact kNN + fuzzy connectivities.

The compute lives in the CUDA library ``_lib/librsc.so`` (C ABI in
include/rsc.h); ``rsc`` is its thin ctypes binding and ``synth`` the seeded
input generators.  Importing the package does not load the library.
"""
from .build import build  # noqa: F401

__all__ = ["build", "rsc", "synth"]


def __getattr__(name):
    if name in ("rsc", "synth"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
