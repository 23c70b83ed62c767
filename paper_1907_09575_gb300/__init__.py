"""GB300-native exact triangle counting (Tom and Karypis, ICPP 2019).

The CUDA library (``_build/libtc.so``, C ABI in ``include/tc.h``) does all the
work; ``paper_1907_09575_gb300.tc`` is its thin ctypes binding and
``paper_1907_09575_gb300.inputs`` holds the seeded synthetic-graph
generators.  The binding is imported lazily so that the input generators can
be used without a GPU.
"""
from __future__ import annotations

import importlib

__all__ = ["tc", "inputs", "build", "preprocess", "triangles", "generate_rmat", "Graph", "TCError"]


def __getattr__(name):
    if name in ("tc", "inputs", "build"):
        return importlib.import_module(f".{name}", __name__)
    if name in ("preprocess", "triangles", "generate_rmat", "Graph", "TCError", "Tuning"):
        return getattr(importlib.import_module(".tc", __name__), name)
    raise AttributeError(name)
