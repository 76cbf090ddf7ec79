"""Voxel-based ray casting of large 3D line sets on GB300 (arXiv 1801.01155).

The CUDA library (``csrc/``, C ABI declared in ``include/lvr.h``) does all the
work; ``lvr`` is its thin ctypes binding. ``synth`` makes seeded inputs.
The binding is imported lazily so that input generation needs no GPU.
"""
from __future__ import annotations

import importlib

__all__ = ["lvr", "synth"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
