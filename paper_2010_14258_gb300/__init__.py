"""GB300-native split-step / learned digital backpropagation (arXiv:2010.14258).

The compute path is ``libldbp.so`` (hand-written CUDA for sm_103a) behind the
C ABI in ``include/ldbp.h``; this package holds the build step, the ctypes
binding and thin torch wrappers.
"""
from . import _lib  # noqa: F401

__all__ = ["_lib"]
