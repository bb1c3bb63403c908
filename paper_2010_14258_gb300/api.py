"""Torch-facing wrappers of the C ABI (argument marshalling only).

Every function takes CUDA tensors, passes their device pointers and the
current CUDA stream to ``libldbp.so`` and returns the outputs; no arithmetic
of the method runs here.
"""
from __future__ import annotations

import torch

from . import _lib


def _stream():
    return ctypes_void(torch.cuda.current_stream().cuda_stream)


def ctypes_void(v):
    import ctypes
    return ctypes.c_void_p(int(v))


def _ptr(t):
    return None if t is None else ctypes_void(t.data_ptr())


def _check_c64(name, t, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.complex64:
        raise ValueError(f"{name} must be complex64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def ldbp_apply(taps, T, c, x, ckpt=None, out=None):
    """Learned-DBP forward (Eq. (7), symmetric FIR steps).  x: complex64 [B, n] or [n]."""
    squeeze = x.dim() == 1
    x2 = x.unsqueeze(0) if squeeze else x
    _check_c64("x", x2)
    _check_c64("taps", taps)
    B, n = x2.shape
    M = len(T)
    if taps.dim() != 2 or taps.shape[0] != M:
        raise ValueError("taps must be [M, stride] with M = len(T)")
    y = torch.empty_like(x2) if out is None else out
    if ckpt is not None:
        _check_c64("ckpt", ckpt, (M, B, n))
    _lib.check(_lib.lib().ldbp_apply(_ptr(taps), taps.shape[1], _lib.i32_array(T), _lib.f32_array(c), M,
                                     _ptr(x2), _ptr(y), n, B, _ptr(ckpt), _stream()))
    return y[0] if squeeze else y


def ubench(kind: int) -> float:
    """Measured lane-operation throughput: 0 FP32 FMA, 1 FP32x2 FMA, 2 sine (ops/s)."""
    import ctypes
    out = ctypes.c_double(0.0)
    _lib.check(_lib.lib().ldbp_ubench(kind, ctypes.byref(out)))
    return out.value
