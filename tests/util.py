"""Shared test helpers: library handle, tensor conversion, error metrics."""
import numpy as np
import pytest


def gpu_lib():
    """Build (if needed) and load libldbp.so; skip when no CUDA device is present."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_14258_gb300 import build
    build.build()
    from paper_2010_14258_gb300 import _lib
    return _lib.lib()


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).cuda()


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def c64(a):
    """Round to complex64 and back: the exact input both sides see."""
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
