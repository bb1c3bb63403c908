"""ctypes binding of ``libldbp.so`` (argument marshalling only).

The library is loaded from this package directory.  There is no fallback: if
the shared library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libldbp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ldbp.h")

_lib = None

c_int, c_int32, c_int64, c_float, c_double, c_void_p, c_uint64 = (
    ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double, ctypes.c_void_p,
    ctypes.c_uint64)
P_int32 = ctypes.POINTER(ctypes.c_int32)
P_float = ctypes.POINTER(ctypes.c_float)


class LdbpFiber(ctypes.Structure):
    _fields_ = [("alpha_db_per_km", c_double), ("beta2_ps2_per_km", c_double), ("gamma_per_w_km", c_double)]


class LdbpLink(ctypes.Structure):
    _fields_ = [("n_spans", c_int32), ("span_km", c_double), ("steps_per_span", c_int32),
                ("symmetric", c_int32), ("ase", c_int32), ("nf_db", c_double), ("carrier_hz", c_double),
                ("seed", c_uint64), ("counter", c_uint64)]


_SIGNATURES = {
    "ldbp_last_error": (ctypes.c_char_p, []),
    "ldbp_version": (c_int, []),
    "ldbp_device_status": (c_int, []),
    "ldbp_wait_probe": (c_int, [c_int32, c_int32, c_void_p]),
    "ssm_forward": (c_int, [ctypes.POINTER(LdbpFiber), ctypes.POINTER(LdbpLink), c_double, c_void_p, c_void_p,
                            c_int64, c_int32, c_void_p]),
    "dbp_apply": (c_int, [ctypes.POINTER(LdbpFiber), ctypes.POINTER(LdbpLink), c_double, c_int32, c_int32,
                          c_void_p, c_void_p, c_int64, c_int32, c_void_p]),
    "ssm_cufft": (c_int, [ctypes.POINTER(LdbpFiber), ctypes.POINTER(LdbpLink), c_double, c_int32, c_int32,
                          c_void_p, c_void_p, c_int64, c_int32, c_void_p]),
    "ldbp_tx": (c_int, [c_void_p, c_void_p, c_int32, c_double, c_void_p, c_int64, c_int32, c_void_p]),
    "ldbp_rx": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_double, c_int64, c_int32, c_void_p, c_void_p,
                        c_void_p, c_float, c_void_p, c_void_p]),
    "ldbp_backward": (c_int, [c_void_p, c_int32, P_int32, P_float, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_int64, c_int32, c_void_p, ctypes.c_size_t, c_void_p]),
    "ldbp_backward_c": (c_int, [c_void_p, c_int32, P_int32, P_float, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_int64, c_int32, c_void_p, ctypes.c_size_t, c_void_p]),
    "ldbp_backward_static": (c_int, [c_void_p, c_int32, P_int32, P_float, c_int32, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_int64, c_int32, c_void_p]),
    "ldbp_backward_workspace": (c_int, [c_int64, c_int32, P_int32, c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "ldbp_adam_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, P_int32, c_int32, c_int32, c_int32, c_float,
                               c_float, c_float, c_float, c_void_p]),
    "ldbp_ragged_plan_create": (c_int, [ctypes.POINTER(c_void_p), c_int32, ctypes.POINTER(c_int64), P_int32,
                                        P_int32, c_int32]),
    "ldbp_ragged_plan_destroy": (c_int, [c_void_p]),
    "ldbp_ragged_set_schedule": (c_int, [c_void_p, c_int32, c_int32]),
    "ldbp_ragged_info": (c_int, [c_void_p, ctypes.POINTER(c_int64), P_int32, P_int32, P_int32, P_int32]),
    "ldbp_ragged_autotune": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ldbp_apply_ragged": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ldbp_ragged_graph_capture": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ldbp_ragged_graph_launch": (c_int, [c_void_p, c_void_p]),
    "ldbp_ubench": (c_int, [c_int32, ctypes.POINTER(c_double)]),
    "ldbp_resample": (c_int, [c_void_p, c_int64, c_void_p, c_int64, c_double, c_int32, c_void_p]),
    "ldbp_apply": (c_int, [c_void_p, c_int32, P_int32, P_float, c_int32, c_void_p, c_void_p, c_int64, c_int32,
                           c_void_p, c_void_p]),
    "ldbp_apply_host_workspace": (ctypes.c_size_t, [c_int64, c_int32]),
    "ldbp_essm_apply": (c_int, [c_void_p, c_int32, P_int32, P_float, c_void_p, c_int32, P_int32, c_int32, c_void_p,
                                c_void_p, c_int64, c_int32, c_void_p, c_void_p]),
    "ldbp_essm_backward_workspace": (c_int, [c_int64, c_int32, P_int32, P_int32, c_int32,
                                             ctypes.POINTER(ctypes.c_size_t)]),
    "ldbp_essm_backward": (c_int, [c_void_p, c_int32, P_int32, P_float, c_void_p, c_int32, P_int32, c_int32, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_void_p, ctypes.c_size_t,
                                   c_void_p]),
    "ldbp_apply_host": (c_int, [c_void_p, c_int32, P_int32, P_float, c_int32, c_void_p, c_void_p, c_int64, c_int32,
                                c_int32, c_void_p, ctypes.c_size_t, c_void_p]),
}


class LdbpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libldbp error {code}: {msg}")
        self.code = code


def lib():
    """Load libldbp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2010_14258_gb300.build.build() first "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc: int):
    if rc != 0:
        msg = lib().ldbp_last_error().decode(errors="replace")
        raise LdbpError(rc, msg)


def declared_symbols():
    """Function names declared in include/ldbp.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(ldbp_[a-z_0-9]+|ssm_[a-z_0-9]+|dbp_[a-z_0-9]+)\s*\(",
                                 text, flags=re.M)))


def i32_array(vals):
    arr = (ctypes.c_int32 * len(vals))(*[int(v) for v in vals])
    return arr


def f32_array(vals):
    return (ctypes.c_float * len(vals))(*[float(v) for v in vals])
