"""ldbp_backward_static: the adjoint for callers that cannot call cudaMalloc
(for example an application that reserves all device memory at start-up, or a
plug-in whose framework forbids new allocations).  Its scratch is a static
device array inside the library instead of a caller workspace.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes when run alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import synth
from tests.test_gpu_ldbp_fwd import _model, _pack, _signal
from tests.util import c64, gpu_lib, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def _setup(Ts, B, n, seed):
    import torch
    gpu_lib()
    from paper_2010_14258_gb300 import api
    taps, c = _model(Ts, seed=seed)
    td = to_dev(_pack(taps))
    xd = to_dev(_signal(B, n, seed, 3e-3))
    gy = to_dev(c64(synth.complex_normal((B, n), seed + 1, 1.0)))
    ck = torch.empty((len(Ts), B, n), dtype=torch.complex64, device="cuda")
    api.ldbp_apply(td, Ts, c, xd, ckpt=ck)
    return api, td, c, ck, gy


def _static_call(td, Ts, c, ck, gy):
    import torch
    from paper_2010_14258_gb300 import _lib
    B, n = gy.shape
    gx = torch.empty_like(gy)
    gt = torch.empty_like(td)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = _lib.lib().ldbp_backward_static(ctypes.c_void_p(td.data_ptr()), td.shape[1], _lib.i32_array(Ts),
                                         _lib.f32_array(c), len(Ts), ctypes.c_void_p(ck.data_ptr()),
                                         ctypes.c_void_p(gy.data_ptr()), ctypes.c_void_p(gx.data_ptr()),
                                         ctypes.c_void_p(gt.data_ptr()), n, B, stream)
    _lib.check(rc)
    torch.cuda.synchronize()
    return to_np(gx), to_np(gt)


def test_static_backward_matches_workspace_backward_on_two_calls():
    import torch
    Ts = [9] * 12 + [5] * 13
    api, td, c, ck, gy = _setup(Ts, 3, 12000, seed=31)
    gx_ref, gt_ref = api.ldbp_backward(td, Ts, c, ck, gy)
    torch.cuda.synchronize()
    gx_ref, gt_ref = to_np(gx_ref), to_np(gt_ref)
    for _ in range(2):  # the static array keeps the previous call's contents
        gx, gt = _static_call(td, Ts, c, ck, gy)
        assert rel_l2(gx, gx_ref) <= 1e-4
        assert rel_l2(gt, gt_ref) <= 1e-4


def test_static_backward_rejects_problems_beyond_its_array():
    import torch
    from paper_2010_14258_gb300 import _lib
    gpu_lib()
    Ts = [31] * 25
    need = ctypes.c_size_t(0)
    _lib.check(_lib.lib().ldbp_backward_workspace(1 << 20, 64, _lib.i32_array(Ts), 25, ctypes.byref(need)))
    assert need.value > (4 << 20)
    # NULL buffers: the size check rejects the call first; were that order ever
    # changed, the NULL checks of ldbp_backward would reject it before any launch
    rc = _lib.lib().ldbp_backward_static(None, 16, _lib.i32_array(Ts), _lib.f32_array([0.0] * 25), 25, None,
                                         None, None, None, 1 << 20, 64, None)
    assert rc == -1
    msg = _lib.lib().ldbp_last_error().decode()
    assert "static array holds 4194304" in msg
    torch.cuda.synchronize()
