"""Failure detection on the GPU: a bounded device wait that runs out.

The library's TMA and cluster-exchange waits are bounded: after an iteration
limit the kernel records a timeout in the device status word and returns,
so the host sees an error code instead of a hung GPU.  ldbp_wait_probe runs
that same bounded wait on a shared-memory mbarrier that can never complete
(one of two expected arrivals, no asynchronous copy involved), so the
timeout path is exercised without a fault, a trap or an unbounded wait.
"""
import numpy as np
import pytest

import synth
from oracle import ldbp as oldbp
from tests.util import gpu_lib, rel_l2

pytestmark = pytest.mark.gpu

LDBP_OK, LDBP_ETIMEOUT = 0, -4


def _stream():
    import ctypes
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_bounded_wait_runs_out_and_status_resets():
    L = gpu_lib()
    assert L.ldbp_device_status() == LDBP_OK          # clear anything left over
    # the phase completes: no timeout recorded
    assert L.ldbp_wait_probe(2, 1000, _stream()) == LDBP_OK
    assert L.ldbp_device_status() == LDBP_OK
    # one arrival of two: the wait gives up after 1000 polls and says so
    assert L.ldbp_wait_probe(1, 1000, _stream()) == LDBP_OK
    assert L.ldbp_device_status() == LDBP_ETIMEOUT
    assert b"bounded device wait" in L.ldbp_last_error()
    # reading the status cleared it
    assert L.ldbp_device_status() == LDBP_OK
    # no arrival at all: same outcome
    assert L.ldbp_wait_probe(0, 10, _stream()) == LDBP_OK
    assert L.ldbp_device_status() == LDBP_ETIMEOUT


def test_context_usable_after_timeout():
    import torch
    from paper_2010_14258_gb300 import api, init
    L = gpu_lib()
    assert L.ldbp_wait_probe(1, 100, _stream()) == LDBP_OK
    assert L.ldbp_device_status() == LDBP_ETIMEOUT
    Ts = [5, 3]
    taps, c = init.ldbp_init(Ts, span_km=80.0, fs=20e9)
    tarr = np.zeros((2, 3), np.complex64)
    for i, h in enumerate(taps):
        tarr[i, :len(h)] = h
    x = synth.gaussian_waveform(1, 4096, 3, 2e-3).astype(np.complex64)
    y = api.ldbp_apply(torch.from_numpy(tarr).cuda(), Ts, c, torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref, _ = oldbp.forward(x.astype(np.complex128), [tarr[i, :len(h)].astype(np.complex128)
                                                      for i, h in enumerate(taps)], np.float32(c).tolist())
    assert rel_l2(y.cpu().numpy(), ref) < 1e-5
    assert L.ldbp_device_status() == LDBP_OK

