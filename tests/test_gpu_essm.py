"""Parity of the filtered-nonlinearity (learned ESSM) kernel with the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import essm
from tests.test_gpu_ldbp_fwd import _model, _pack, _signal
from tests.util import c64, gpu_lib, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def _etas(kappas, seed):
    """Low-pass real filters (normalised to unit sum) with a random perturbation."""
    out = []
    for i, k in enumerate(kappas):
        t = np.arange(-k, k + 1)
        e = np.exp(-0.5 * (t / max(k / 2.0, 0.5)) ** 2)
        e = e + 0.05 * np.random.default_rng(seed + i).normal(size=e.size)
        out.append((e / e.sum()).astype(np.float32).astype(np.float64))
    return out


def _run(taps, Ts, c, etas, kappas, x):
    import torch
    from paper_2010_14258_gb300 import api
    gpu_lib()
    stride = max(len(e) for e in etas)
    ed = np.zeros((len(etas), stride), np.float32)
    for i, e in enumerate(etas):
        ed[i, : len(e)] = e
    y = api.ldbp_essm_apply(to_dev(_pack(taps)), Ts, c, torch.from_numpy(ed).cuda(), kappas, to_dev(x))
    torch.cuda.synchronize()
    return to_np(y)


CASES = [
    ([9] * 25, [20] * 25, 2, 12000, 3e-3),
    ([5, 3] * 6, [0, 4, 8] * 4, 2, 9001, 4e-3),      # odd n (plain loads), kappa 0 steps
    ([17, 1, 9, 3], [24, 24, 1, 7], 1, 8192, 2e-3),  # longest supported filter, T = 1 steps
]


@pytest.mark.parametrize("Ts,kappas,B,n,pw", CASES)
def test_essm_forward_parity(Ts, kappas, B, n, pw):
    taps, c = _model(Ts, seed=len(Ts) + n)
    etas = _etas(kappas, n)
    x = _signal(B, n, n + 1, pw)
    y = _run(taps, Ts, c, etas, kappas, x)
    ref, _ = essm.forward(x, taps, c, etas)
    assert rel_l2(y, ref) <= 1e-4


@pytest.mark.parametrize("n", [1, 7, 100, 4097])
def test_essm_short_waveforms_wrap(n):
    Ts, kappas = [5, 3], [6, 2]
    taps, c = _model(Ts, seed=n)
    etas = _etas(kappas, 3)
    x = c64(synth.gaussian_waveform(2, n, 5 + n, 4e-3))
    y = _run(taps, Ts, c, etas, kappas, x)
    ref, _ = essm.forward(x, taps, c, etas)
    assert rel_l2(y, ref) <= 1e-5 * len(Ts)


def test_unit_filter_matches_ldbp_apply():
    import torch
    from paper_2010_14258_gb300 import api
    Ts = [9] * 10
    taps, c = _model(Ts, seed=8)
    x = _signal(2, 8192, 9, 3e-3)
    y = _run(taps, Ts, c, [np.array([1.0])] * 10, [0] * 10, x)
    y0 = to_np(api.ldbp_apply(to_dev(_pack(taps)), Ts, c, to_dev(x)))
    assert rel_l2(y, y0) <= 1e-6


def _eta_dev(etas):
    import torch
    stride = max(len(e) for e in etas)
    ed = np.zeros((len(etas), stride), np.float32)
    for i, e in enumerate(etas):
        ed[i, : len(e)] = e
    return torch.from_numpy(ed).cuda()


@pytest.mark.parametrize("Ts,kappas,B,n", [
    ([9] * 8, [6] * 8, 2, 9000),
    ([5, 3, 1, 7], [20, 0, 3, 8], 1, 8192),
    ([3, 3], [2, 1], 2, 1001),
    ([9] * 4, [17, 20, 18, 19], 2, 8192),   # the exact kappa 17..20 filter class
    ([17, 9], [20, 5], 1, 8192),            # the same class with the wider FIR class
    ([9, 3], [17, 24], 1, 6000),            # the kappa <= 24 class
])
def test_essm_backward_parity(Ts, kappas, B, n):
    import torch
    from paper_2010_14258_gb300 import api
    from tests.test_gpu_ldbp_bwd import _grad_signal
    gpu_lib()
    taps, c = _model(Ts, seed=n + 1)
    etas = _etas(kappas, n + 2)
    x = _signal(B, n, n + 3, 3e-3)
    gy = _grad_signal(B, n, n + 4)
    td, xd, ed = to_dev(_pack(taps)), to_dev(x), _eta_dev(etas)
    ck = torch.empty((len(Ts),) + tuple(xd.shape), dtype=torch.complex64, device="cuda")
    y = api.ldbp_essm_apply(td, Ts, c, ed, kappas, xd, ckpt=ck)
    gx, gt, ge = api.ldbp_essm_backward(td, Ts, c, ed, kappas, ck, to_dev(gy))
    torch.cuda.synchronize()
    rgx, rgt, rge = essm.backward(x, taps, c, etas, gy)
    assert rel_l2(to_np(gx), rgx) <= 1e-4
    for i in range(len(Ts)):
        h = rgt[i]
        assert rel_l2(to_np(gt)[i, : len(h)], h) <= 1e-4, i
        e = rge[i]
        assert rel_l2(ge.cpu().numpy()[i, : len(e)].astype(np.float64), e) <= 1e-4, i
        assert np.all(ge.cpu().numpy()[i, len(e):] == 0)
    _, inputs = essm.forward(x, taps, c, etas)
    assert rel_l2(to_np(ck[-1]), inputs[-1]) <= 1e-4
