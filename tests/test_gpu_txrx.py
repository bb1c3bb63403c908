"""Parity of the transmitter, receiver/loss kernels and the cuFFT comparison path with the oracle."""
import numpy as np
import pytest

import synth
from oracle import nlse, txrx
from tests.util import c64, gpu_lib, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def _api():
    gpu_lib()
    from paper_2010_14258_gb300 import api
    return api


@pytest.mark.parametrize("B,nsym,sps", [(3, 1024, 2), (2, 4096, 4), (64, 16384, 2)])
def test_tx_parity(B, nsym, sps):
    import torch
    api = _api()
    s = c64(synth.qam16_symbols(B, nsym, 5 + B))
    P = np.linspace(0.5e-3, 4e-3, B).astype(np.float32)
    x = api.tx(to_dev(s), torch.from_numpy(P).cuda(), sps=sps)
    torch.cuda.synchronize()
    ref = txrx.tx(s, sps, 0.1, P.astype(np.float64))
    assert rel_l2(to_np(x), ref) <= 1e-5


def test_rx_stats_and_grad_parity():
    import torch
    api = _api()
    B, nsym, sps = 4, 8192, 2
    s = c64(synth.qam16_symbols(B, nsym, 9))
    P = np.array([1e-3, 2e-3, 0.5e-3, 3e-3], np.float32)
    x = txrx.tx(s, sps, 0.1, P.astype(np.float64))
    y = c64(x * np.exp(0.3j) + synth.gaussian_waveform(B, nsym * sps, 3, 2e-5))
    st, phi, g = api.rx(to_dev(y), to_dev(s), torch.from_numpy(P).cuda(), sps=sps, grad=True)
    torch.cuda.synchronize()
    ev = txrx.evaluate(y, s, sps, 0.1, P.astype(np.float64))
    gref, _ = txrx.loss_grad(y, s, sps, 0.1, P.astype(np.float64))
    mse = st[:, 0].cpu().numpy()
    assert np.max(np.abs(mse / ev["mse"] - 1)) <= 1e-4
    assert np.max(np.abs(phi.cpu().numpy() - ev["phi"])) <= 1e-5
    assert abs(api.snr_db(st) - ev["snr_db"]) <= 0.01
    assert rel_l2(to_np(g), gref) <= 1e-5


def test_back_to_back_tx_rx_is_exact():
    import torch
    api = _api()
    s = to_dev(c64(synth.qam16_symbols(2, 4096, 1)))
    p = torch.tensor([1e-3, 2e-3], device="cuda")
    x = api.tx(s, p)
    st, phi, _ = api.rx(x, s, p)
    torch.cuda.synchronize()
    assert float(st[:, 0].max()) < 1e-10 and float(phi.abs().max()) < 1e-5


@pytest.mark.parametrize("mode", ["channel_sym", "channel_asym_ase", "dbp_asym", "dbp_sym"])
def test_cufft_path_matches_oracle(mode):
    import torch
    api = _api()
    fs = 20e9
    fib = synth.Fiber()
    sym = mode.endswith("sym") and not mode.endswith("asym")
    link = synth.Link(3, 80.0, 4, sym if mode.startswith("channel") else True, "ase" in mode, seed=77, counter=3)
    x = c64(txrx.tx(synth.qam16_symbols(2, 4096, 2), 2, 0.1, 2e-3))
    if mode.startswith("channel"):
        out = api.ssm_cufft(fib, link, fs, to_dev(x))
        ref = nlse.channel(x, fib, link, fs)
    else:
        out = api.ssm_cufft(fib, link, fs, to_dev(x), dbp_steps_per_span=2, dbp_symmetric=sym)
        ref = nlse.dbp(x, fib, link, fs, steps_per_span=2, symmetric=sym)
    torch.cuda.synchronize()
    assert rel_l2(to_np(out), ref) <= 1e-4
