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


@pytest.mark.parametrize("B,n_out,r,bw", [(3, 1024, 3, 1.0), (2, 1024, 3, 0.6), (2, 2048, 3, 1.0), (1, 512, 5, 1.0),
                                          (2, 512, 4, 0.5), (2, 512, 1, 0.8), (1, 4096, 4, 1.0), (2, 512, 8, 0.7)])
def test_resample_down_matches_oracle(B, n_out, r, bw):
    # brick-wall low-pass + sampling at the DSP rate (Sec. IV-A), wideband input
    # so that the filter cuts; the plain low-pass (r = 1) included
    import torch
    api = _api()
    x = c64(synth.gaussian_waveform(B, n_out * r, 40 + B, 1.0))
    y = api.resample(to_dev(x), n_out, bw)
    torch.cuda.synchronize()
    assert rel_l2(to_np(y), txrx.lowpass_sample(x, n_out, bw)) <= 2e-6


@pytest.mark.parametrize("B,n_in,r", [(3, 1024, 3), (2, 2048, 3), (1, 512, 7), (2, 512, 8), (1, 4096, 2)])
def test_resample_up_matches_oracle(B, n_in, r):
    import torch
    api = _api()
    x = c64(synth.gaussian_waveform(B, n_in, 50 + B, 1.0))
    y = api.resample(to_dev(x), n_in * r)
    torch.cuda.synchronize()
    assert rel_l2(to_np(y), txrx.interpolate(x, n_in * r)) <= 2e-6


def test_resample_in_place_low_pass():
    import torch
    api = _api()
    x = c64(synth.gaussian_waveform(2, 1024, 57, 1.0))
    xd = to_dev(x)
    api.resample(xd, 1024, 0.5, out=xd)
    torch.cuda.synchronize()
    assert rel_l2(to_np(xd), txrx.lowpass_sample(x, 1024, 0.5)) <= 2e-6


@pytest.mark.parametrize("symmetric,ase", [(True, True), (False, False)])
def test_analog_rate_link_matches_oracle(symmetric, ase):
    # The system model of Sec. IV-A: transmit waveform on the analog grid
    # (rho_a = 6 samples/symbol, here interpolated from the DSP-rate transmitter),
    # split-step channel on that 3 * 2^k grid (the fused cluster kernel), brick-wall
    # low-pass and sampling at rho_d = 2.  Oracle: the same chain in FP64 at rho_a.
    import torch
    api = _api()
    B, nsym, rho_a, rho_d, Rs = 2, 512, 6, 2, 10e9
    s = c64(synth.qam16_symbols(B, nsym, 21))
    P = np.array([1.585e-3, 3e-3], np.float32)
    fib = synth.Fiber()
    link = synth.Link(2, 80.0, 6, symmetric, ase, seed=9, counter=1)
    xd = api.tx(to_dev(s), torch.from_numpy(P).cuda(), sps=rho_d)
    xa = api.resample(xd, nsym * rho_a)
    ya = api.ssm_forward(fib, link, rho_a * Rs, xa)
    r = api.resample(ya, nsym * rho_d)
    torch.cuda.synchronize()
    ref = txrx.lowpass_sample(nlse.channel(txrx.tx(s, rho_a, 0.1, P.astype(np.float64)), fib, link, rho_a * Rs),
                              nsym * rho_d)
    assert rel_l2(to_np(r), ref) <= 1e-4


def test_analog_rate_link_full_size_sampled():
    # the analog-rate workload: 2048 frames of the paper's 1024 symbols at
    # rho_a = 6 (n = 6144), 25 x 80 km at 100 StPS with ASE on the fused kernel,
    # then the front end down to rho_d = 2; frames 0 and 2047 against the oracle
    import torch
    api = _api()
    B, nsym, rho_a, rho_d, Rs = 2048, 1024, 6, 2, 10e9
    s = synth.qam16_symbols(B, nsym, 71)
    pw = np.full(B, 1.585e-3, np.float32)
    fib = synth.Fiber()
    link = synth.Link(25, 80.0, 100, True, True, seed=5, counter=3)
    xa = api.resample(api.tx(to_dev(c64(s)), torch.from_numpy(pw).cuda(), sps=rho_d), nsym * rho_a)
    ya = api.ssm_forward(fib, link, rho_a * Rs, xa)
    r = api.resample(ya, nsym * rho_d)
    torch.cuda.synchronize()
    ch0 = nlse.channel(to_np(xa[0:1]), fib, link, rho_a * Rs)
    assert rel_l2(to_np(ya[0:1]), ch0) <= 1e-4
    assert rel_l2(to_np(r[0:1]), txrx.lowpass_sample(ch0, nsym * rho_d)) <= 1e-4
    # the last frame alone with ASE off on both sides (a one-frame oracle run
    # draws the noise of waveform index 0, not of index 2047)
    link0 = synth.Link(25, 80.0, 100, True, False)
    y0 = api.ssm_forward(fib, link0, rho_a * Rs, xa[B - 1:B].contiguous())
    torch.cuda.synchronize()
    assert rel_l2(to_np(y0), nlse.channel(to_np(xa[B - 1:B]), fib, link0, rho_a * Rs)) <= 1e-4


def test_resample_full_size_sampled_waveforms():
    # 2048 frames of 1024 symbols at rho_a = 6 (n = 6144) down to rho_d = 2 and
    # back up; frames 0 and 2047 against the oracle.
    import torch
    api = _api()
    B, nsym = 2048, 1024
    g = torch.Generator(device="cuda").manual_seed(61)
    x = torch.randn(B, 6 * nsym, dtype=torch.complex64, device="cuda", generator=g)
    y = api.resample(x, 2 * nsym)
    z = api.resample(y, 6 * nsym)
    torch.cuda.synchronize()
    for b in (0, B - 1):
        xb = to_np(x[b:b + 1])
        ref = txrx.lowpass_sample(xb, 2 * nsym)
        assert rel_l2(to_np(y[b:b + 1]), ref) <= 2e-6
        assert rel_l2(to_np(z[b:b + 1]), txrx.interpolate(ref, 6 * nsym)) <= 4e-6


def test_receiver_serves_the_validated_equaliser():
    # Receiver with full-length DBP as the fallback of LDBP: the served output is
    # bit-identical to ldbp_apply when validation accepts LDBP and to dbp_apply
    # otherwise; the validation SNRs are those of the receiver chain on each.
    import torch
    api = _api()
    from paper_2010_14258_gb300 import init, receiver
    fs, pw = 20e9, 10 ** (2.0 / 10) * 1e-3
    fib = synth.Fiber()
    link = synth.Link(25, 80.0, 4, True, False)
    s = to_dev(c64(synth.qam16_symbols(2, 4096, 31)))
    p = torch.full((2,), pw, dtype=torch.float32, device="cuda")
    y = api.ssm_forward(fib, link, fs, api.tx(s, p))
    Ts = [9] * 25
    taps, c = init.ldbp_init(Ts, span_km=80.0, fs=fs)
    tp = np.zeros((25, 5), np.complex64)
    for i, h in enumerate(taps):
        tp[i, : len(h)] = h
    td = torch.from_numpy(tp).cuda()
    ref_l = api.ldbp_apply(td, Ts, c, y)
    ref_d = api.dbp_apply(fib, link, fs, y, 1, False)
    st_l, _, _ = api.rx(ref_l, s, p)
    st_d, _, _ = api.rx(ref_d, s, p)
    for tol, use in ((1e3, True), (-1e3, False)):
        r = receiver.Receiver(td, Ts, c, fib, link, fs, tolerance_db=tol)
        d = r.validate(y, s, p)
        assert d.use_ldbp is use
        assert abs(d.snr_ldbp_db - api.snr_db(st_l)) <= 1e-9
        assert abs(d.snr_dbp_db - api.snr_db(st_d)) <= 1e-9
        out = r.backpropagate(y)
        torch.cuda.synchronize()
        assert torch.equal(out, ref_l if use else ref_d)
