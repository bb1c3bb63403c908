"""Pins of the receiver front-end oracle (Sec. IV-A, Table I): brick-wall
low-pass at bandwidth Delta B followed by sampling at the DSP rate, and the
band-limited interpolation that goes the other way."""
import numpy as np
import pytest

import synth
from oracle import nlse, txrx


def _tone(kappa, n, B=1):
    m = np.arange(n)
    return np.tile(np.exp(2j * np.pi * kappa * m / n), (B, 1))


@pytest.mark.parametrize("bandwidth", [1.0, 0.5, 0.3])
def test_single_tones_pass_reject_and_do_not_alias(bandwidth):
    # A tone at bin kappa of the analog grid is exp(j 2 pi kappa m / n_a).  After
    # the front end it must be the same frequency on the DSP grid,
    # exp(j 2 pi kappa k / n_d), when |kappa| < bandwidth n_d / 2, and exactly
    # zero otherwise -- in particular a tone above f_s / 2 must not fold back.
    n_d, r = 64, 3
    n_a = n_d * r
    edge = bandwidth * n_d / 2
    for kappa in [0, 1, 5, 9, 10, 15, 16, 31, -31, 32, -32, 33, 40, 70, 95, -70, -95]:
        out = txrx.lowpass_sample(_tone(kappa, n_a), n_d, bandwidth)
        if abs(kappa) < edge:
            ref = _tone(kappa, n_d)
        else:
            ref = np.zeros((1, n_d))
        assert np.max(np.abs(out - ref)) < 1e-12, (kappa, bandwidth)


def test_band_edge_at_nyquist_is_rejected():
    # Delta B = f_s: the bins kappa = +-n_d / 2 sit exactly on the band edge and
    # are rejected (open passband); the bins just inside pass at full amplitude.
    n_d, n_a = 32, 192
    assert np.max(np.abs(txrx.lowpass_sample(_tone(16, n_a), n_d))) < 1e-13
    assert np.max(np.abs(txrx.lowpass_sample(_tone(-16, n_a), n_d))) < 1e-13
    assert np.allclose(np.abs(txrx.lowpass_sample(_tone(15, n_a), n_d)), 1.0, atol=1e-13)


def test_analog_rate_tx_sampled_down_is_dsp_rate_tx():
    # Eq. (11) describes one continuous-time waveform; sampled at rho_a = 6 and
    # passed through the front end it must equal the same waveform sampled at
    # rho_d = 2 (the RRC band |f| <= 0.55 R_s lies inside |f| < f_s / 2).
    s = synth.qam16_symbols(3, 256, seed=7)
    P = np.array([1e-3, 2e-3, 0.5e-3])
    xa = txrx.tx(s, 6, 0.1, P)
    xd = txrx.tx(s, 2, 0.1, P)
    out = txrx.lowpass_sample(xa, xd.shape[-1])
    assert np.max(np.abs(out - xd)) < 1e-12 * np.max(np.abs(xd))
    up = txrx.interpolate(xd, xa.shape[-1])
    assert np.max(np.abs(up - xa)) < 1e-12 * np.max(np.abs(xa))
    # and the receiver chain at rho_d recovers the symbols back to back
    ev = txrx.evaluate(out, s, 2, 0.1, P)
    assert ev["snr_db"] > 250


@pytest.mark.parametrize("symmetric", [True, False])
def test_dispersive_propagation_commutes_with_the_front_end(symmetric):
    # With gamma = 0 every step is diagonal on the DFT grid and bin kappa is the
    # same frequency on both grids, so simulating at the analog rate and then
    # filtering/sampling equals filtering/sampling and then simulating at the
    # DSP rate -- for a wideband input that the front end does cut.
    fib = synth.Fiber(0.2, -21.7, 0.0)
    link = synth.Link(2, 80.0, 4, symmetric, False)
    n_d, r, fs = 256, 3, 20e9
    xa = synth.gaussian_waveform(2, n_d * r, 11, 1e-3)
    left = txrx.lowpass_sample(nlse.channel(xa, fib, link, fs * r), n_d)
    right = nlse.channel(txrx.lowpass_sample(xa, n_d), fib, link, fs)
    assert np.max(np.abs(left - right)) < 1e-12 * np.max(np.abs(right))


def test_ase_power_after_the_front_end_is_rate_independent():
    # White ASE simulated at f_a = 3 f_s has per-sample variance PSD f_a; the
    # front end keeps n_d - 1 of the n_d bins of width f_s / n_d, so the
    # sampled noise has variance PSD f_s (n_d - 1) / n_d whatever the analog rate.
    fib = synth.Fiber(0.2, -21.7, 0.0)
    link = synth.Link(1, 80.0, 1, True, True, 5.0, 1.946e14, 5, 0)
    n_d, r, fs, B = 2048, 3, 20e9, 16
    a = nlse.si_alpha(0.2)
    y = nlse.channel(np.zeros((B, n_d * r), dtype=complex), fib, link, fs * r)
    out = txrx.lowpass_sample(y, n_d)
    expect = nlse.ase_sigma2(a, 80e3, 5.0, 1.946e14, fs) * (n_d - 1) / n_d
    assert abs(np.mean(np.abs(out) ** 2) / expect - 1) < 0.03
    # and the kept bins are exactly those of the analog-rate realisation
    Y = np.fft.fft(y, axis=-1) / (n_d * r)
    R = np.fft.fft(out, axis=-1) / n_d
    k = np.r_[0:n_d // 2, -(n_d // 2) + 1:0]
    assert np.max(np.abs(R[:, k % n_d] - Y[:, k % (n_d * r)])) < 1e-12 * np.max(np.abs(Y))


def test_parseval_of_the_front_end():
    # ||r||^2 = (n_d / n_a^2) sum over kept bins |Y_kappa|^2
    n_d, r = 128, 6
    y = synth.gaussian_waveform(3, n_d * r, 12, 1.0)
    out = txrx.lowpass_sample(y, n_d, 0.8)
    Y = np.fft.fft(y, axis=-1)
    kept = txrx.brickwall_mask(n_d * r, 0.8 * n_d) > 0
    assert kept.sum() == 2 * 51 + 1
    lhs = np.sum(np.abs(out) ** 2, axis=-1)
    rhs = n_d / (n_d * r) ** 2 * np.sum(np.abs(Y[:, kept]) ** 2, axis=-1)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=0)


def test_interpolation_round_trip_and_errors():
    n_d, r = 96, 4
    x = synth.gaussian_waveform(2, n_d, 13, 1.0)
    X = np.fft.fft(x, axis=-1)
    X[:, n_d // 2] = 0  # the Nyquist bin is outside the interpolation band
    x = np.fft.ifft(X, axis=-1)
    up = txrx.interpolate(x, n_d * r)
    assert np.max(np.abs(up[:, ::r] - x)) < 1e-12
    assert np.max(np.abs(txrx.lowpass_sample(up, n_d) - x)) < 1e-12
    with pytest.raises(ValueError):
        txrx.lowpass_sample(up, 100)
    with pytest.raises(ValueError):
        txrx.lowpass_sample(up, n_d, 1.5)
    with pytest.raises(ValueError):
        txrx.interpolate(x, 100)


def test_wdm_channel_selection_at_37p5_ghz():
    # The 32 GBd WDM case of Sec. V: rho_a = 10 (Table I), channels on a 50 GHz
    # grid, Delta B = 37.5 GHz at f_s = 64 GHz.  Read two-sided (|f| < 18.75 GHz)
    # the front end returns exactly the centre channel sampled at rho_d = 2: its
    # RRC band |f| <= 17.6 GHz passes and the neighbours (32.4..67.6 GHz off
    # centre) are rejected.  Read one-sided (|f| < 37.5 GHz) the neighbours'
    # inner edges (32.4..37.5 GHz) would pass and fold back into the band when
    # sampled at f_s = 64 GHz.
    nsym, Rs, rho_a, rho_d, P = 256, 32e9, 10, 2, 1e-3
    n_a, n_d = nsym * rho_a, nsym * rho_d
    t = np.arange(n_a) / (rho_a * Rs)
    s = synth.qam16_symbols(3, nsym, seed=17)
    centre = txrx.tx(s[0], rho_a, 0.1, P)
    wdm = centre + sum(txrx.tx(s[i], rho_a, 0.1, P) * np.exp(2j * np.pi * f * t)
                       for i, f in ((1, -50e9), (2, 50e9)))
    bw = 37.5e9 / (rho_d * Rs)
    out = txrx.lowpass_sample(wdm, n_d, bw)
    ref = txrx.tx(s[0], rho_d, 0.1, P)
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))
    bin_hz = Rs / nsym
    wide = np.fft.ifft(np.fft.fft(wdm, axis=-1) * txrx.brickwall_mask(n_a, 2 * 37.5e9 / bin_hz), axis=-1)
    one_sided = wide[:, :: rho_a // rho_d]
    assert np.max(np.abs(one_sided - ref)) > 1e-2 * np.max(np.abs(ref))
