"""Transmitter, receiver chain, loss and effective SNR, FP64 (oracle side).

* Transmit signal, Eq. (11): x(t) = sqrt(P) sum_k s_k p(t - k/R_s), p an RRC
  pulse with 10 % roll-off; the symbol sequence is periodic (so the sampled
  waveform is circular).  Sampled at fs = rho R_s, the pulse is applied in the
  frequency domain with H(f) = sqrt(rho RC(f/R_s)), RC the raised-cosine
  spectrum, so that RRC * RRC sampled every rho-th sample is the identity
  (Nyquist).  The waveform is scaled by sqrt(P rho), giving mean |x_m|^2 = P
  for unit-energy symbols (a reading of the power normalisation).
* Receiver, Eq. (12): s_hat = e^{-j phi} M f_theta(r), M = matched RRC filter
  followed by keeping every rho-th sample (offset 0: the zero-phase FD filter
  has no delay), divided by sqrt(P rho); phi = arg(s^H s_tilde) (genie-aided,
  Remark 6).
* Loss (Sec. IV-B): l = ||s_hat - s||^2 / N_sym, averaged over the batch.
* Effective SNR, Eq. (14): read as the ratio of sums
  sum_b ||s_b||^2 / sum_b ||s_hat_b - s_b||^2 (in dB); the per-waveform values
  N_sym / ||s_hat_b - s_b||^2 are also returned.
* Gradient of the loss w.r.t. the LDBP output (convention dl/dRe + j dl/dIm):
  phi is treated as a constant (it minimises the loss over a common rotation,
  so its total-derivative contribution vanishes), and the matched filter is
  real and even, hence self-adjoint.

* Receiver front end (Sec. IV-A, Table I): the channel is simulated at
  rho_a > rho_d samples/symbol; the received waveform is low-pass filtered by
  an ideal brick-wall filter of bandwidth Delta B and sampled at t = k / f_s.
  Both grids span the same period N_sym / R_s, so DFT bin kappa is the same
  frequency kappa R_s / N_sym on either grid.  Readings: Delta B is the total
  (two-sided) bandwidth and Table I's Delta B = f_s is taken (the text's 2 f_s
  would alias at t = k / f_s; the 37.5 GHz of the 32 GBd WDM case only makes
  sense two-sided); the passband is open, |f| < Delta B / 2, so at
  Delta B = f_s the Nyquist bin of the sampled grid is rejected.  The same
  band limit defines the opposite direction, band-limited interpolation of a
  DSP-rate waveform onto the analog grid.

Pins: back-to-back recovery s_hat = s, Parseval power of the TX waveform,
finite differences of the loss, AWGN SNR estimator; front end: single-tone
closed forms (pass, reject, no alias, band edge), rho_a-rate TX sampled down
equals rho_d-rate TX, gamma = 0 propagation commutes with the front end, ASE
power after the front end independent of the simulation rate, interpolation
round trip.
"""
from __future__ import annotations

import numpy as np


def raised_cosine(nu, rolloff: float):
    """Raised-cosine spectrum of unit symbol rate at normalised frequency nu = f/R_s."""
    a = np.abs(nu)
    lo, hi = (1.0 - rolloff) / 2.0, (1.0 + rolloff) / 2.0
    out = np.zeros_like(a)
    out[a <= lo] = 1.0
    mid = (a > lo) & (a <= hi)
    out[mid] = 0.5 * (1.0 + np.cos(np.pi / rolloff * (a[mid] - lo)))
    return out


def rrc_response(n: int, sps: int, rolloff: float):
    """H_k = sqrt(sps * RC(f_k / R_s)) on the fftfreq grid."""
    nu = np.fft.fftfreq(n) * sps
    return np.sqrt(sps * raised_cosine(nu, rolloff))


def tx(symbols, sps: int, rolloff: float, power_w):
    """Eq. (11) sampled at sps samples/symbol; power_w scalar or per waveform [B]."""
    s = np.atleast_2d(np.asarray(symbols, dtype=np.complex128))
    B, nsym = s.shape
    n = nsym * sps
    u = np.zeros((B, n), dtype=np.complex128)
    u[:, ::sps] = s
    H = rrc_response(n, sps, rolloff)
    x = np.fft.ifft(np.fft.fft(u, axis=-1) * H, axis=-1)
    p = np.broadcast_to(np.asarray(power_w, dtype=np.float64), (B,))
    return x * np.sqrt(p * sps)[:, None]


def matched_filter(y, sps: int, rolloff: float, power_w):
    """M y / sqrt(P rho): FD RRC, keep every sps-th sample (Eq. (12))."""
    y = np.atleast_2d(np.asarray(y, dtype=np.complex128))
    B, n = y.shape
    H = rrc_response(n, sps, rolloff)
    z = np.fft.ifft(np.fft.fft(y, axis=-1) * H, axis=-1)[:, ::sps]
    p = np.broadcast_to(np.asarray(power_w, dtype=np.float64), (B,))
    return z / np.sqrt(p * sps)[:, None]


def phase_correct(z, s):
    phi = np.angle(np.sum(np.conj(s) * z, axis=-1))
    return z * np.exp(-1j * phi)[:, None], phi


def evaluate(y, s, sps: int, rolloff: float, power_w):
    """Receiver chain + loss + SNR.  Returns dict with mse[B], snr_db, snr_db_per, phi[B]."""
    s = np.atleast_2d(s)
    z = matched_filter(y, sps, rolloff, power_w)
    sh, phi = phase_correct(z, s)
    err = np.sum(np.abs(sh - s) ** 2, axis=-1)
    nsym = s.shape[-1]
    return dict(mse=err / nsym, loss=float(np.mean(err / nsym)),
                snr_db=float(10 * np.log10(np.sum(np.abs(s) ** 2) / np.sum(err))),
                snr_db_per=10 * np.log10(nsym / err), phi=phi, s_hat=sh)


def loss_grad(y, s, sps: int, rolloff: float, power_w):
    """Gradient of mean_b ||s_hat_b - s_b||^2 / N_sym w.r.t. y (phi held constant)."""
    s = np.atleast_2d(s)
    B, nsym = s.shape
    n = nsym * sps
    ev = evaluate(y, s, sps, rolloff, power_w)
    g_sh = 2.0 * (ev["s_hat"] - s) / (nsym * B)
    g_z = g_sh * np.exp(1j * ev["phi"])[:, None]
    p = np.broadcast_to(np.asarray(power_w, dtype=np.float64), (B,))
    up = np.zeros((B, n), dtype=np.complex128)
    up[:, ::sps] = g_z / np.sqrt(p * sps)[:, None]
    H = rrc_response(n, sps, rolloff)
    return np.fft.ifft(np.fft.fft(up, axis=-1) * H, axis=-1), ev


def brickwall_mask(n: int, band_bins: float):
    """Ideal low-pass on an n-bin DFT grid: 1 where |kappa| < band_bins / 2 (kappa signed, fftfreq order)."""
    kappa = np.fft.fftfreq(n) * n
    return (np.abs(kappa) < band_bins / 2.0).astype(np.float64)


def lowpass_sample(y, n_out: int, bandwidth: float = 1.0):
    """Receiver front end (Sec. IV-A): brick-wall low-pass, then sampling at t = k / f_s.

    y [B, n_in] on the analog grid (rho_a samples/symbol), n_out = rho_d N_sym
    with n_in a multiple of n_out.  Delta B = bandwidth * f_s spans
    bandwidth * n_out bins.  The filtered waveform is formed on the analog grid
    and every (n_in / n_out)-th sample is kept, offset 0.
    """
    y = np.atleast_2d(np.asarray(y, dtype=np.complex128))
    n_in = y.shape[-1]
    if n_out < 1 or n_in % n_out:
        raise ValueError("n_in must be a multiple of n_out")
    if not 0.0 < bandwidth <= 1.0:
        raise ValueError("bandwidth must be in (0, 1]")
    mask = brickwall_mask(n_in, bandwidth * n_out)
    z = np.fft.ifft(np.fft.fft(y, axis=-1) * mask, axis=-1)
    return z[:, :: n_in // n_out]


def interpolate(x, n_out: int):
    """Band-limited periodic interpolation of x [B, n_in] onto n_out >= n_in points.

    The samples at t = m T / n_out of the trigonometric polynomial with bins
    |kappa| < n_in / 2 that takes the values x at t = k T / n_in (the Nyquist
    bin, whose frequency sign is ambiguous, is left out).  n_out is a multiple
    of n_in.
    """
    x = np.atleast_2d(np.asarray(x, dtype=np.complex128))
    B, n_in = x.shape
    if n_out % n_in:
        raise ValueError("n_out must be a multiple of n_in")
    X = np.fft.fft(x, axis=-1) * brickwall_mask(n_in, n_in)
    kappa = np.rint(np.fft.fftfreq(n_in) * n_in).astype(np.int64)
    Y = np.zeros((B, n_out), dtype=np.complex128)
    Y[:, kappa % n_out] = X * (n_out / n_in)
    return np.fft.ifft(Y, axis=-1)
