"""Split-step Fourier method for the NLSE, FP64 (oracle side).

Definitions followed (Sec. III, III-A, III-C, IV-A of the paper):

* NLSE, Eq. (4):  du/dz = -(alpha/2) u - j (beta2/2) d^2u/dt^2 + j gamma |u|^2 u.
* Time-discretised NLSE, Eq. (5): A = F^-1 diag(H_k) F with
  H_k = j (beta2/2) omega_k^2, omega_k = 2 pi f_k on the DFT grid.  The
  printed index rule skips a bin; the grid used here is numpy's fftfreq
  (f_k/fs = k/n for k < n/2, (k-n)/n otherwise).  Only omega^2 enters, so the
  sign of the Nyquist bin is irrelevant.
* Linear operator (Sec. III-A): A_z = e^{-alpha z/2} F^-1 diag(e^{z H_k}) F.
  DFT is unnormalised e^{-j 2 pi k m / n}; the inverse carries 1/n.
* Nonlinear operator (Sec. III-A): sigma_z(x) = x exp(j gamma L_eff(z) |x|^2),
  L_eff(z) = (1 - e^{-alpha z}) / alpha.
* Asymmetric SSM, Eq. (6); symmetric SSM, Eq. (8).
* Link (Sec. IV-A): N_sp spans, an EDFA with gain e^{alpha L_sp} (power) after
  each span, white Gaussian ASE with PSD (e^{alpha L_sp} - 1) h nu_s n_sp,
  n_sp = NF / (2 (1 - e^{-alpha L_sp})).
* DBP (Sec. IV): solve the propagation backwards, i.e. the same operators with
  (beta2, gamma, alpha) -> (-beta2, -gamma, -alpha), spans in reverse order
  with the amplifier gain undone first.

Readings (the paper is silent or ambiguous):

* Symmetric step: the Kerr rotation sits at the step midpoint with the exact
  loss integral about the midpoint, l_mid(d) = 2 sinh(alpha d/2)/alpha.
* Asymmetric channel step: Kerr first (power at the segment start, where
  L_eff is exact), then the lossy linear step.  Asymmetric DBP is Eq. (6)
  literally: linear step (with gain) then Kerr with -gamma L_eff(d); it is the
  exact inverse of the asymmetric channel step.
* ASE is single polarisation, variance sigma^2 = PSD * fs per complex sample,
  added after the amplifier.  Its realisation is defined in the frequency
  domain: w = iDFT(W), W_k = sqrt(n sigma^2 / 2) g_k with g from
  ``philox.ase_normals``; a DFT of white Gaussian noise is white Gaussian, so
  the statistics are those of the paper.

Parity pins (tests/test_oracle_nlse.py): gamma = 0 closed form, beta2 = 0
closed form, alpha = 0 energy conservation, DBP-of-forward identity on the
same grid, fundamental soliton, symmetric O(M^-2) / asymmetric O(M^-1)
convergence, ASE variance formula; DBP with explicit (non-uniform) steps:
beta2 = 0 and gamma = 0 closed forms for any step sizes.
"""
from __future__ import annotations

import numpy as np

from . import philox

PLANCK = 6.626e-34  # Table I


def si_alpha(alpha_db_per_km: float) -> float:
    """Power attenuation coefficient in 1/m from dB/km."""
    return alpha_db_per_km * np.log(10.0) / 10.0 / 1e3


def si_beta2(beta2_ps2_per_km: float) -> float:
    """Group-velocity dispersion in s^2/m from ps^2/km."""
    return beta2_ps2_per_km * 1e-24 / 1e3


def si_gamma(gamma_per_w_km: float) -> float:
    """Kerr parameter in 1/(W m) from 1/(W km)."""
    return gamma_per_w_km / 1e3


def omega_grid(n: int, fs: float) -> np.ndarray:
    """omega_k = 2 pi f_k, fftfreq ordering (Eq. (5))."""
    return 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / fs)


def leff(alpha: float, z: float) -> float:
    """Effective nonlinear length (1 - e^{-alpha z})/alpha (Sec. III-A)."""
    if alpha == 0.0:
        return z
    return -np.expm1(-alpha * z) / alpha


def lmid(alpha: float, z: float) -> float:
    """Loss integral of a step of length z about its midpoint: 2 sinh(alpha z/2)/alpha."""
    if alpha == 0.0:
        return z
    return 2.0 * np.sinh(alpha * z / 2.0) / alpha


def linear_step(u, beta2: float, alpha: float, z: float, fs: float):
    """A_z u = e^{-alpha z/2} F^-1 diag(exp(j (beta2/2) omega_k^2 z)) F u (Sec. III-A)."""
    n = u.shape[-1]
    w = omega_grid(n, fs)
    U = np.fft.fft(u, axis=-1)
    U = U * np.exp(1j * (beta2 / 2.0) * w ** 2 * z)
    return np.fft.ifft(U, axis=-1) * np.exp(-alpha * z / 2.0)


def kerr(u, c: float):
    """Pointwise sigma(x) = x exp(j c |x|^2) (Sec. III-A)."""
    return u * np.exp(1j * c * np.abs(u) ** 2)


def ase_sigma2(alpha: float, span_m: float, nf_db: float, carrier_hz: float, fs: float) -> float:
    """Per-sample ASE variance PSD * fs (Sec. IV-A, Table I)."""
    nf = 10.0 ** (nf_db / 10.0)
    g = np.exp(alpha * span_m)
    nsp = nf / (2.0 * (1.0 - 1.0 / g))
    psd = (g - 1.0) * PLANCK * carrier_hz * nsp
    return psd * fs


def ase_noise(n: int, batch: int, span: int, sigma2: float, seed: int, counter: int):
    """Time-domain ASE realisation w = iDFT(W), W_k = sqrt(n sigma^2/2) g_k."""
    g = philox.ase_normals(n, batch, span, seed, counter)
    W = np.sqrt(n * sigma2 / 2.0) * g
    return np.fft.ifft(W, axis=-1)


def channel(x, fiber, link, fs: float, steps=None):
    """Forward split-step propagation over the link (Eqs. (6)/(8), Sec. IV-A).

    x: complex [B, n] (or [n]) launch waveform in sqrt(W).
    fiber: object with alpha_db_per_km, beta2_ps2_per_km, gamma_per_w_km.
    link: object with n_spans, span_km, steps_per_span, symmetric, ase,
          nf_db, carrier_hz, seed, counter.
    """
    u = np.array(x, dtype=np.complex128, copy=True)
    squeeze = u.ndim == 1
    if squeeze:
        u = u[None, :]
    alpha, beta2, gamma = si_alpha(fiber.alpha_db_per_km), si_beta2(fiber.beta2_ps2_per_km), si_gamma(fiber.gamma_per_w_km)
    Lsp = link.span_km * 1e3
    N = link.steps_per_span if steps is None else steps
    d = Lsp / N
    gain = np.exp(alpha * Lsp / 2.0)
    sig2 = ase_sigma2(alpha, Lsp, link.nf_db, link.carrier_hz, fs) if link.ase else 0.0
    for s in range(link.n_spans):
        for _ in range(N):
            if link.symmetric:
                u = linear_step(u, beta2, alpha, d / 2.0, fs)
                u = kerr(u, gamma * lmid(alpha, d))
                u = linear_step(u, beta2, alpha, d / 2.0, fs)
            else:
                u = kerr(u, gamma * leff(alpha, d))
                u = linear_step(u, beta2, alpha, d, fs)
        u = u * gain
        if link.ase:
            u = u + ase_noise(u.shape[-1], u.shape[0], s, sig2, link.seed, link.counter)
    return u[0] if squeeze else u


def dbp(y, fiber, link, fs: float, steps_per_span: int, symmetric: bool):
    """Digital backpropagation: the SSM run backwards (Sec. IV, Eqs. (6)/(8)).

    Spans in reverse order; per span the amplifier gain is undone, then the
    steps are applied with (beta2, gamma, alpha) -> (-beta2, -gamma, -alpha).
    """
    u = np.array(y, dtype=np.complex128, copy=True)
    squeeze = u.ndim == 1
    if squeeze:
        u = u[None, :]
    alpha, beta2, gamma = si_alpha(fiber.alpha_db_per_km), si_beta2(fiber.beta2_ps2_per_km), si_gamma(fiber.gamma_per_w_km)
    Lsp = link.span_km * 1e3
    N = steps_per_span
    d = Lsp / N
    gain = np.exp(alpha * Lsp / 2.0)
    for _ in range(link.n_spans):
        u = u / gain
        for _ in range(N):
            if symmetric:
                u = linear_step(u, -beta2, -alpha, d / 2.0, fs)
                u = kerr(u, -gamma * lmid(alpha, d))
                u = linear_step(u, -beta2, -alpha, d / 2.0, fs)
            else:
                u = linear_step(u, -beta2, -alpha, d, fs)
                u = kerr(u, -gamma * leff(alpha, d))
    return u[0] if squeeze else u


def dbp_steps(y, fiber, n_spans: int, span_km: float, steps_km, fs: float, symmetric: bool):
    """DBP (Sec. IV) with explicit step sizes: steps_km lists the steps of one
    span in DBP order (the first step starts at the span end, where the
    amplifier gain has been undone); every span uses the same list.  With
    steps_km = [L_sp / N] * N this is ``dbp``.  Non-uniform steps are the
    logarithmic step sizes of Sec. IV-C (Example 1).
    """
    u = np.array(y, dtype=np.complex128, copy=True)
    squeeze = u.ndim == 1
    if squeeze:
        u = u[None, :]
    alpha, beta2, gamma = si_alpha(fiber.alpha_db_per_km), si_beta2(fiber.beta2_ps2_per_km), si_gamma(fiber.gamma_per_w_km)
    Lsp = span_km * 1e3
    gain = np.exp(alpha * Lsp / 2.0)
    for _ in range(n_spans):
        u = u / gain
        for dk in steps_km:
            d = dk * 1e3
            if symmetric:
                u = linear_step(u, -beta2, -alpha, d / 2.0, fs)
                u = kerr(u, -gamma * lmid(alpha, d))
                u = linear_step(u, -beta2, -alpha, d / 2.0, fs)
            else:
                u = linear_step(u, -beta2, -alpha, d, fs)
                u = kerr(u, -gamma * leff(alpha, d))
    return u[0] if squeeze else u


def cd_memory_samples(beta2_ps2_per_km: float, delta_f_hz: float, length_km: float, fs: float) -> float:
    """T_cd = 2 pi |beta2| Delta_f L fs (Eq. (15))."""
    return 2.0 * np.pi * abs(si_beta2(beta2_ps2_per_km)) * delta_f_hz * length_km * 1e3 * fs
