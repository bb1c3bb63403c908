"""Host-side (FP64) set-up of learned-DBP parameters.

* Step sizes: uniform delta = L_sp / StPS per span (the configurations here use
  uniform steps); `merge_half_steps` combines adjacent half-steps of a
  symmetric-SSM layout into the layer lengths delta'_1..delta'_{M+1}
  (Sec. IV-C, Example 1).
* Filters: least-squares fit of the CD-inverting response exp(j xi w^2),
  xi = -beta2 delta' fs^2 / 2, w = 2 pi f / fs (Sec. IV-C).  A symmetric FIR
  has the real-basis response h_0 + sum_k 2 h_k cos(k w), so the fit is a real
  least-squares problem on the cosine basis with a complex target, solved on a
  dense grid of w restricted to |w| <= w_max (the signal band by default: the
  in-band criterion of the constrained variant the paper uses).  A small ridge
  term bounds the out-of-band gain.
* Nonlinear coefficients: c_i = -gamma L_eff(delta'_i) (Sec. III-A), fixed
  during training (Sec. III-B, Remark 1).
"""
from __future__ import annotations

import math

import numpy as np


def _si(fiber):
    a = fiber.alpha_db_per_km * math.log(10.0) / 10.0 / 1e3
    b2 = fiber.beta2_ps2_per_km * 1e-27
    g = fiber.gamma_per_w_km * 1e-3
    return a, b2, g


def effective_length(alpha: float, z: float) -> float:
    return z if alpha == 0.0 else -math.expm1(-alpha * z) / alpha


def merge_half_steps(deltas):
    """delta'_1 = delta_1/2, delta'_i = (delta_{i-1} + delta_i)/2, delta'_{M+1} = delta_M/2."""
    d = list(deltas)
    return [d[0] / 2.0] + [(d[i - 1] + d[i]) / 2.0 for i in range(1, len(d))] + [d[-1] / 2.0]


def _cos_basis(w, K):
    C = np.ones((len(w), K + 1))
    for k in range(1, K + 1):
        C[:, k] = 2.0 * np.cos(k * w)
    return C


def ls_symmetric_fir(T: int, xi: float, w_max: float = math.pi, gain: float = 1.0, grid: int = 2048,
                     max_oob_gain: float = 1.0) -> np.ndarray:
    """Half-taps (h_0..h_K) whose response h_0 + sum 2 h_k cos(k w) fits gain exp(j xi w^2) in band.

    The in-band error (|w| <= w_max) is minimised with an out-of-band penalty
    lam |H(w)|^2 that grows until the out-of-band gain is at most
    max_oob_gain |gain| (the in-band fit with an out-of-band gain cap that the
    paper uses), so that a cascade of many steps does not amplify out-of-band
    noise.
    """
    K = (T - 1) // 2
    w = np.linspace(-math.pi, math.pi, 2 * grid + 1)
    inb = np.abs(w) <= w_max + 1e-12
    C = _cos_basis(w, K)
    target = gain * np.exp(1j * xi * w * w)
    Ci, Co = C[inb], C[~inb]
    rhs = Ci.T @ target[inb]
    cap = max_oob_gain * abs(gain)
    lam = 0.0
    for _ in range(200):
        A = Ci.T @ Ci + lam * (Co.T @ Co) + 1e-9 * len(w) * np.eye(K + 1)
        h = np.linalg.solve(A, rhs.real) + 1j * np.linalg.solve(A, rhs.imag)
        if Co.shape[0] == 0 or float(np.max(np.abs(Co @ h))) <= cap:
            break
        lam = 1e-4 if lam == 0.0 else lam * 1.5
    return h


def signal_band(sps: int = 2, rolloff: float = 0.1) -> float:
    """Normalised angular half-bandwidth pi (1 + rolloff) / sps of the RRC signal."""
    return math.pi * (1.0 + rolloff) / sps


def ldbp_init(Ts, span_km: float, fs: float, steps_per_span: int = 1, fiber=None, w_max=None,
              sps: int = 2, rolloff: float = 0.1):
    """Filters and Kerr coefficients for asymmetric-SSM-based LDBP with uniform steps.

    Returns (taps, c): taps[i] is the complex half-tap vector of step i and
    c[i] = -gamma L_eff(delta) its nonlinear coefficient.
    """
    if fiber is None:
        import synth
        fiber = synth.Fiber()
    alpha, b2, gamma = _si(fiber)
    delta = span_km * 1e3 / steps_per_span
    xi = -b2 * delta * fs * fs / 2.0
    wm = signal_band(sps, rolloff) * 1.05 if w_max is None else w_max
    taps = [ls_symmetric_fir(T, xi, wm) for T in Ts]
    c = [-gamma * effective_length(alpha, delta)] * len(Ts)
    return taps, c
