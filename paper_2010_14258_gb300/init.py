"""Host-side (FP64) set-up of learned-DBP parameters.

* Step sizes: uniform delta = L_sp / StPS per span, or logarithmic step sizes
  (Sec. IV-C: the heuristic with adjusting factor 0.4, `log_step_sizes`);
  `merge_half_steps` combines adjacent half-steps of a symmetric-SSM layout
  into the layer lengths delta'_1..delta'_{M+1} (Sec. IV-C, Example 1), and
  `symmetric_layers` adds each layer's gain and Kerr coefficient.
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


def log_step_sizes(span_km: float, steps_per_span: int, fiber=None, zeta: float = 0.4):
    """Logarithmic step sizes of one span (km), in DBP order (Sec. IV-C).

    Reading of the heuristic the paper uses with adjusting factor zeta = 0.4:
    the steps keep the nonlinear phase of a loss profile exp(-zeta alpha z)
    constant, i.e. from the span start (full power)
        d_n = -ln((1 - n s) / (1 - (n - 1) s)) / (zeta alpha),
        s = (1 - exp(-zeta alpha L_sp)) / StPS,  n = 1..StPS,
    which sum to L_sp; DBP traverses the span from its end, so the list is
    returned reversed.  For L_sp = 100 km and 2 StPS this gives 70.4 / 29.6 km,
    the values of Example 1.
    """
    if fiber is None:
        import synth
        fiber = synth.Fiber()
    alpha = _si(fiber)[0] * 1e3  # 1/km
    K = int(steps_per_span)
    if alpha == 0.0 or zeta == 0.0:
        return [span_km / K] * K
    za = zeta * alpha
    s = -math.expm1(-za * span_km) / K
    fwd = [-math.log((1.0 - n * s) / (1.0 - (n - 1) * s)) / za for n in range(1, K + 1)]
    return fwd[::-1]


def lmid(alpha: float, z: float) -> float:
    """Loss integral of a step about its midpoint, 2 sinh(alpha z / 2) / alpha."""
    return z if alpha == 0.0 else 2.0 * math.sinh(alpha * z / 2.0) / alpha


def symmetric_layers(n_spans: int, span_km: float, steps_km, fiber=None):
    """Layers of symmetric-SSM-based LDBP (Sec. III-C, IV-C): l = M + 1 layers.

    steps_km: the step sizes of one span in DBP order (uniform or
    `log_step_sizes`), repeated for every span.  DBP undoes the amplifier gain
    at the start of each span and then applies, per step d, a linear half-step
    (dispersion -beta2, gain e^{alpha d/4}), the Kerr step with
    c = -gamma l_mid(d) and another linear half-step.  Adjacent half-steps
    merge (scalars commute with the linear operator), so layer m has length
    delta'_m (`merge_half_steps`), amplitude gain e^{alpha delta'_m / 2},
    divided by the span's amplifier gain e^{alpha L_sp / 2} where a span
    starts, and Kerr coefficient c_m; the last layer is linear-only (c = 0).
    Returns (delta_km, gain, c) lists of length M + 1.
    """
    if fiber is None:
        import synth
        fiber = synth.Fiber()
    alpha, _, gamma = _si(fiber)
    steps = [float(d) for d in steps_km]
    K = len(steps)
    d_all = steps * int(n_spans)
    M = len(d_all)
    dprime = merge_half_steps(d_all)
    G = math.exp(alpha * span_km * 1e3 / 2.0)
    gains, cs = [], []
    for m in range(M + 1):
        g = math.exp(alpha * dprime[m] * 1e3 / 2.0)
        if m < M and m % K == 0:  # the layer that holds the start of a span (in DBP order)
            g /= G
        gains.append(g)
        cs.append(-gamma * lmid(alpha, d_all[m] * 1e3) if m < M else 0.0)
    return dprime, gains, cs


def ldbp_init_symmetric(Ts, n_spans: int, span_km: float, fs: float, steps_per_span: int = 2, fiber=None,
                        log_steps: bool = True, w_max=None, sps: int = 2, rolloff: float = 0.1):
    """Filters and Kerr coefficients of symmetric-SSM-based LDBP (l = M + 1 layers).

    Ts: one filter length for every layer, or a list of l lengths.  Each layer's
    filter is the least-squares fit of gain_m exp(j xi_m w^2),
    xi_m = -beta2 delta'_m fs^2 / 2, on the signal band.
    """
    if fiber is None:
        import synth
        fiber = synth.Fiber()
    _, b2, _ = _si(fiber)
    steps = log_step_sizes(span_km, steps_per_span, fiber) if log_steps else [span_km / steps_per_span] * steps_per_span
    dprime, gains, cs = symmetric_layers(n_spans, span_km, steps, fiber)
    L = len(dprime)
    Ts = [int(Ts)] * L if np.isscalar(Ts) else list(Ts)
    if len(Ts) != L:
        raise ValueError(f"need {L} filter lengths, got {len(Ts)}")
    wm = signal_band(sps, rolloff) * 1.05 if w_max is None else w_max
    taps = [ls_symmetric_fir(T, -b2 * d * 1e3 * fs * fs / 2.0, wm, gain=g) for T, d, g in zip(Ts, dprime, gains)]
    return taps, cs


def unit_filters(Ts):
    """Unit filters h = (1, 0, ..., 0) (Sec. V-E): the link-agnostic initialisation."""
    out = []
    for T in Ts:
        h = np.zeros((T - 1) // 2 + 1, np.complex128)
        h[0] = 1.0
        out.append(h)
    return out


def random_filters(Ts, seed: int):
    """Random filters (Sec. V-E): real and imaginary parts i.i.d. N(0, 1), each filter
    divided by sum_{k=-K}^{K} |h_k|^2 (the paper's normalisation; its printed bounds
    -T..T read as -K..K, over both halves of the symmetric filter)."""
    rng = np.random.default_rng(seed)
    out = []
    for T in Ts:
        K = (T - 1) // 2
        h = rng.normal(size=K + 1) + 1j * rng.normal(size=K + 1)
        energy = abs(h[0]) ** 2 + 2.0 * float(np.sum(np.abs(h[1:]) ** 2))
        out.append(h / energy)
    return out
