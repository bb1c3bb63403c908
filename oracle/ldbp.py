"""Learned DBP model, its adjoint and its reference initialisation, FP64 (oracle side).

Model (Eq. (7) with the symmetric-FIR constraint of Sec. III-B):
  f_theta(x) = sigma_M(A^(M) ... sigma_1(A^(1) x)),
  A^(i) = circular convolution whose rows are circular shifts of
  (h_K, ..., h_1, h_0, h_1, ..., h_K, 0, ..., 0), theta = {(h_0..h_K)^(i)},
  T_i = 2 K_i + 1; sigma_i(x) = x exp(j c_i |x|^2) with a fixed c_i
  (c_i = -gamma L_eff(delta_i) for DBP; c_i = 0 gives the linear-only last
  layer of a symmetric-SSM-based model, Sec. III-C).
  FIR (circular, index mod n): y_m = sum_{k=-K}^{K} h_|k| x_{m-k}.

Adjoint (gradients in the convention g = dl/dRe + j dl/dIm of a real loss):
  Kerr y = x e^{j c |x|^2}:  gx = e^{-j c |x|^2} gy - 2 c Im(y conj(gy)) x
  FIR  y = A x:               gx = A^H gy  (the same symmetric FIR with conj taps)
  taps:  dl/dh_0 = sum_m gv_m conj(x_m);  dl/dh_k = sum_m gv_m conj(x_{m-k} + x_{m+k})
The Kerr adjoint follows from Wirtinger calculus: with E = e^{j c |x|^2},
dy = E (1 + j c |x|^2) dx + j c E x^2 dx*, so 2 dl/dx* = conj(E)(1 - j c |x|^2) g +
j c E x^2 conj(g) = conj(E) g - 2 c Im(y conj(g)) x; it is pinned by
central finite differences on the FP64 forward (tests/test_oracle_ldbp.py).

Least-squares initialisation (Sec. IV-C): minimise ||B h - d||^2 with
d_i = exp(j xi w_i^2), B the (N+1) x T DTFT matrix e^{-j k w_i}, k = -K..K,
w_i = 2 pi i / N, i = -N/2..N/2, xi = -beta2 delta' fs^2 / 2, and the symmetric
tie h_{-k} = h_k.  The constrained variant the paper uses is in a reference
that is not available, so this is the unconstrained fit, optionally restricted
to a band |w| <= w_max.

Pins: dense circulant brute force, adjoint identity <Ax, y> = <x, A^H y>,
finite-difference gradients (taps, input and the coefficients c), LDBP ==
asymmetric FD DBP when T = n (n odd).
"""
from __future__ import annotations

import numpy as np


def fir(x, h):
    """Circular symmetric FIR with half-taps h = (h_0, ..., h_K) along the last axis."""
    y = h[0] * x
    for k in range(1, len(h)):
        y = y + h[k] * (np.roll(x, k, axis=-1) + np.roll(x, -k, axis=-1))
    return y


def circulant_matrix(h, n: int) -> np.ndarray:
    """Dense n x n matrix A^(i) of Sec. III-B (row m, column (m-k) mod n holds h_|k|)."""
    A = np.zeros((n, n), dtype=np.complex128)
    K = len(h) - 1
    for m in range(n):
        for k in range(-K, K + 1):
            A[m, (m - k) % n] += h[abs(k)]
    return A


def kerr(x, c):
    return x * np.exp(1j * c * np.abs(x) ** 2)


def forward(x, taps, c):
    """Eq. (7) with FIR steps.  taps: list of half-tap vectors; c: per-step coefficients.

    Returns (y, inputs) where inputs[i] is the input of step i.
    """
    u = np.asarray(x, dtype=np.complex128)
    inputs = []
    for h, ci in zip(taps, c):
        inputs.append(u)
        u = kerr(fir(u, np.asarray(h, dtype=np.complex128)), ci)
    return u, inputs


def backward(x, taps, c, gy):
    """Reverse sweep of the model.  Returns (gx, gtaps) with gtaps[i] shaped like taps[i].

    x: [..., n]; gy: gradient at the output, same shape.
    Tap gradients are summed over all leading (batch) axes.
    """
    _, inputs = forward(x, taps, c)
    g = np.asarray(gy, dtype=np.complex128)
    gtaps = [None] * len(taps)
    for i in reversed(range(len(taps))):
        h = np.asarray(taps[i], dtype=np.complex128)
        u = inputs[i]
        v = fir(u, h)
        w = kerr(v, c[i])
        gv = np.exp(-1j * c[i] * np.abs(v) ** 2) * g - 2.0 * c[i] * np.imag(w * np.conj(g)) * v
        gh = np.zeros(len(h), dtype=np.complex128)
        gh[0] = np.sum(gv * np.conj(u))
        for k in range(1, len(h)):
            gh[k] = np.sum(gv * np.conj(np.roll(u, k, axis=-1) + np.roll(u, -k, axis=-1)))
        gtaps[i] = gh
        g = fir(gv, np.conj(h))
    return g, gtaps


def grad_c(x, taps, c, gy):
    """Gradients of a real loss with respect to the nonlinear coefficients c_i
    (the learnable scaling of the nonlinear steps, Remark 1: c_i = eta_i gamma
    L_eff(delta_i)).  With w = v e^{j c p}, p = |v|^2 and g the gradient at w,
    dl/dc = Re(conj(g) dw/dc) summed = -sum_m p_m Im(w_m conj(g_m)).
    Summed over all leading (batch) axes; the reverse sweep is that of backward.
    """
    _, inputs = forward(x, taps, c)
    g = np.asarray(gy, dtype=np.complex128)
    gc = [0.0] * len(taps)
    for i in reversed(range(len(taps))):
        h = np.asarray(taps[i], dtype=np.complex128)
        v = fir(inputs[i], h)
        w = kerr(v, c[i])
        gc[i] = float(-np.sum(np.abs(v) ** 2 * np.imag(w * np.conj(g))))
        gv = np.exp(-1j * c[i] * np.abs(v) ** 2) * g - 2.0 * c[i] * np.imag(w * np.conj(g)) * v
        g = fir(gv, np.conj(h))
    return gc


def ls_taps(T: int, xi: float, N: int = 1024, w_max: float = np.pi, gain: float = 1.0):
    """Unconstrained least-squares symmetric FIR fit of gain*exp(j xi w^2) (Sec. IV-C).

    Returns the half-vector (h_0, ..., h_K), K = (T-1)/2.
    """
    K = (T - 1) // 2
    i = np.arange(-N // 2, N // 2 + 1)
    w = 2.0 * np.pi * i / N
    keep = np.abs(w) <= w_max + 1e-12
    w = w[keep]
    d = gain * np.exp(1j * xi * w ** 2)
    # Symmetric tie: column k of the reduced matrix is e^{-j k w} + e^{+j k w} for k > 0.
    B = np.empty((len(w), K + 1), dtype=np.complex128)
    B[:, 0] = 1.0
    for k in range(1, K + 1):
        B[:, k] = np.exp(-1j * k * w) + np.exp(1j * k * w)
    h, *_ = np.linalg.lstsq(B, d, rcond=None)
    return h


def dbp_taps_full(n: int, xi: float, gain: float = 1.0):
    """Half-taps of the length-n (n odd) symmetric FIR equal to iDFT(gain exp(j xi w_k^2))."""
    assert n % 2 == 1
    w = 2.0 * np.pi * np.fft.fftfreq(n)
    h = np.fft.ifft(gain * np.exp(1j * xi * w ** 2))
    return h[: (n - 1) // 2 + 1]
