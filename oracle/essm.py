"""Learned enhanced SSM (filtered DBP), FP64 (oracle side; test infrastructure only).

Model (Sec. III-C, Eqs. (9)-(10): the filtered nonlinear step of the enhanced
SSM, one filter per step): the LDBP model of Eq. (7) whose nonlinear steps
use a low-pass filtered power,
    [sigma_i(x)]_j = x_j exp(j c_i sum_{k=-kappa_i}^{kappa_i} eta^(i)_k |x_{j-k}|^2),
indices modulo n, with real filters eta^(i) = (eta_{-kappa}, ..., eta_0, ...,
eta_kappa) (not necessarily symmetric) and c_i = -gamma L_eff(delta_i) for DBP.
theta = {h^(i), eta^(i)}.  With eta^(i) = (1) (kappa_i = 0) this is LDBP.

Pins (tests/test_oracle_essm.py): the unit filter reduces to ldbp.forward; the
filtered power equals a dense real circulant matrix times |x|^2 (brute force);
a constant-modulus input a gets the uniform phase c a^2 sum_k eta_k.
"""
from __future__ import annotations

import numpy as np

from . import ldbp


def filtered_power(x, eta):
    """p_j = sum_{k=-kappa}^{kappa} eta_k |x_{j-k}|^2 (circular), eta = (eta_{-kappa}, ..., eta_kappa)."""
    eta = np.asarray(eta, dtype=np.float64)
    kappa = (len(eta) - 1) // 2
    p = np.abs(np.asarray(x)) ** 2
    out = np.zeros_like(p)
    for k in range(-kappa, kappa + 1):
        out = out + eta[k + kappa] * np.roll(p, k, axis=-1)
    return out


def forward(x, taps, c, etas):
    """Filtered-nonlinearity LDBP forward.  Returns (y, inputs), inputs[i] the input of step i."""
    u = np.asarray(x, dtype=np.complex128)
    inputs = []
    for h, ci, eta in zip(taps, c, etas):
        inputs.append(u)
        v = ldbp.fir(u, np.asarray(h, dtype=np.complex128))
        u = v * np.exp(1j * ci * filtered_power(v, eta))
    return u, inputs


def backward(x, taps, c, etas, gy):
    """Reverse sweep of the filtered-nonlinearity model.

    Returns (gx, gtaps, getas) for the loss gradient gy (convention
    g = dl/dRe + j dl/dIm of a real loss), summed over leading (batch) axes.
    Per step, with v = A u, p = |v|^2, phi = eta * p (circular), w = v e^{j c phi}
    and g the gradient at w:
      a_j = dl/dphi_j = -c Im(w_j conj(g_j)),
      dl/dp_m = sum_k eta_k a_{m+k}          (the filter transposed),
      g_v = e^{-j c phi} g + 2 (dl/dp) v,
      dl/deta_k = sum_j a_j p_{j-k},
    then the FIR adjoint and tap gradients of ldbp.backward.
    """
    _, inputs = forward(x, taps, c, etas)
    g = np.asarray(gy, dtype=np.complex128)
    gtaps, getas = [None] * len(taps), [None] * len(taps)
    for i in reversed(range(len(taps))):
        h = np.asarray(taps[i], dtype=np.complex128)
        eta = np.asarray(etas[i], dtype=np.float64)
        kappa = (len(eta) - 1) // 2
        u = inputs[i]
        v = ldbp.fir(u, h)
        p = np.abs(v) ** 2
        phi = filtered_power(v, eta)
        w = v * np.exp(1j * c[i] * phi)
        a = -c[i] * np.imag(w * np.conj(g))
        dp = np.zeros_like(p)
        for k in range(-kappa, kappa + 1):
            dp = dp + eta[k + kappa] * np.roll(a, -k, axis=-1)
        getas[i] = np.array([np.sum(a * np.roll(p, k, axis=-1)) for k in range(-kappa, kappa + 1)])
        gv = np.exp(-1j * c[i] * phi) * g + 2.0 * dp * v
        gh = np.zeros(len(h), dtype=np.complex128)
        gh[0] = np.sum(gv * np.conj(u))
        for k in range(1, len(h)):
            gh[k] = np.sum(gv * np.conj(np.roll(u, k, axis=-1) + np.roll(u, -k, axis=-1)))
        gtaps[i] = gh
        g = ldbp.fir(gv, np.conj(h))
    return g, gtaps, getas
