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
