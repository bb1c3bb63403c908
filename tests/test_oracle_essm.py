"""Pins of the filtered-nonlinearity (learned ESSM) oracle."""
import numpy as np

import synth
from oracle import essm, ldbp


def test_unit_filter_is_ldbp():
    taps = [synth.complex_normal(3, 1, 0.4), synth.complex_normal(5, 2, 0.3)]
    c = [0.7, -1.1]
    x = synth.complex_normal(64, 3, 0.8).reshape(1, 64)
    y0, _ = ldbp.forward(x, taps, c)
    y1, _ = essm.forward(x, taps, c, [np.array([1.0]), np.array([0.0, 1.0, 0.0])])
    assert np.allclose(y0, y1, rtol=0, atol=1e-14)


def test_filtered_power_dense_circulant():
    # brute force: the filter is a real circulant matrix acting on |x|^2; an
    # asymmetric eta catches a flipped index (eta_k applied to |x_{j+k}|^2)
    n, kappa = 23, 4
    rng = np.random.default_rng(5)
    eta = rng.normal(size=2 * kappa + 1)
    x = synth.complex_normal(n, 6, 1.0)
    C = np.zeros((n, n))
    for j in range(n):
        for k in range(-kappa, kappa + 1):
            C[j, (j - k) % n] += eta[k + kappa]
    assert np.allclose(essm.filtered_power(x, eta), C @ np.abs(x) ** 2, rtol=0, atol=1e-13)
    assert not np.allclose(essm.filtered_power(x, eta[::-1]), C @ np.abs(x) ** 2, atol=1e-6)


def test_constant_modulus_gets_uniform_phase():
    n, a, ci = 40, 0.6, -0.9
    eta = np.array([0.1, 0.25, 0.3, 0.2, 0.05])
    x = a * np.exp(2j * np.pi * np.arange(n) / n * 3)
    y, _ = essm.forward(x.reshape(1, n), [np.array([1.0 + 0j])], [ci], [eta])
    assert np.allclose(y[0], x * np.exp(1j * ci * a * a * eta.sum()), rtol=0, atol=1e-14)
