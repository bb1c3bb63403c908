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


def _loss_grad(x, taps, c, etas, t):
    y, _ = essm.forward(x, taps, c, etas)
    return float(np.sum(np.abs(y - t) ** 2)), 2.0 * (y - t)


def test_backward_unit_filter_is_ldbp_backward():
    taps = [synth.complex_normal(3, 20, 0.5), synth.complex_normal(5, 21, 0.4)]
    c = [0.8, -1.2]
    x = synth.complex_normal(96, 22, 0.7).reshape(2, 48)
    gy = synth.complex_normal(96, 23, 1.0).reshape(2, 48)
    gx0, gt0 = ldbp.backward(x, taps, c, gy)
    gx1, gt1, ge1 = essm.backward(x, taps, c, [np.array([1.0])] * 2, gy)
    assert np.allclose(gx0, gx1, atol=1e-13) and all(np.allclose(a, b, atol=1e-12) for a, b in zip(gt0, gt1))


def test_backward_finite_differences():
    # central differences of the FP64 forward for the filter taps eta, the FIR
    # taps and the input, with asymmetric eta (kappa 2 and 3)
    rng = np.random.default_rng(30)
    n = 40
    taps = [synth.complex_normal(3, 31, 0.5), synth.complex_normal(2, 32, 0.5)]
    c = [1.1, -0.7]
    etas = [rng.normal(0.2, 0.3, 5), rng.normal(0.1, 0.3, 7)]
    x = synth.complex_normal(2 * n, 33, 0.8).reshape(2, n)
    t = synth.complex_normal(2 * n, 34, 0.8).reshape(2, n)
    _, gy = _loss_grad(x, taps, c, etas, t)
    gx, gt, ge = essm.backward(x, taps, c, etas, gy)
    e = 1e-6
    for i in range(2):
        for k in range(len(etas[i])):
            ep = [a.copy() for a in etas]
            em = [a.copy() for a in etas]
            ep[i][k] += e
            em[i][k] -= e
            fd = (_loss_grad(x, taps, c, ep, t)[0] - _loss_grad(x, taps, c, em, t)[0]) / (2 * e)
            assert abs(ge[i][k] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, k)
        for k in range(len(taps[i])):
            for d in (1.0, 1j):
                tp = [a.copy() for a in taps]
                tm = [a.copy() for a in taps]
                tp[i][k] += e * d
                tm[i][k] -= e * d
                fd = (_loss_grad(x, tp, c, etas, t)[0] - _loss_grad(x, tm, c, etas, t)[0]) / (2 * e)
                got = gt[i][k].real if d == 1.0 else gt[i][k].imag
                assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (i, k, d)
    for j in (0, 7, 39):
        for d in (1.0, 1j):
            xp, xm = x.copy(), x.copy()
            xp[1, j] += e * d
            xm[1, j] -= e * d
            fd = (_loss_grad(xp, taps, c, etas, t)[0] - _loss_grad(xm, taps, c, etas, t)[0]) / (2 * e)
            got = gx[1, j].real if d == 1.0 else gx[1, j].imag
            assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd))
