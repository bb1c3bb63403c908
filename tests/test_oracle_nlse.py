"""Pins of the FP64 split-step oracle against what the paper and the mathematics fix."""
import numpy as np
import pytest

import synth
from oracle import nlse, philox
from tests.conftest import golden_path


def _read_golden(name):
    rows = {}
    for line in open(golden_path(name)):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows[parts[0]] = float(parts[1])
    return rows


def test_philox_known_answers():
    for line in open(golden_path("philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        ctr = np.array(w[0:4], dtype=np.uint64)
        key = np.array(w[4:6], dtype=np.uint64)
        out = philox.philox4x32_10(ctr[None, :], key[None, :])[0]
        assert [int(v) for v in out] == w[6:10]


def test_ase_normals_statistics():
    g = philox.ase_normals(4096, 8, span=3, seed=1234, counter=7)
    assert abs(np.mean(g)) < 0.03
    assert abs(np.mean(np.abs(g) ** 2) - 2.0) < 0.05
    assert abs(np.mean(g.real * g.imag)) < 0.03
    k = np.mean(g.real ** 4) / np.mean(g.real ** 2) ** 2
    assert abs(k - 3.0) < 0.15
    # distinct spans / counters give independent draws
    g2 = philox.ase_normals(4096, 8, span=4, seed=1234, counter=7)
    assert abs(np.mean(g * np.conj(g2))) < 0.05


def _fiber(alpha=0.2, beta2=-21.7, gamma=1.3):
    return synth.Fiber(alpha, beta2, gamma)


def _link(**kw):
    base = dict(n_spans=2, span_km=80.0, steps_per_span=8, symmetric=True, ase=False)
    base.update(kw)
    return synth.Link(**base)


def _x(n=512, B=2, pw=1e-3, seed=0):
    return synth.gaussian_waveform(B, n, seed, pw)


@pytest.mark.parametrize("symmetric", [True, False])
def test_gamma0_is_closed_form_allpass(symmetric):
    fs = 20e9
    x = _x()
    f = _fiber(gamma=0.0)
    link = _link(symmetric=symmetric, steps_per_span=7)
    y = nlse.channel(x, f, link, fs)
    # closed form: exp(j beta2/2 w^2 L) over the whole link; loss and gain cancel
    L = link.n_spans * link.span_km * 1e3
    w = 2 * np.pi * np.fft.fftfreq(x.shape[-1], 1 / fs)
    b2 = -21.7e-27
    ref = np.fft.ifft(np.fft.fft(x, axis=-1) * np.exp(1j * b2 / 2 * w ** 2 * L), axis=-1)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("symmetric", [True, False])
def test_beta0_is_closed_form_spm(symmetric):
    fs = 20e9
    x = _x(pw=5e-3)
    f = _fiber(beta2=0.0)
    link = _link(symmetric=symmetric, steps_per_span=5)
    y = nlse.channel(x, f, link, fs)
    a = 0.2 * np.log(10) / 10 / 1e3
    Lsp = 80e3
    leff = (1 - np.exp(-a * Lsp)) / a
    ref = x * np.exp(1j * 1.3e-3 * leff * link.n_spans * np.abs(x) ** 2)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-12


def test_alpha0_energy_conserved():
    fs = 20e9
    x = _x(pw=10e-3)
    y = nlse.channel(x, _fiber(alpha=0.0), _link(steps_per_span=13), fs)
    e0 = np.sum(np.abs(x) ** 2, axis=-1)
    e1 = np.sum(np.abs(y) ** 2, axis=-1)
    assert np.max(np.abs(e1 / e0 - 1)) < 1e-12


@pytest.mark.parametrize("symmetric", [True, False])
def test_dbp_inverts_forward_on_same_grid(symmetric):
    fs = 20e9
    x = _x(pw=8e-3)
    link = _link(symmetric=symmetric, steps_per_span=6, n_spans=3)
    y = nlse.channel(x, _fiber(), link, fs)
    xr = nlse.dbp(y, _fiber(), link, fs, steps_per_span=6, symmetric=symmetric)
    assert np.linalg.norm(xr - x) / np.linalg.norm(x) < 1e-12
    # a different DBP grid does not invert exactly but is close at low power
    x1 = _x(pw=0.5e-3)
    y1 = nlse.channel(x1, _fiber(), link, fs)
    xr2 = nlse.dbp(y1, _fiber(), link, fs, steps_per_span=1, symmetric=symmetric)
    assert 1e-9 < np.linalg.norm(xr2 - x1) / np.linalg.norm(x1) < 0.1


def test_fundamental_soliton_keeps_shape():
    # alpha = 0, beta2 < 0: u = sqrt(P0) sech(t/T0) with P0 = |beta2|/(gamma T0^2)
    # propagates as u(0,t) exp(j z / (2 L_D)), L_D = T0^2/|beta2|  (Eq. (4)).
    T0 = 20e-12
    b2 = -21.7e-27
    g = 1.3e-3
    P0 = abs(b2) / (g * T0 ** 2)
    LD = T0 ** 2 / abs(b2)
    assert abs(P0 - 0.0417) < 1e-3 and abs(LD - 18.43e3) < 20
    n = 1024
    window = 80 * T0
    fs = n / window
    t = (np.arange(n) - n // 2) / fs
    u0 = np.sqrt(P0) / np.cosh(t / T0)
    z = 5 * LD
    link = synth.Link(n_spans=1, span_km=z / 1e3, steps_per_span=400, symmetric=True, ase=False)
    y = nlse.channel(u0, _fiber(alpha=0.0), link, fs)
    ref = u0 * np.exp(1j * z / (2 * LD))
    assert np.max(np.abs(y - ref)) / np.sqrt(P0) < 2e-4
    # with the sign of beta2 flipped the pulse disperses: the pin sees the sign
    y_bad = nlse.channel(u0, _fiber(alpha=0.0, beta2=+21.7), link, fs)
    assert np.max(np.abs(y_bad - ref)) / np.sqrt(P0) > 0.3


def test_convergence_orders():
    fs = 40e9
    x = _x(n=256, B=1, pw=40e-3, seed=3)
    f = _fiber()
    def run(N, sym):
        return nlse.channel(x, f, synth.Link(1, 80.0, N, sym, False), fs)
    ref = run(2048, True)
    for sym, order in ((True, 2.0), (False, 1.0)):
        e8 = np.linalg.norm(run(8, sym) - ref)
        e32 = np.linalg.norm(run(32, sym) - ref)
        slope = np.log(e8 / e32) / np.log(4)
        assert abs(slope - order) < 0.3, (sym, slope)


def test_cd_memory_matches_paper():
    g = _read_golden("paper_numbers.txt")
    t1 = nlse.cd_memory_samples(-21.683, 1.1 * 10.7e9, 25 * 80, 2 * 10.7e9)
    t2 = nlse.cd_memory_samples(-21.683, 1.1 * 32e9, 10 * 100, 2 * 32e9)
    assert round(t1) == g["cd_memory_10p7GBd_2000km"]
    assert round(t2) == g["cd_memory_32GBd_1000km"]


def test_ase_noise_variance_and_whiteness():
    a = 0.2 * np.log(10) / 10 / 1e3
    fs = 20e9
    s2 = nlse.ase_sigma2(a, 80e3, 5.0, 1.946e14, fs)
    # n_sp = NF / (2 (1 - e^{-alpha L})) and PSD = (e^{alpha L} - 1) h nu n_sp
    nsp = 10 ** 0.5 / (2 * (1 - 10 ** -1.6))
    assert abs(s2 / fs - (10 ** 1.6 - 1) * 6.626e-34 * 1.946e14 * nsp) / (s2 / fs) < 1e-12
    w = nlse.ase_noise(8192, 4, span=0, sigma2=s2, seed=99, counter=0)
    assert abs(np.mean(np.abs(w) ** 2) / s2 - 1) < 0.03
    r1 = np.mean(w[:, 1:] * np.conj(w[:, :-1])) / s2
    assert abs(r1) < 0.03
    # the channel with ASE and gamma = beta2 = 0 adds exactly n_spans noise terms
    x = np.zeros((4, 8192), dtype=complex)
    link = synth.Link(3, 80.0, 2, True, True, 5.0, 1.946e14, 99, 0)
    y = nlse.channel(x, _fiber(beta2=0.0, gamma=0.0), link, fs)
    ref = sum(nlse.ase_noise(8192, 4, s, s2, 99, 0) for s in range(3))
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("symmetric", [True, False])
def test_dbp_explicit_steps_closed_forms(symmetric):
    # Non-uniform steps (70.4 / 29.6 km, the logarithmic sizes of Example 1):
    # beta2 = 0 must give the exact SPM inverse y exp(-j N gamma L_eff(L_sp) |y|^2)
    # for any step sizes (the loss integrals telescope); gamma = 0 the exact
    # all-pass dispersion inverse; uniform steps must equal dbp().
    class F:
        def __init__(self, a, b, g):
            self.alpha_db_per_km, self.beta2_ps2_per_km, self.gamma_per_w_km = a, b, g
    n, fs, N, L = 256, 20e9, 3, 100.0
    steps = [70.42, 29.58]
    y = synth.gaussian_waveform(2, n, 31, 5e-3)
    f0 = F(0.2, 0.0, 1.3)
    out = nlse.dbp_steps(y, f0, N, L, steps, fs, symmetric)
    a = nlse.si_alpha(0.2)
    ref = y * np.exp(-1j * N * nlse.si_gamma(1.3) * nlse.leff(a, L * 1e3) * np.abs(y) ** 2)
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(y))
    f1 = F(0.2, -21.7, 0.0)
    out = nlse.dbp_steps(y, f1, N, L, steps, fs, symmetric)
    w = nlse.omega_grid(n, fs)
    ref = np.fft.ifft(np.fft.fft(y, axis=-1) * np.exp(1j * (-nlse.si_beta2(-21.7) / 2) * w ** 2 * N * L * 1e3), axis=-1)
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(y))
    fib = synth.Fiber()
    link = synth.Link(N, L, 4, symmetric, False)
    assert np.allclose(nlse.dbp_steps(y, fib, N, L, [L / 4] * 4, fs, symmetric),
                       nlse.dbp(y, fib, link, fs, 4, symmetric), rtol=0, atol=1e-14)
