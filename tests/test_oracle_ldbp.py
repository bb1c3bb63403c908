"""Pins of the FP64 LDBP oracle: brute force, adjoint identities, finite differences,
the T = n special case and the paper's tap / pruning arithmetic."""
import numpy as np
import pytest

import synth
from oracle import ldbp, nlse, train, txrx
from tests.conftest import golden_path


def _golden():
    rows = {}
    for line in open(golden_path("paper_numbers.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p = line.split()
        rows[p[0]] = float(p[1])
    return rows


def _taps(Ts, seed):
    out = []
    for i, T in enumerate(Ts):
        K = (T - 1) // 2
        h = synth.complex_normal(K + 1, seed + i, 0.3)
        h[0] += 1.0
        out.append(h)
    return out


def test_fir_equals_dense_circulant():
    n = 11
    for T in (1, 3, 5, 9):
        h = _taps([T], 7)[0]
        x = synth.complex_normal(n, 3)
        A = ldbp.circulant_matrix(h, n)
        assert np.allclose(A @ x, ldbp.fir(x, h), atol=1e-13)
        # rows are circular shifts of (h_K..h_1 h_0 h_1..h_K 0..0) (Sec. III-B)
        K = (T - 1) // 2
        row0 = np.zeros(n, complex)
        for k in range(-K, K + 1):
            row0[(-k) % n] += h[abs(k)]
        assert np.allclose(A[0], row0)
        assert np.allclose(A[3], np.roll(row0, 3))


def test_fir_adjoint_identity():
    n = 64
    h = _taps([9], 1)[0]
    x = synth.complex_normal(n, 2)
    y = synth.complex_normal(n, 3)
    lhs = np.vdot(y, ldbp.fir(x, h))          # <A x, y>
    rhs = np.vdot(ldbp.fir(y, np.conj(h)), x)  # <x, A^H y>
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _fd_check(n, Ts, c, seed, rtol):
    taps = _taps(Ts, seed)
    x = synth.complex_normal((2, n), seed + 100, 1.0)
    r = synth.complex_normal((2, n), seed + 200, 1.0)

    def loss(xx, tt):
        y, _ = ldbp.forward(xx, tt, c)
        return np.real(np.vdot(r, y))  # Re sum conj(r) y  => gy = r

    gx, gtaps = ldbp.backward(x, taps, c, r)
    eps = 1e-6
    rng = np.random.default_rng(seed)
    for _ in range(3):
        d = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
        fd = (loss(x + eps * d, taps) - loss(x - eps * d, taps)) / (2 * eps)
        an = np.real(np.vdot(gx, d))
        assert abs(fd - an) <= rtol * max(1.0, abs(an)), (fd, an)
    for i in range(len(taps)):
        for k in range(len(taps[i])):
            for unit in (1.0, 1j):
                tp = [t.copy() for t in taps]
                tm = [t.copy() for t in taps]
                tp[i][k] += eps * unit
                tm[i][k] -= eps * unit
                fd = (loss(x, tp) - loss(x, tm)) / (2 * eps)
                an = np.real(np.conj(gtaps[i][k]) * unit)
                assert abs(fd - an) <= rtol * max(1.0, abs(an)), (i, k, fd, an)


def test_gradients_finite_differences_small():
    _fd_check(64, [5, 3, 7], [-0.3, -0.5, 0.0], seed=11, rtol=1e-6)


@pytest.mark.slow
def test_gradients_finite_differences_1024_m4():
    # the training-size instance: 1024 samples, M = 4
    _fd_check(1024, [31, 15, 9, 3], [-0.05, -0.05, -0.05, -0.05], seed=5, rtol=1e-6)


def test_ldbp_full_length_equals_fd_dbp():
    # With T = n (n odd) the symmetric taps iDFT(exp(j xi w^2)) make the circular
    # FIR identical to the FD linear step, so LDBP is 1-StPS asymmetric DBP.
    n = 257
    fs = 20e9
    fib = synth.Fiber()
    link = synth.Link(3, 80.0, 1, False, False)
    x = synth.gaussian_waveform(2, n, 4, 2e-3)
    y = nlse.channel(x, fib, link, fs, steps=20)
    ref = nlse.dbp(y, fib, link, fs, steps_per_span=1, symmetric=False)
    b2 = nlse.si_beta2(fib.beta2_ps2_per_km)
    a = nlse.si_alpha(fib.alpha_db_per_km)
    L = 80e3
    xi = -b2 * L * fs ** 2 / 2
    h = ldbp.dbp_taps_full(n, xi)
    c = -nlse.si_gamma(fib.gamma_per_w_km) * nlse.leff(a, L)
    out, _ = ldbp.forward(y, [h] * 3, [c] * 3)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-12


def test_ls_taps_special_cases():
    # T = 1: best constant fit of exp(j xi w^2) is its mean over the grid
    xi = 0.35
    h = ldbp.ls_taps(1, xi, N=64)
    w = 2 * np.pi * np.arange(-32, 33) / 64
    assert abs(h[0] - np.mean(np.exp(1j * xi * w ** 2))) < 1e-12
    # xi = 0: the fit is the unit impulse for any length
    h = ldbp.ls_taps(9, 0.0)
    assert abs(h[0] - 1) < 1e-12 and np.max(np.abs(h[1:])) < 1e-12
    # longer filters fit better
    errs = []
    for T in (3, 9, 31):
        h = ldbp.ls_taps(T, xi)
        ww = np.linspace(-np.pi, np.pi, 1001)
        resp = h[0] + sum(2 * h[k] * np.cos(k * ww) for k in range(1, len(h)))
        errs.append(np.mean(np.abs(resp - np.exp(1j * xi * ww ** 2)) ** 2))
    assert errs[0] > errs[1] > errs[2]


def test_paper_tap_and_pruning_arithmetic():
    g = _golden()
    Ts = [5] * 13 + [3] * 12
    assert sum(T - 1 for T in Ts) + 1 == g["total_impulse_length_13x5_12x3"]
    assert train.pruning_steps([11] * 5, [7] * 5) == g["pruning_steps_example2"]
    # real multiplications: 7 per nonlinear step, 4 per folded tap pair (Sec. V-B)
    assert 25 * 7 == g["nonlinear_rm_per_sample_25_steps"]
    # h0-normalised folded filters: one complex multiply per tap pair plus one
    # overall gain (38 pairs + 1 = 39 complex multiplies of 4 RMs)
    assert (sum((T - 1) // 2 for T in Ts) + 1) * 4 == g["linear_rm_per_sample_13x5_12x3"]
    it = train.pruning_iterations(10, 100)
    assert len(it) == 10 and it == sorted(it) and it[-1] <= 60
    gaps = np.diff([0] + it)
    assert gaps[0] + gaps[1] < gaps[-1] + gaps[-2]   # front-loaded


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    p = rng.standard_normal(12)
    m = np.zeros(12)
    v = np.zeros(12)
    tp = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3)
    for t in range(1, 6):
        g = rng.standard_normal(12)
        p, m, v = train.adam(p, g, m, v, t)
        tp.grad = torch.tensor(g)
        opt.step()
    assert np.allclose(p, tp.detach().numpy(), atol=1e-12)


def test_tx_rx_back_to_back_and_power():
    s = synth.qam16_symbols(3, 1024, 9)
    P = np.array([1e-3, 2e-3, 0.5e-3])
    x = txrx.tx(s, 2, 0.1, P)
    pw = np.mean(np.abs(x) ** 2, axis=-1)
    assert np.all(np.abs(pw / P - 1) < 0.05)
    ev = txrx.evaluate(x * np.exp(0.7j), s, 2, 0.1, P)
    assert np.max(np.abs(ev["s_hat"] - s)) < 1e-12
    assert np.allclose(ev["phi"], 0.7)


def test_awgn_snr_estimator():
    s = synth.qam16_symbols(4, 4096, 10)
    P = 1e-3
    x = txrx.tx(s, 2, 0.1, P)
    sigma2 = 1e-5
    w = synth.gaussian_waveform(4, x.shape[-1], 11, sigma2)
    ev = txrx.evaluate(x + w, s, 2, 0.1, P)
    expect = 10 * np.log10(P * 2 / sigma2)
    assert abs(ev["snr_db"] - expect) < 0.15


def test_loss_gradient_finite_differences():
    s = synth.qam16_symbols(2, 64, 12)
    P = np.array([1e-3, 3e-3])
    y = txrx.tx(s, 2, 0.1, P) + synth.gaussian_waveform(2, 128, 13, 1e-5)
    gy, ev = txrx.loss_grad(y, s, 2, 0.1, P)
    rng = np.random.default_rng(1)
    eps = 1e-9
    for _ in range(4):
        d = rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape)
        fd = (txrx.evaluate(y + eps * d, s, 2, 0.1, P)["loss"]
              - txrx.evaluate(y - eps * d, s, 2, 0.1, P)["loss"]) / (2 * eps)
        an = np.real(np.vdot(gy, d))
        assert abs(fd - an) < 1e-5 * abs(an) + 1e-9


def _rescaled(taps, c, s):
    """Remark 4: scaling the signal before every nonlinear step by s_i and
    undoing it in the next filter, with c_i / |s_i|^2 in the Kerr step, leaves
    the model unchanged.  taps/c of M steps, s of M - 1 complex scales."""
    out_t, out_c, prev = [], [], 1.0
    for i, (h, ci) in enumerate(zip(taps, c)):
        si = s[i] if i < len(s) else 1.0
        out_t.append(np.asarray(h) * si / prev)
        out_c.append(ci / abs(si) ** 2)
        prev = si
    return out_t, out_c


def test_overparameterisation_invariance_remark4():
    # Remark 4: rescaled filters and nonlinear coefficients give the same model;
    # in particular every coefficient can be normalised to +-1 (last step linear).
    rng = np.random.default_rng(4)
    M, n = 5, 257
    taps = [synth.complex_normal(3 + i % 3, 40 + i, 0.5) for i in range(M)]
    c = [float(v) for v in rng.uniform(-2.0, 2.0, M - 1)] + [0.0]
    x = synth.complex_normal(n, 7, 0.7).reshape(1, n)
    ref, _ = ldbp.forward(x, taps, c)
    s = [complex(a, b) for a, b in rng.normal(size=(M - 1, 2))]
    t2, c2 = _rescaled(taps, c, s)
    y2, _ = ldbp.forward(x, t2, c2)
    assert np.allclose(y2, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    s_unit = [np.sqrt(abs(ci)) for ci in c[:-1]]
    t3, c3 = _rescaled(taps, c, s_unit)
    assert np.allclose(np.abs(c3[:-1]), 1.0) and c3[-1] == 0.0
    y3, _ = ldbp.forward(x, t3, c3)
    assert np.allclose(y3, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # a plausible mistake (rescaling c by |s| instead of |s|^2) breaks it
    bad = [ci / abs(si) for ci, si in zip(c[:-1], s)] + [0.0]
    yb, _ = ldbp.forward(x, t2, bad)
    assert not np.allclose(yb, ref, rtol=0, atol=1e-6 * np.abs(ref).max())


def test_log_step_sizes_and_layers_example1():
    # Example 1: L_sp = 100 km, 2 spans, symmetric SSM with 2 StPS: logarithmic
    # steps of about 70 and 30 km, merged layer lengths 35, 50, 50, 50, 15 km
    from paper_2010_14258_gb300 import init
    d = init.log_step_sizes(100.0, 2)
    assert abs(d[0] - 70) < 0.5 and abs(d[1] - 30) < 0.5 and abs(sum(d) - 100.0) < 1e-9
    dp, g, c = init.symmetric_layers(2, 100.0, d)
    assert len(dp) == 5 and np.allclose(dp, [35, 50, 50, 50, 15], atol=0.5)
    assert np.isclose(dp[1], dp[2]) and np.isclose(dp[2], dp[3]) and c[-1] == 0.0
    # the gains of a span (and its amplifier) multiply to one
    assert np.isclose(np.prod(g), 1.0)
    # uniform steps: plain halving and merging
    assert init.log_step_sizes(80.0, 4, zeta=0.0) == [20.0] * 4


@pytest.mark.parametrize("log_steps", [True, False])
def test_symmetric_ldbp_layers_equal_symmetric_dbp(log_steps):
    # With exact full-length filters (T = n odd), the symmetric-SSM-based LDBP
    # built from symmetric_layers (l = M + 1 layers: merged half-steps, gains,
    # c = -gamma l_mid, last layer linear) is symmetric DBP with the same steps.
    from paper_2010_14258_gb300 import init
    n, fs, N, L, K = 255, 64e9, 3, 100.0, 2
    fib = synth.Fiber()
    steps = init.log_step_sizes(L, K) if log_steps else [L / K] * K
    y = synth.gaussian_waveform(2, n, 17, 4e-3)
    ref = nlse.dbp_steps(y, fib, N, L, steps, fs, True)
    dp, g, c = init.symmetric_layers(N, L, steps)
    b2 = nlse.si_beta2(fib.beta2_ps2_per_km)
    taps = [gi * ldbp.dbp_taps_full(n, -b2 * d * 1e3 * fs ** 2 / 2) for d, gi in zip(dp, g)]
    out, _ = ldbp.forward(y, taps, c)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-11


def test_grad_c_finite_differences():
    # Remark 1 (learnable scaling of the nonlinear steps): dl/dc_i by central
    # finite differences of the FP64 forward, for l = sum |y - t|^2 (g = 2 (y - t))
    rng = np.random.default_rng(12)
    n, M = 64, 4
    taps = [synth.complex_normal(3 + 2 * (i % 2), 60 + i, 0.5) for i in range(M)]
    c = [float(v) for v in rng.uniform(-1.5, 1.5, M)]
    x = synth.complex_normal(2 * n, 61, 0.8).reshape(2, n)
    t = synth.complex_normal(2 * n, 62, 0.8).reshape(2, n)

    def loss(cc):
        y, _ = ldbp.forward(x, taps, cc)
        return float(np.sum(np.abs(y - t) ** 2))

    y, _ = ldbp.forward(x, taps, c)
    gc = ldbp.grad_c(x, taps, c, 2.0 * (y - t))
    for i in range(M):
        e = 1e-6
        cp, cm = list(c), list(c)
        cp[i] += e
        cm[i] -= e
        fd = (loss(cp) - loss(cm)) / (2 * e)
        assert abs(gc[i] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, gc[i], fd)
