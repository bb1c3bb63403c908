"""Parity of the fused LDBP forward kernel (CUDA, FP32) with the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import ldbp as oldbp
from oracle import nlse, txrx
from tests.util import c64, gpu_lib, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def _model(Ts, seed, ls=True, fs=20e9, span_km=80.0):
    """Gain-capped LS taps of one span's dispersion (plus a 1 % perturbation),
    c = -gamma L_eff(span).  The gain cap keeps the 25-step cascade well
    conditioned, so FP32 and FP64 results stay comparable."""
    from paper_2010_14258_gb300 import init
    base, cs = init.ldbp_init(Ts, span_km=span_km, fs=fs)
    taps = []
    for i, (T, h) in enumerate(zip(Ts, base)):
        if not ls:
            h = np.eye(1, (T - 1) // 2 + 1)[0].astype(complex)
        h = h + synth.complex_normal(len(h), seed + i, 0.01 * abs(h[0]))
        taps.append(c64(h))
    return taps, [float(np.float32(ci)) for ci in cs]


def _signal(B, n, seed, pw):
    """Band-limited 16-QAM RRC waveform (2 samples/symbol) of mean power pw, n even;
    odd n uses white Gaussian samples instead."""
    if n % 2:
        return c64(synth.gaussian_waveform(B, n, seed, pw))
    s = synth.qam16_symbols(B, n // 2, seed)
    return c64(txrx.tx(s, 2, 0.1, pw))


def _pack(taps, stride=None):
    stride = stride or max(len(h) for h in taps)
    arr = np.zeros((len(taps), stride), np.complex128)
    for i, h in enumerate(taps):
        arr[i, : len(h)] = h
    return arr


def _run(taps, Ts, c, x, ckpt=False):
    import torch
    from paper_2010_14258_gb300 import api
    gpu_lib()
    td = to_dev(_pack(taps))
    xd = to_dev(x)
    ck = torch.empty((len(Ts),) + tuple(xd.shape), dtype=torch.complex64, device="cuda") if ckpt else None
    y = api.ldbp_apply(td, Ts, c, xd, ckpt=ck)
    torch.cuda.synchronize()
    return to_np(y), (to_np(ck) if ckpt else None)


CASES = [
    # (Ts, B, n, power_w)
    ([3] * 25, 3, 10000, 5e-3),          # several tiles + ragged tail
    ([5] * 25, 2, 12290, 5e-3),
    ([9] * 25, 2, 9001, 2e-3),           # odd n: unaligned rows, plain-load path
    ([15] * 25, 2, 16384, 2e-3),
    ([31, 15, 9, 3] * 2, 2, 8192, 2e-3),
    ([5, 3] * 12 + [5], 2, 8000, 4e-3),  # alternating lengths after pruning
    ([33] * 4, 1, 6000, 2e-3),           # longest supported filter
    ([1, 3, 1, 5], 2, 4096, 1e-2),       # T = 1 steps
]


def fp32_floor(x, taps, c, trials=2, seed=0):
    """Relative change of the FP64 forward output when x is perturbed at FP32
    rounding level: the error floor of any FP32 evaluation of this cascade.
    25 steps of 3-tap LS filters (in-band gain up to 1.1 per step) raise it
    above 1e-4; well-conditioned cascades stay near 1e-7."""
    rng = np.random.default_rng(seed)
    ref, _ = oldbp.forward(x, taps, c)
    worst = 0.0
    for _ in range(trials):
        xp = x * (1 + 6e-8 * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)))
        yp, _ = oldbp.forward(xp, taps, c)
        worst = max(worst, rel_l2(yp, ref))
    return ref, worst


def derived_tol(floor, M):
    """Tolerance of an FP32 evaluation of an M-step cascade against the FP64
    oracle: the stated 1e-4, or 2 sqrt(M) times the floor where that is larger.
    Each of the M steps rounds its output at about the size of the input
    perturbation that defines the floor (one FP32 ulp; at most twice that),
    the rest of the cascade amplifies a step's error no more than it amplifies
    the input, and the M independent roundings add in quadrature."""
    return max(1e-4, 2.0 * np.sqrt(M) * floor)


@pytest.mark.parametrize("Ts,B,n,pw", CASES)
def test_ldbp_forward_parity(Ts, B, n, pw):
    taps, c = _model(Ts, seed=len(Ts) * 7 + n)
    x = _signal(B, n, n, pw)
    y, _ = _run(taps, Ts, c, x)
    ref, floor = fp32_floor(x, taps, c)
    tol = derived_tol(floor, len(Ts))
    err = rel_l2(y, ref)
    print(f"T={Ts[:3]}... M={len(Ts)}: floor {floor:.1e}, tolerance {tol:.1e}, error {err:.1e}")
    assert err <= tol


@pytest.mark.parametrize("n", [1, 2, 7, 64, 511, 4096, 4097])
def test_ldbp_forward_short_waveforms_wrap(n):
    # waveforms shorter than a tile wrap around several times (circular index)
    Ts = [5, 9, 3]
    taps, c = _model(Ts, seed=n)
    x = c64(synth.gaussian_waveform(3, n, 100 + n, 5e-3))
    y, _ = _run(taps, Ts, c, x)
    ref, _ = oldbp.forward(x, taps, c)
    assert rel_l2(y, ref) <= 1e-5 * len(Ts)


def test_ldbp_single_step_error_and_checkpoints():
    Ts = [9] * 25
    taps, c = _model(Ts, seed=3)
    x = _signal(2, 20000, 5, 5e-3)
    y, ck = _run(taps, Ts, c, x, ckpt=True)
    ref, inputs = oldbp.forward(x, taps, c)
    assert rel_l2(y, ref) <= 1e-4
    for i in range(len(Ts)):
        # checkpoint i is the input of step i
        assert rel_l2(ck[i], inputs[i]) <= 1e-4
        # one step applied to the oracle's own input: error <= 1e-5 per step
        yi, _ = _run([taps[i]], [Ts[i]], [c[i]], c64(inputs[i]))
        ri, _ = oldbp.forward(c64(inputs[i]), [taps[i]], [c[i]])
        assert rel_l2(yi, ri) <= 1e-5


def test_linear_only_layers_and_large_phase():
    # c = 0 layers are pure FIR; a large Kerr phase (up to ~1 rad) stays accurate
    Ts = [7, 7, 7]
    taps, _ = _model(Ts, seed=9, ls=False)
    x = c64(synth.gaussian_waveform(2, 5000, 9, 1.0))
    for c in ([0.0, 0.0, 0.0], [-0.3, 0.25, 0.0]):
        y, _ = _run(taps, Ts, c, x)
        ref, _ = oldbp.forward(x, taps, c)
        assert rel_l2(y, ref) <= 1e-5 * 10


@pytest.mark.parametrize("T", [3, 9, 15])
def test_full_size_sampled(T):
    # the benchmark's launch: 256 x 65536 at M = 25 (fixed-width instances);
    # compare sampled waveforms over their full length
    import torch
    from paper_2010_14258_gb300 import api
    gpu_lib()
    Ts = [T] * 25
    taps, c = _model(Ts, seed=2)
    B, n = 256, 65536
    g = torch.Generator(device="cuda").manual_seed(0)
    xd = (torch.randn(B, n, generator=g, device="cuda", dtype=torch.complex64) * (2e-3 ** 0.5))
    y = api.ldbp_apply(to_dev(_pack(taps)), Ts, c, xd)
    torch.cuda.synchronize()
    for b in (0, 77, 255):
        xb = to_np(xd[b])
        ref, floor = fp32_floor(xb, taps, c)
        assert rel_l2(to_np(y[b]), ref) <= derived_tol(floor, len(Ts))


@pytest.mark.parametrize("phi_max", [0.25, 0.49, 0.75, 0.99, 3.0, 40.0])
def test_kerr_step_tiers_elementwise(phi_max):
    # One Kerr-only step (T = 1, h_0 = 1: the filter is exact) with phases
    # spread over [0, phi_max]: each warp's largest phase selects the series
    # of degree 5/6 (|phase| <= 0.5), 7/8 (<= 1) or the range-reducing path.  Every sample must
    # match the FP64 rotation to a few FP32 ulps, plus the FP32 rounding of
    # the phase itself (about 2^-23 of phi).
    n = 8192
    rng = np.random.default_rng(int(phi_max * 100))
    p = rng.uniform(0.0, 1.0, (2, n))
    x = c64(np.sqrt(p) * np.exp(2j * np.pi * rng.uniform(size=(2, n))))
    c = [float(np.float32(phi_max))]
    taps = [np.array([1.0 + 0j])]
    y, _ = _run(taps, [1], c, x)
    ref, _ = oldbp.forward(x, taps, c)
    err = np.abs(y - ref) / np.maximum(np.abs(ref), 1e-30)
    assert err.max() <= 4e-7 + 2e-7 * phi_max


@pytest.mark.parametrize("chunks,pinned", [(1, True), (3, True), (5, False)])
def test_apply_host_matches_device_call(chunks, pinned):
    # the host-buffer call runs the same kernel per chunk of waveforms:
    # bitwise equal to ldbp_apply on device copies, and to the oracle
    import torch
    from paper_2010_14258_gb300 import api
    gpu_lib()
    Ts = [9, 5, 3]
    taps, c = _model(Ts, seed=11)
    x = _signal(5, 6000, 12, 4e-3)
    td = to_dev(_pack(taps))
    xh = torch.from_numpy(x.astype(np.complex64)).contiguous()
    yh = torch.zeros_like(xh)
    if pinned:
        xh, yh = xh.pin_memory(), yh.pin_memory()
    api.ldbp_apply_host(td, Ts, c, xh, yh, chunks=chunks)
    torch.cuda.synchronize()
    yd = api.ldbp_apply(td, Ts, c, to_dev(x))
    assert np.array_equal(yh.numpy(), to_np(yd))
    ref, _ = oldbp.forward(x, taps, c)
    assert rel_l2(yh.numpy(), ref) <= 1e-4


def test_remark4_rescaled_model_same_output():
    # Remark 4 on the CUDA path: filters rescaled by s_i / s_{i-1} and Kerr
    # coefficients by 1 / |s_i|^2 give the same outputs (to FP32 rounding)
    Ts = [9] * 12 + [5] * 12 + [3]
    taps, c = _model(Ts, seed=44)
    c[-1] = 0.0
    rng = np.random.default_rng(44)
    s = [rng.uniform(0.5, 2.0) * np.exp(2j * np.pi * rng.uniform()) for _ in range(len(Ts) - 1)]
    t2, c2, prev = [], [], 1.0
    for i, (h, ci) in enumerate(zip(taps, c)):
        si = s[i] if i < len(s) else 1.0
        t2.append(c64(np.asarray(h) * si / prev))
        c2.append(float(np.float32(ci / abs(si) ** 2)))
        prev = si
    x = _signal(2, 16384, 45, 3e-3)
    y1, _ = _run(taps, Ts, c, x)
    y2, _ = _run(t2, Ts, c2, x)
    ref, floor = fp32_floor(x, taps, c)
    assert rel_l2(y1, ref) <= derived_tol(floor, len(Ts))
    assert rel_l2(y2, y1) <= 2 * derived_tol(floor, len(Ts))


@pytest.mark.parametrize("stps,T", [(2, 15), (4, 9)])
def test_symmetric_log_step_ldbp_parity(stps, T):
    # symmetric-SSM-based LDBP with logarithmic steps (Sec. IV-C) at 32 GBd,
    # 2 samples per symbol, 10 x 100 km: l = 10 * StPS + 1 layers, the last
    # one linear-only, layer gains != 1
    from paper_2010_14258_gb300 import init
    taps, c = init.ldbp_init_symmetric(T, 10, 100.0, 64e9, steps_per_span=stps)
    taps = [c64(h) for h in taps]
    c = [float(np.float32(v)) for v in c]
    Ts = [T] * len(taps)
    assert len(Ts) == 10 * stps + 1 and c[-1] == 0.0
    x = _signal(2, 16384, 50 + stps, 1e-3 * 10 ** 0.4)
    y, _ = _run(taps, Ts, c, x)
    ref, floor = fp32_floor(x, taps, c)
    assert rel_l2(y, ref) <= max(1e-4, 10 * floor)


def test_ldbp_effective_snr_matches_oracle():
    # Effective SNR (Eq. (14)) after LDBP, CUDA path vs FP64 oracle on the same
    # received waveform: 4096 16-QAM symbols at 2 dBm over 25 x 80 km (oracle
    # channel, 4 symmetric steps/span, no ASE), then 1-StPS LDBP with T = 9.
    fs, pw = 20e9, 10 ** (2.0 / 10) * 1e-3
    s = synth.qam16_symbols(1, 4096, 23)
    x = txrx.tx(s, 2, 0.1, pw)
    r = c64(nlse.channel(x, synth.Fiber(), synth.Link(25, 80.0, 4, True, False), fs))
    Ts = [9] * 25
    taps, c = _model(Ts, seed=23)
    y, _ = _run(taps, Ts, c, r)
    ref, floor = fp32_floor(r, taps, c)
    assert rel_l2(y, ref) <= max(1e-4, 10 * floor)
    snr_gpu = txrx.evaluate(y, s, 2, 0.1, pw)["snr_db"]
    snr_ref = txrx.evaluate(ref, s, 2, 0.1, pw)["snr_db"]
    assert abs(snr_gpu - snr_ref) <= 0.01
