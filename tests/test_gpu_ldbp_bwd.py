"""Parity of the hand-written LDBP adjoint (CUDA, FP32) with the FP64 oracle and
FP64 finite differences."""
import numpy as np
import pytest

import synth
from oracle import ldbp as oldbp
from oracle import txrx
from tests.test_gpu_ldbp_fwd import _model, _pack, _signal
from tests.util import c64, gpu_lib, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def _gpu_grads(taps, Ts, c, x, gy):
    import torch
    gpu_lib()
    from paper_2010_14258_gb300 import api
    td = to_dev(_pack(taps))
    xd = to_dev(x)
    M = len(Ts)
    ck = torch.empty((M,) + tuple(xd.shape), dtype=torch.complex64, device="cuda")
    api.ldbp_apply(td, Ts, c, xd, ckpt=ck)
    gx, gt = api.ldbp_backward(td, Ts, c, ck, to_dev(gy))
    torch.cuda.synchronize()
    return to_np(gx), to_np(gt)


def _grad_signal(B, n, seed):
    """A loss gradient shaped like the receiver's (matched-filter band), unit power."""
    if n % 2:
        return c64(synth.complex_normal((B, n), seed, 1.0))
    return c64(txrx.tx(synth.qam16_symbols(B, n // 2, seed), 2, 0.1, 1.0))


def fp32_sensitivity(x, taps, c, gy, trials=2, seed=0):
    """Relative change of the FP64 adjoint when x and gy are perturbed at FP32
    rounding level (2^-24 relative): the error floor of any FP32 evaluation.
    Short filters with in-band gain above one make the 25-step cascade
    ill-conditioned; the parity tolerance scales with this floor."""
    rng = np.random.default_rng(seed)
    rgx, rgt = oldbp.backward(x, taps, c, gy)
    sx, st = 0.0, 0.0
    for _ in range(trials):
        def pert(a):
            return a * (1 + 6e-8 * (rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)))
        px, pt = oldbp.backward(pert(x), taps, c, pert(gy))
        sx = max(sx, rel_l2(px, rgx))
        st = max(st, max(rel_l2(a, b) for a, b in zip(pt, rgt)))
    return rgx, rgt, sx, st


def _check(Ts, B, n, pw, seed, tol=1e-4):
    # tolerance max(tol, 2 sqrt(2M) s): the adjoint rounds at 2M sites (the
    # recomputed forward step and the reverse step, each at about the size of
    # the perturbation behind s), no site's error is amplified more than the
    # input's, and the roundings add in quadrature
    taps, c = _model(Ts, seed=seed)
    x = _signal(B, n, seed, pw)
    gy = _grad_signal(B, n, seed + 1)
    gx, gt = _gpu_grads(taps, Ts, c, x, gy)
    rgx, rgt, sx, st = fp32_sensitivity(x, taps, c, gy)
    k = 2.0 * np.sqrt(2 * len(Ts))
    assert rel_l2(gx, rgx) <= max(tol, k * sx)
    for i, h in enumerate(rgt):
        assert rel_l2(gt[i, : len(h)], h) <= max(tol, k * st), i
        assert np.all(gt[i, len(h):] == 0)


@pytest.mark.parametrize("Ts,B,n", [
    ([3] * 25, 2, 10000),
    ([5] * 25, 2, 10000),
    ([7] * 25, 3, 16384),
    ([5, 3] * 12 + [5], 2, 9000),
    ([9, 7] * 12 + [9], 2, 10000),
    ([9, 1, 7, 5, 3] * 5, 2, 8192),
    ([15, 13, 9, 1] * 6 + [15], 2, 8192),
    ([21] * 10, 1, 9000),
    ([33] * 3, 1, 7000),
    ([9] * 25, 1, 16384),
    ([15] * 25, 1, 12000),
    ([31] * 25, 1, 12000),
    ([31, 15, 9, 3], 3, 8192),
    ([33, 1, 3], 2, 5000),
    ([1, 1], 2, 4096),
])
def test_backward_parity(Ts, B, n):
    _check(Ts, B, n, 3e-3, seed=len(Ts) + n)


@pytest.mark.parametrize("n", [1, 7, 64, 1023, 4097])
def test_backward_short_and_odd(n):
    _check([5, 9, 3], 2, n, 5e-3, seed=n)


@pytest.mark.parametrize("n", [1, 7, 64, 1023, 4097, 8193])
def test_backward_uniform_width_short_and_odd(n):
    # models with one width in every step run the fixed-width adjoint
    _check([7] * 4, 2, n, 5e-3, seed=n + 1)


def test_backward_vs_fp64_finite_differences_1024_m4():
    # the gradient-check instance of the training workload: 1024 samples, M = 4
    Ts = [31, 15, 9, 3]
    taps, c = _model(Ts, seed=21)
    x = _signal(1, 1024, 21, 5e-3)
    r = _grad_signal(1, 1024, 22)
    gx, gt = _gpu_grads(taps, Ts, c, x, r)

    def loss(tt):
        y, _ = oldbp.forward(x, tt, c)
        return np.real(np.vdot(r, y))

    eps = 1e-6
    worst = 0.0
    for i in range(len(Ts)):
        fd = np.zeros(len(taps[i]), complex)
        for k in range(len(taps[i])):
            for unit in (1.0, 1j):
                tp = [t.copy() for t in taps]
                tm = [t.copy() for t in taps]
                tp[i][k] += eps * unit
                tm[i][k] -= eps * unit
                d = (loss(tp) - loss(tm)) / (2 * eps)
                fd[k] += d * (1 if unit == 1.0 else 1j)
        worst = max(worst, rel_l2(gt[i, : len(taps[i])], fd))
    assert worst <= 1e-4


def test_backward_is_deterministic():
    Ts = [9] * 10
    taps, c = _model(Ts, seed=5)
    x = _signal(4, 20000, 5, 3e-3)
    gy = _grad_signal(4, 20000, 6)
    a = _gpu_grads(taps, Ts, c, x, gy)
    b = _gpu_grads(taps, Ts, c, x, gy)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_autograd_function():
    import torch
    gpu_lib()
    from paper_2010_14258_gb300 import api
    Ts = [5, 3, 5]
    taps, c = _model(Ts, seed=8)
    x = _signal(2, 4096, 8, 3e-3)
    r = _grad_signal(2, 4096, 9)
    td = to_dev(_pack(taps)).requires_grad_(True)
    xd = to_dev(x).requires_grad_(True)
    y = api.LDBPFunction.apply(xd, td, Ts, c)
    loss = (torch.conj(to_dev(r)) * y).real.sum()
    loss.backward()
    rgx, rgt = oldbp.backward(x, taps, c, r)
    assert rel_l2(to_np(xd.grad), rgx) <= 1e-4
    for i, h in enumerate(rgt):
        assert rel_l2(to_np(td.grad)[i, : len(h)], h) <= 1e-4


def test_training_shape_sampled():
    # 32768-sample waveforms, M = 25, T = 31 (the start of the pruning schedule)
    _check([31] * 25, 3, 32768, 2e-3, seed=77)


def test_training_shape_pruned_sampled():
    # the same shape at the end of the pruning schedule (T = 7 in every step)
    _check([7] * 25, 3, 32768, 2e-3, seed=78)


def test_training_shape_alternating_sampled():
    # the same shape with the alternating 5/3 targets of Sec. V-B (mixed widths)
    _check([5, 3] * 12 + [5], 3, 32768, 2e-3, seed=79)


@pytest.mark.parametrize("Ts,B,n", [([9] * 25, 2, 12000), ([7] * 25, 2, 12001), ([5, 3] * 6 + [1], 2, 9001)])
def test_backward_c_gradients_match_oracle(Ts, B, n):
    # Remark 1: gradients of the nonlinear coefficients (learnable scaling);
    # one linear-only layer (c = 0) still has a c-gradient
    import torch
    gpu_lib()
    from paper_2010_14258_gb300 import api
    taps, c = _model(Ts, seed=n)
    c[-1] = 0.0
    x = _signal(B, n, n + 2, 3e-3)
    gy = _grad_signal(B, n, n + 3)
    td, xd = to_dev(_pack(taps)), to_dev(x)
    ck = torch.empty((len(Ts),) + tuple(xd.shape), dtype=torch.complex64, device="cuda")
    api.ldbp_apply(td, Ts, c, xd, ckpt=ck)
    gx, gt, gc = api.ldbp_backward(td, Ts, c, ck, to_dev(gy), want_gc=True)
    _, gt0 = api.ldbp_backward(td, Ts, c, ck, to_dev(gy))
    torch.cuda.synchronize()
    ref = np.array(oldbp.grad_c(x, taps, c, gy))
    got = gc.cpu().numpy().astype(np.float64)
    assert rel_l2(got, ref) <= 1e-4
    assert np.array_equal(to_np(gt), to_np(gt0))  # the tap gradients do not change
