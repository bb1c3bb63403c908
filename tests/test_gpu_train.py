"""Optimiser parity and the end-to-end training test: LDBP trained on the GPU
with the library's own forward/adjoint kernels gains over its untrained
initialisation, over the same model without nonlinear steps and over
1-step-per-span frequency-domain DBP."""
import numpy as np
import pytest

from oracle import train as otrain
from tests.util import gpu_lib

pytestmark = pytest.mark.gpu


def test_adam_kernel_matches_oracle_and_masks_pruned_taps():
    import torch
    gpu_lib()
    from paper_2010_14258_gb300 import api
    rng = np.random.default_rng(0)
    M, stride = 3, 5
    T = [9, 5, 1]
    theta = (rng.standard_normal((M, stride)) + 1j * rng.standard_normal((M, stride))).astype(np.complex64)
    taps = torch.from_numpy(theta.copy()).cuda()
    m = torch.zeros((M, stride, 2), dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    th = theta.view(np.float32).astype(np.float64).reshape(M, stride, 2)
    mm = np.zeros_like(th)
    vv = np.zeros_like(th)
    for t in range(1, 6):
        g = (rng.standard_normal((M, stride)) + 1j * rng.standard_normal((M, stride))).astype(np.complex64)
        api.adam_step(taps, torch.from_numpy(g).cuda(), m, v, T, t, lr=1e-2)
        gr = g.view(np.float32).astype(np.float64).reshape(M, stride, 2)
        th, mm, vv = otrain.adam(th, gr, mm, vv, t, lr=1e-2)
        for i, Ti in enumerate(T):  # the mask of Sec. IV-C: pruned taps are zero
            th[i, (Ti - 1) // 2 + 1:] = 0
            mm[i, (Ti - 1) // 2 + 1:] = 0
            vv[i, (Ti - 1) // 2 + 1:] = 0
    torch.cuda.synchronize()
    out = taps.cpu().numpy().view(np.float32).reshape(M, stride, 2)
    assert np.max(np.abs(out - th)) < 1e-5
    assert np.all(taps.cpu().numpy()[0, 5:] == 0) and np.all(taps.cpu().numpy()[2, 1:] == 0)


def test_training_gains_over_untrained_and_linear_only_and_dbp():
    gpu_lib()
    from paper_2010_14258_gb300.train import Trainer, TrainConfig
    kw = dict(batch=16, nsym=4096, n_spans=10, channel_steps=20, powers_dbm=(4, 5, 6), t_start=9, t_end=7,
              iters=1200, lr=3e-4, seed=1, prune_frac=0.5)
    tr = Trainer(TrainConfig(**kw))
    e0 = tr.evaluate(frames=2, power_dbm=5.0)
    tr.fit()
    e1 = tr.evaluate(frames=2, power_dbm=5.0)
    assert tr.T == [7] * 10                      # every filter pruned 9 -> 7
    assert e1["ldbp"] > e0["ldbp"] + 3.0         # learning gains over the LS initialisation
    assert e1["ldbp"] > e1["dbp"] + 1.0          # and over 1-StPS FD DBP
    lin = Trainer(TrainConfig(**dict(kw, linear_only=True, iters=600)))
    lin.fit()
    e2 = lin.evaluate(frames=2, power_dbm=5.0)
    assert e1["ldbp"] > e2["ldbp"] + 10.0        # the nonlinear steps matter


def test_checkpoint_resume_is_bit_identical(tmp_path):
    import torch
    gpu_lib()
    from paper_2010_14258_gb300.train import Trainer, TrainConfig
    kw = dict(batch=4, nsym=2048, n_spans=4, channel_steps=5, powers_dbm=(3,), t_start=9, t_end=5, iters=40,
              lr=3e-4, seed=2)
    a = Trainer(TrainConfig(**kw))
    for it in range(20):
        a.train_step(it)
    a.save(tmp_path / "ck.npz")
    for it in range(20, 40):
        a.train_step(it)
    b = Trainer(TrainConfig(**kw))
    b.load(tmp_path / "ck.npz")
    for it in range(20, 40):
        b.train_step(it)
    torch.cuda.synchronize()
    assert a.T == b.T
    assert np.array_equal(a.taps.cpu().numpy(), b.taps.cpu().numpy())


def test_alternating_pruning_targets():
    # the alternating lengths of Sec. V-B (5 at even, 3 at odd step indices):
    # 2 + 3 + 2 + 3 pruning steps, every filter ends at its own target and the
    # masked taps are zero
    gpu_lib()
    from paper_2010_14258_gb300.train import Trainer, TrainConfig
    tr = Trainer(TrainConfig(batch=4, nsym=2048, n_spans=4, channel_steps=5, powers_dbm=(3,), t_start=9, t_end=5,
                             t_end_odd=3, iters=40, lr=3e-4, seed=4, prune_frac=0.5))
    assert len(tr.schedule) == 2 + 3 + 2 + 3
    tr.fit()
    assert tr.T == [5, 3, 5, 3]
    h = tr.taps.cpu().numpy()
    for i, T in enumerate(tr.T):
        assert np.all(h[i, (T + 1) // 2:] == 0)


def test_learnable_nonlinear_coefficients_train():
    # Remark 1: with learnable c the coefficients move and training still gains
    gpu_lib()
    from paper_2010_14258_gb300.train import Trainer, TrainConfig
    kw = dict(batch=16, nsym=4096, n_spans=10, channel_steps=20, powers_dbm=(4, 5, 6), t_start=9, t_end=9,
              iters=600, lr=3e-4, seed=4, learn_c=True)
    tr = Trainer(TrainConfig(**kw))
    c0 = list(tr.c)
    e0 = tr.evaluate(frames=2, power_dbm=5.0)
    tr.fit()
    e1 = tr.evaluate(frames=2, power_dbm=5.0)
    assert max(abs(a - b) / abs(b) for a, b in zip(tr.c, c0)) > 1e-3
    assert all(np.isfinite(tr.c))
    assert e1["ldbp"] > e0["ldbp"] + 3.0


def test_unit_filter_initialisation_trains():
    # Sec. V-E: unit filters (no knowledge of the link's dispersion) start with no
    # CD compensation and converge, more slowly than the LS initialisation
    gpu_lib()
    from paper_2010_14258_gb300.train import Trainer, TrainConfig
    kw = dict(batch=16, nsym=4096, n_spans=10, channel_steps=20, powers_dbm=(4, 5, 6), t_start=9, t_end=9,
              iters=1500, lr=1e-3, lr_final=1e-4, seed=5, init="unit")
    tr = Trainer(TrainConfig(**kw))
    e0 = tr.evaluate(frames=2, power_dbm=5.0)
    tr.fit()
    e1 = tr.evaluate(frames=2, power_dbm=5.0)
    assert e1["ldbp"] > e0["ldbp"] + 10.0
    rnd = Trainer(TrainConfig(**dict(kw, init="random", iters=50)))
    rnd.fit()
    assert np.all(np.isfinite(rnd.taps.cpu().numpy()))


def test_learned_essm_trains():
    # learned enhanced SSM (Sec. III-C): FIR taps and per-step |v|^2 filters
    # (unit-initialised) trained jointly by Adam through ldbp_essm_backward
    gpu_lib()
    from paper_2010_14258_gb300.train import Trainer, TrainConfig
    kw = dict(batch=16, nsym=4096, n_spans=10, channel_steps=20, powers_dbm=(4, 5, 6), t_start=9, t_end=9,
              iters=600, lr=3e-4, seed=6, kappa=8)
    tr = Trainer(TrainConfig(**kw))
    eta0 = tr.eta.clone()
    e0 = tr.evaluate(frames=2, power_dbm=5.0)
    tr.fit()
    e1 = tr.evaluate(frames=2, power_dbm=5.0)
    assert float((tr.eta - eta0).abs().max()) > 1e-3
    assert e1["ldbp"] > e0["ldbp"] + 3.0
