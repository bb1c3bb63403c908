"""Host-side logic of the package that needs no GPU: initialisation, schedules,
argument checks of the Python binding."""
import math

import numpy as np
import pytest
import torch

from oracle import train as otrain
from paper_2010_14258_gb300 import api, init, train


def test_ls_fir_out_of_band_gain_is_capped():
    # the in-band LS fit with the out-of-band penalty keeps |H(w)| <= cap |gain| outside the band
    wm = init.signal_band(2, 0.1) * 1.05
    for T, xi, gain in ((3, 0.35, 1.0), (9, 0.35, 1.0), (15, 2.2, 3.16), (31, 2.2, 0.22)):
        h = init.ls_symmetric_fir(T, xi, wm, gain=gain)
        w = np.linspace(-math.pi, math.pi, 4001)
        H = h[0] + sum(2 * h[k] * np.cos(k * w) for k in range(1, len(h)))
        oob = np.abs(w) > wm + 1e-9
        assert np.max(np.abs(H[oob])) <= abs(gain) * (1 + 1e-6)


def test_ls_fir_in_band_error_decreases_with_length():
    wm = init.signal_band(2, 0.1)
    w = np.linspace(-wm, wm, 2001)
    errs = []
    for T in (3, 5, 9, 15):
        h = init.ls_symmetric_fir(T, 0.35, wm)
        H = h[0] + sum(2 * h[k] * np.cos(k * w) for k in range(1, len(h)))
        errs.append(np.max(np.abs(H - np.exp(1j * 0.35 * w * w))))
    assert all(a > b for a, b in zip(errs, errs[1:]))


def test_pruning_schedule_matches_the_oracle_reading():
    for steps, iters in ((10, 1000), (175, 150000), (1, 5)):
        assert train.pruning_schedule(steps, iters, 0.6) == otrain.pruning_iterations(steps, iters, 0.6)
    assert otrain.pruning_steps([11] * 5, [7] * 5) == 10  # Example 2


def test_merge_half_steps_and_log_steps_sum_to_the_link():
    d = init.log_step_sizes(100.0, 4)
    assert abs(sum(d) - 100.0) < 1e-9 and d == sorted(d, reverse=True)  # DBP order: long steps first
    dp, g, c = init.symmetric_layers(3, 100.0, d)
    assert len(dp) == 13 and abs(sum(dp) - 300.0) < 1e-9
    assert all(ci < 0 for ci in c[:-1]) and c[-1] == 0.0


def test_unit_and_random_filter_initialisation():
    u = init.unit_filters([1, 3, 9])
    assert [len(h) for h in u] == [1, 2, 5] and all(h[0] == 1 and not np.any(h[1:]) for h in u)
    r = init.random_filters([5, 9], seed=3)
    for h in r:  # normalised by sum_{k=-K}^{K} |h_k|^2 as printed: the energy becomes its own inverse
        e = abs(h[0]) ** 2 + 2 * np.sum(np.abs(h[1:]) ** 2)
        assert 0 < e < 10


def test_binding_rejects_bad_tensors_before_any_launch():
    taps = torch.zeros(2, 3, dtype=torch.complex64)
    x = torch.zeros(1, 16, dtype=torch.complex64)
    with pytest.raises(ValueError):
        api.ldbp_essm_apply(taps, [3, 3], [0.0, 0.0], torch.zeros(2, 3), [1, 1], x)  # eta not on a GPU
    with pytest.raises(ValueError):
        api.ldbp_apply_host(taps, [3, 3], [0.0, 0.0], x.to(torch.complex128), x)  # not complex64


class _FakeBackend:
    """Stands in for the library: tags which equaliser ran and reports set SNRs."""

    def __init__(self, snr_ldbp, snr_dbp):
        self.snr = {"ldbp": snr_ldbp, "dbp": snr_dbp}
        self.calls = []

    def ldbp_apply(self, taps, T, c, y):
        self.calls.append("ldbp")
        return ("ldbp", y)

    def dbp_apply(self, fiber, link, fs, y, steps, symmetric):
        self.calls.append("dbp")
        return ("dbp", y)

    def rx(self, z, symbols, power_w, sps=2, rolloff=0.1):
        return z[0], None, None

    def snr_db(self, stats):
        return self.snr[stats]


def _receiver(snr_ldbp, snr_dbp, tol=0.1):
    from paper_2010_14258_gb300 import receiver
    be = _FakeBackend(snr_ldbp, snr_dbp)
    return receiver.Receiver(None, [3], [0.0], None, None, 20e9, tolerance_db=tol, backend=be), be


def test_receiver_falls_back_to_dbp_until_validated():
    r, be = _receiver(25.9, 25.7)
    assert not r.uses_ldbp
    assert r.backpropagate("y")[0] == "dbp"


@pytest.mark.parametrize("snr_ldbp, snr_dbp, use", [(25.9, 25.7, True), (25.6, 25.7, True),
                                                     (25.5, 25.7, False), (19.0, 25.7, False)])
def test_receiver_uses_ldbp_only_within_the_tolerance(snr_ldbp, snr_dbp, use):
    r, be = _receiver(snr_ldbp, snr_dbp)
    d = r.validate("y", "s", 1e-3)
    assert (d.snr_ldbp_db, d.snr_dbp_db) == (snr_ldbp, snr_dbp)
    assert be.calls == ["ldbp", "dbp"]
    assert r.uses_ldbp is use
    assert r.backpropagate("y")[0] == ("ldbp" if use else "dbp")


def test_receiver_revalidation_can_withdraw_the_model():
    r, be = _receiver(25.9, 25.7)
    r.validate("y", "s", 1e-3)
    assert r.uses_ldbp
    be.snr["ldbp"] = 20.0  # e.g. the link changed
    r.validate("y", "s", 1e-3)
    assert not r.uses_ldbp and r.backpropagate("y")[0] == "dbp"


def test_training_log_record():
    import json
    rec = train.iteration_record(7, 1e-2, 5e-4, [9, 7, 5])
    assert rec == {"step": 7, "loss": 1e-2, "snr_db": 20.0, "lr": 5e-4, "taps": 21, "T": [9, 7, 5]}
    assert json.loads(json.dumps(rec)) == rec


def test_receiver_chain_runs_rx_on_the_served_output():
    r, be = _receiver(25.9, 25.7)
    assert r("y", "s", 1e-3) == ("dbp", None)  # before validation: DBP
    r.validate("y", "s", 1e-3)
    assert r("y", "s", 1e-3) == ("ldbp", None)
