"""Pins of two oracle functions against what the paper and the mathematics fix.

* oracle.train.choose_filter (Sec. IV-C, Example 2): a pruning step always
  removes the OUTERMOST tap pair of one filter; the filter is the one whose
  outermost tap is smallest among the filters still above their target
  (reading of "pruned by magnitude"); ties go to the lowest step index.
  Hand-built cases, each one failing a plausible mistake.
* oracle.txrx.raised_cosine (Eq. (11), Sec. IV-A: RRC roll-off 0.1): the RC
  spectrum is 1 on |nu| <= (1-b)/2, 0 on |nu| >= (1+b)/2, 1/2 at the Nyquist
  frequency, and vestigially symmetric about it; its inverse Fourier
  transform is the textbook time-domain RC pulse
  sinc(t) cos(pi b t) / (1 - (2 b t)^2).  A smaller or larger roll-off moves
  the support edges and fails.
The product's pruning rule (train.prune_choice) is checked against the
oracle's on random states.
"""
import numpy as np
import pytest

from oracle import train as otrain
from oracle import txrx


def _filters(outer, T):
    """Half-tap vectors of lengths T with a large centre tap and the given outermost taps."""
    out = []
    for h_out, t in zip(outer, T):
        K = (t - 1) // 2
        h = np.zeros(17, np.complex128)
        h[0] = 1.0
        h[1:K] = 0.9  # inner taps larger than any outermost tap below
        h[K] = h_out
        out.append(h)
    return out


def test_choose_filter_smallest_outermost_tap():
    taps = _filters([0.3, 0.1, 0.2], [7, 7, 7])
    assert otrain.choose_filter(taps, [7, 7, 7], [3, 3, 3]) == 1


def test_choose_filter_skips_filters_at_target():
    taps = _filters([0.3, 0.1, 0.2], [7, 5, 7])
    assert otrain.choose_filter(taps, [7, 5, 7], [3, 5, 3]) == 2
    assert otrain.choose_filter(taps, [3, 5, 3], [3, 5, 3]) == -1


def test_choose_filter_ties_go_to_lowest_index():
    taps = _filters([0.2, 0.2, 0.2], [9, 9, 9])
    assert otrain.choose_filter(taps, [9, 9, 9], [3, 3, 3]) == 0
    taps = _filters([0.5, 0.2, 0.2], [9, 9, 9])
    assert otrain.choose_filter(taps, [9, 9, 9], [3, 3, 3]) == 1


def test_choose_filter_uses_the_outermost_tap_of_the_current_length():
    # filter 0: small centre tap, large outermost tap; filter 1 the opposite.
    h0 = np.zeros(8, np.complex128); h0[0] = 0.01; h0[3] = 0.6
    h1 = np.zeros(8, np.complex128); h1[0] = 2.0; h1[3] = 0.05
    assert otrain.choose_filter([h0, h1], [7, 7], [1, 1]) == 1
    # taps beyond the current length (already pruned) do not count
    h0[4] = 1e-9
    h1[3] = 0.05; h1[2] = 0.7
    assert otrain.choose_filter([h0, h1], [7, 5], [1, 1]) == 0


def test_choose_filter_compares_complex_magnitudes():
    h0 = np.zeros(4, np.complex128); h0[1] = -0.5
    h1 = np.zeros(4, np.complex128); h1[1] = 0.3j
    h2 = np.zeros(4, np.complex128); h2[1] = 0.25 + 0.25j  # |.| = 0.354
    assert otrain.choose_filter([h0, h1, h2], [3, 3, 3], [1, 1, 1]) == 1


def test_product_pruning_rule_matches_the_oracle():
    pytest.importorskip("torch")
    from paper_2010_14258_gb300 import train
    rng = np.random.default_rng(11)
    for _ in range(300):
        M = int(rng.integers(1, 26))
        target = int(rng.choice([1, 3, 5]))
        T = [int(rng.choice([1, 3, 5, 7, 9, 31])) for _ in range(M)]
        taps = rng.standard_normal((M, 16)) + 1j * rng.standard_normal((M, 16))
        if rng.random() < 0.3:  # exact ties
            taps[:, :] = np.round(taps, 1)
        assert train.prune_choice(taps, T, target) == otrain.choose_filter(list(taps), T, [target] * M)
        per = [int(rng.choice([1, 3, 5])) for _ in range(M)]
        assert train.prune_choice(taps, T, per) == otrain.choose_filter(list(taps), T, per)


@pytest.mark.parametrize("b", [0.1, 0.25, 1.0])
def test_raised_cosine_flat_top_support_and_nyquist_point(b):
    lo, hi = (1 - b) / 2, (1 + b) / 2
    nu = np.linspace(-1.5, 1.5, 30001)
    rc = txrx.raised_cosine(nu, b)
    assert np.all(rc[np.abs(nu) <= lo - 1e-12] == 1.0)
    assert np.all(rc[np.abs(nu) >= hi + 1e-12] == 0.0)
    # strictly inside the transition band on both sides of its edges
    eps = 1e-4
    for edge_in in (lo + eps, hi - eps):
        v = txrx.raised_cosine(np.array([edge_in, -edge_in]), b)
        assert np.all((v > 0.0) & (v < 1.0))
    assert np.allclose(txrx.raised_cosine(np.array([0.5, -0.5]), b), 0.5, atol=1e-15)
    # vestigial symmetry about the Nyquist frequency
    x = np.linspace(0, b / 2, 101)
    assert np.allclose(txrx.raised_cosine(0.5 - x, b) + txrx.raised_cosine(0.5 + x, b), 1.0, atol=1e-14)


def test_raised_cosine_roll_off_is_the_stated_one():
    # with b = 0.1 the spectrum is nonzero up to 0.55 and below 1 from 0.45 on;
    # b = 0.05 or 0.2 would put these edges elsewhere
    rc = txrx.raised_cosine(np.array([0.449, 0.451, 0.549, 0.551]), 0.1)
    assert rc[0] == 1.0 and rc[1] < 1.0 and rc[2] > 0.0 and rc[3] == 0.0
    # quarter points of the transition: 0.5 (1 +- cos(pi/4))
    q = txrx.raised_cosine(np.array([0.475, 0.525]), 0.1)
    assert np.allclose(q, [0.5 * (1 + np.sqrt(0.5)), 0.5 * (1 - np.sqrt(0.5))], atol=1e-14)


@pytest.mark.parametrize("b", [0.1, 0.3])
def test_raised_cosine_inverse_transform_is_the_rc_pulse(b):
    # sample the spectrum finely over a long symbol window and transform
    sps, nsym = 16, 512
    n = sps * nsym
    H = txrx.raised_cosine(np.fft.fftfreq(n) * sps, b)
    p = np.real(np.fft.ifft(H)) * sps          # pulse at t = m / sps symbols
    t = np.fft.fftfreq(n) * n / sps
    with np.errstate(divide="ignore", invalid="ignore"):
        ref = np.sinc(t) * np.cos(np.pi * b * t) / (1 - (2 * b * t) ** 2)
    sing = np.isclose(np.abs(2 * b * t), 1.0)
    ref[sing] = np.pi / 4 * np.sinc(1 / (2 * b))
    near = np.abs(t) <= 40
    # the periodic window folds the tails; they decay as t^-3, so compare near t = 0
    assert np.max(np.abs(p[near] - ref[near])) < 2e-4
    assert abs(p[0] - 1.0) < 1e-4                 # Nyquist: p(0) = 1, p(k) = 0
    k = (np.abs(t - np.round(t)) < 1e-12) & (np.abs(t) >= 1) & near
    assert np.max(np.abs(p[k])) < 2e-4
