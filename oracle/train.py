"""Optimiser and pruning bookkeeping, FP64 (oracle side).

* Adam (Sec. IV-B uses Adam, Table I: learning rate 1e-3), restated from
  Kingma & Ba's algorithm: m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
  theta <- theta - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps), applied
  to the real and imaginary parts of every tap separately.
* Pruning (Sec. IV-C, Example 2): each pruning step removes the two outermost
  taps of one filter (mask them to zero), at predefined iterations, with more
  steps early in training.  Readings: pruning steps fall at
  floor(frac * iters * (j / P)^2), j = 1..P (front-loaded); the filter pruned
  at each step is, among filters still longer than their target, the one
  whose outermost tap has the smallest magnitude (ties: lowest step index).
"""
from __future__ import annotations

import numpy as np


def adam(theta, g, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update on real arrays (t counts from 1).  Returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def pruning_steps(t_start, t_end) -> int:
    """Number of pruning steps: sum_i (T'_i - T_i) / 2 (Example 2)."""
    return int(sum((a - b) // 2 for a, b in zip(t_start, t_end)))


def pruning_iterations(total_steps: int, iters: int, frac: float = 0.6):
    return [int(np.floor(frac * iters * (j / total_steps) ** 2)) for j in range(1, total_steps + 1)]


def choose_filter(taps, lengths, targets) -> int:
    """Index of the filter whose outermost tap is smallest among those above target."""
    best, best_mag = -1, np.inf
    for i, (h, T, Tt) in enumerate(zip(taps, lengths, targets)):
        if T > Tt:
            mag = abs(h[(T - 1) // 2])
            if mag < best_mag:
                best, best_mag = i, mag
    return best
