"""Seeded synthetic inputs shared by the tests, the benchmark and the training loop.

This module draws random numbers and names workloads; it holds none of the
split-step, filtering or receiver arithmetic.  Both the CUDA path and the
FP64 oracle receive what it returns as plain inputs.

Workload recipes follow the link and signal parameters the paper states
(Sec. IV-A system model; Table I: alpha = 0.2 dB/km, gamma = 1.3 /W/km,
nu_s = 1.946e14 Hz, NF = 5 dB, RRC roll-off 0.1, 2 samples/symbol).
"""
from __future__ import annotations

import dataclasses
import numpy as np

# 16-QAM alphabet {+-1, +-3}^2 scaled to unit mean energy (E|s|^2 = 1).
_QAM16_LEVELS = np.array([-3.0, -1.0, 1.0, 3.0])
QAM16 = ((_QAM16_LEVELS[:, None] + 1j * _QAM16_LEVELS[None, :]).reshape(-1)
         / np.sqrt(10.0))


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def qam16_indices(batch: int, nsym: int, seed: int) -> np.ndarray:
    """Uniform i.i.d. 16-QAM symbol indices, shape [batch, nsym], uint8."""
    return rng(seed).integers(0, 16, size=(batch, nsym), dtype=np.uint8)


def qam16_symbols(batch: int, nsym: int, seed: int) -> np.ndarray:
    """Uniform i.i.d. 16-QAM symbols with E|s|^2 = 1, complex128 [batch, nsym]."""
    return QAM16[qam16_indices(batch, nsym, seed)]


def gaussian_waveform(batch: int, n: int, seed: int, power: float = 1.0) -> np.ndarray:
    """Circular complex Gaussian samples with E|x|^2 = power, complex128 [batch, n]."""
    g = rng(seed)
    z = g.standard_normal((batch, n)) + 1j * g.standard_normal((batch, n))
    return z * np.sqrt(power / 2.0)


def launch_powers_dbm(batch: int, seed: int, grid_dbm) -> np.ndarray:
    """Per-frame launch power drawn uniformly from a discrete set (dBm)."""
    grid = np.asarray(grid_dbm, dtype=np.float64)
    return grid[rng(seed).integers(0, len(grid), size=batch)]


def complex_normal(shape, seed: int, std: float = 1.0) -> np.ndarray:
    """Circular complex Gaussian perturbation with E|z|^2 = std^2."""
    g = rng(seed)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) * (std / np.sqrt(2.0))


def ragged_lengths(count: int, seed: int, log2_lo: float = 12.0, log2_hi: float = 18.0):
    """Waveform lengths log-uniform over [2^lo, 2^hi], rounded to even."""
    g = rng(seed)
    n = np.round(2.0 ** g.uniform(log2_lo, log2_hi, size=count)).astype(np.int64)
    return n + (n % 2)


def ragged_spans(count: int, seed: int, lo: int = 5, hi: int = 40) -> np.ndarray:
    return rng(seed + 1).integers(lo, hi + 1, size=count).astype(np.int64)


def ragged_taps(count: int, seed: int, choices=(3, 5, 9, 15, 31)) -> np.ndarray:
    return np.asarray(choices, dtype=np.int64)[rng(seed + 2).integers(0, len(choices), size=count)]


@dataclasses.dataclass(frozen=True)
class Fiber:
    """Standard single-mode fiber in the paper's units (Table I)."""
    alpha_db_per_km: float = 0.2
    beta2_ps2_per_km: float = -21.7
    gamma_per_w_km: float = 1.3


@dataclasses.dataclass(frozen=True)
class Link:
    n_spans: int = 10
    span_km: float = 80.0
    steps_per_span: int = 50
    symmetric: bool = True
    ase: bool = False
    nf_db: float = 5.0
    carrier_hz: float = 1.946e14
    seed: int = 0
    counter: int = 0


@dataclasses.dataclass(frozen=True)
class Signal:
    baud: float = 10e9
    sps: int = 2
    rolloff: float = 0.1
    nsym: int = 8192

    @property
    def fs(self) -> float:
        return self.baud * self.sps

    @property
    def n(self) -> int:
        return self.nsym * self.sps


# Named workloads (sizes and link shapes of the paper's 10 GBd / 32 GBd links).
PLAIN_SSM_16K = dict(signal=Signal(10e9, 2, 0.1, 8192), fiber=Fiber(),
                     link=Link(10, 80.0, 50, True, False), dbp_steps=1,
                     power_dbm=2.0, seed=1)
LDBP_INFER_256x64K = dict(signal=Signal(10e9, 2, 0.1, 32768), fiber=Fiber(),
                          link=Link(25, 80.0, 100, True, True), batch=256,
                          taps=(3, 5, 9, 15), power_dbm=0.0, seed=2)
LDBP_TRAIN_64x32K = dict(signal=Signal(10e9, 2, 0.1, 16384), fiber=Fiber(),
                         link=Link(25, 80.0, 100, True, True), batch=64,
                         powers_dbm=tuple(range(-4, 7)), t_start=31, t_end=3, seed=3)
CHANNEL_128x128K = dict(signal=Signal(32e9, 4, 0.1, 32768), fiber=Fiber(),
                        link=Link(10, 100.0, 200, True, True), batch=128,
                        power_dbm=0.0, seed=4)
RAGGED_1000 = dict(count=1000, seed=5, taps=(3, 5, 9, 15, 31), spans=(5, 40),
                   log2_len=(12.0, 18.0), span_km=80.0, fiber=Fiber(),
                   signal=Signal(10e9, 2, 0.1, 0))
