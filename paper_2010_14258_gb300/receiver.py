"""Receiver DSP chain of Sec. IV-A with full-length DBP as the fallback of LDBP.

The chain is (i) backpropagation, (ii) the matched filter with downsampling and
(iii) the phase-offset correction (Eq. (12)).  A learned model enters the chain
only after validation: on held-out received waveforms its effective SNR
(Eq. (14)) is compared with that of full-length frequency-domain DBP (Sec. IV,
the split-step method LDBP approximates with short filters) on the same
waveforms.  If LDBP is more than ``tolerance_db`` below DBP, or has not been
validated yet, the receiver backpropagates with DBP instead.

All arithmetic runs in the library's kernels (ldbp_apply, dbp_apply, ldbp_rx);
this module only chooses between them.
"""
from __future__ import annotations

import dataclasses


@dataclasses.dataclass(frozen=True)
class Decision:
    """Outcome of one validation: the two effective SNRs (dB) and the margin."""
    snr_ldbp_db: float
    snr_dbp_db: float
    tolerance_db: float

    @property
    def use_ldbp(self) -> bool:
        return self.snr_ldbp_db >= self.snr_dbp_db - self.tolerance_db


class Receiver:
    """LDBP receiver with a validated fallback to full-length FD DBP.

    taps, T, c: the LDBP model as ldbp_apply takes it (device taps [M, stride],
    per-step lengths, per-step nonlinear coefficients).  fiber, link, fs,
    dbp_steps_per_span, dbp_symmetric: the DBP that serves as the fallback and
    as the SNR reference.  backend: the module providing ldbp_apply,
    dbp_apply, rx and snr_db (the package's ``api`` unless given).
    """

    def __init__(self, taps, T, c, fiber, link, fs, dbp_steps_per_span=1, dbp_symmetric=False,
                 tolerance_db=0.1, sps=2, rolloff=0.1, backend=None):
        if backend is None:
            from . import api as backend
        self.backend = backend
        self.taps, self.T, self.c = taps, list(T), list(c)
        self.fiber, self.link, self.fs = fiber, link, float(fs)
        self.dbp_steps_per_span, self.dbp_symmetric = int(dbp_steps_per_span), bool(dbp_symmetric)
        self.tolerance_db = float(tolerance_db)
        self.sps, self.rolloff = int(sps), float(rolloff)
        self.decision = None

    def ldbp(self, y):
        return self.backend.ldbp_apply(self.taps, self.T, self.c, y)

    def dbp(self, y):
        return self.backend.dbp_apply(self.fiber, self.link, self.fs, y, self.dbp_steps_per_span,
                                      self.dbp_symmetric)

    def _snr(self, z, symbols, power_w):
        stats, _, _ = self.backend.rx(z, symbols, power_w, sps=self.sps, rolloff=self.rolloff)
        return self.backend.snr_db(stats)

    def validate(self, y, symbols, power_w) -> Decision:
        """Effective SNR of LDBP and of DBP on the same received waveforms y [B, n]."""
        self.decision = Decision(self._snr(self.ldbp(y), symbols, power_w),
                                 self._snr(self.dbp(y), symbols, power_w), self.tolerance_db)
        return self.decision

    @property
    def uses_ldbp(self) -> bool:
        return self.decision is not None and self.decision.use_ldbp

    def backpropagate(self, y):
        """LDBP if the last validation accepted it, else DBP."""
        return self.ldbp(y) if self.uses_ldbp else self.dbp(y)

    def __call__(self, y, symbols, power_w):
        """The whole chain: backpropagation, matched filter, phase correction.
        Returns (stats [B, 2], phi [B]) as ``rx`` does."""
        stats, phi, _ = self.backend.rx(self.backpropagate(y), symbols, power_w, sps=self.sps,
                                        rolloff=self.rolloff)
        return stats, phi
