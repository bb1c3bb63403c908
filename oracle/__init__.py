"""FP64 CPU oracle for the split-step / learned-DBP hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA library (no kernels, tables, constants or
pre/post-processing); the only common dependency is the seeded input module
``synth``, which holds none of the method's arithmetic.

Every function is a plain, unblocked restatement of the paper's definitions in
complex128 / float64, using numpy's FFT and least squares as library steps.
Citations name the section, equation, remark or example of
Haeger & Pfister, "Physics-Based Deep Learning for Fiber-Optic Communication
Systems" (IEEE JSAC 2021, arXiv:2010.14258).  Displayed equations are numbered
in order of appearance (Eq. (4) NLSE, (5) time-discretised NLSE, (6)
asymmetric SSM, (7) parameterised model, (8) symmetric SSM, (9)-(10) enhanced
SSM, (11) transmit signal, (12) receiver chain, (13) expected MSE,
(14) effective SNR, (15) CD memory).

Parity status per function is listed in each module header.
"""
from . import philox, nlse, ldbp, txrx, train  # noqa: F401
