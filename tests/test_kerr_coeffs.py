"""The Kerr-step polynomial constants compiled into csrc/ldbp_tile.cuh are the
ones the committed generator (paper_2010_14258_gb300/kerr_coeffs.py, Remez
exchange in FP64) produces, and they approximate sin and cos - 1 on their
tiers to the stated equal-ripple error."""
import os
import re

import numpy as np
import pytest

from paper_2010_14258_gb300 import kerr_coeffs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2010_14258_gb300", "csrc", "ldbp_tile.cuh")


def _constants():
    text = open(HEADER).read()
    return {m.group(1): float(m.group(2)) for m in re.finditer(r"\b(k(?:Sin|Cos)[AB]\d)\s*=\s*([-+0-9.eE]+)f", text)}


TIERS = [("A", 0.5, [1, 3, 5], [2, 4, 6], 2.5e-8, 1e-9), ("B", 1.0, [1, 3, 5, 7], [2, 4, 6, 8], 1.1e-8, 7e-10)]


@pytest.mark.parametrize("tier,X,sp,cp,esin,ecos", TIERS)
def test_header_constants_are_the_generators(tier, X, sp, cp, esin, ecos):
    k = _constants()
    a, ea = kerr_coeffs.remez(np.sin, sp, X)
    b, eb = kerr_coeffs.remez(lambda x: np.cos(x) - 1.0, cp, X)
    assert ea <= esin and eb <= ecos
    for q, v in zip(sp, a):
        assert k[f"kSin{tier}{q}"] == pytest.approx(v, rel=1e-12, abs=1e-15)
    for q, v in zip(cp, b):
        assert k[f"kCos{tier}{q}"] == pytest.approx(v, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("tier,X,sp,cp,esin,ecos", TIERS)
def test_header_polynomials_approximate_sin_and_cos(tier, X, sp, cp, esin, ecos):
    # independent of the generator: the constants as compiled (rounded to
    # float) against numpy's sin / cos on a fine grid of the tier
    k = {n: float(np.float32(v)) for n, v in _constants().items()}
    x = np.linspace(-X, X, 400001)
    s = sum(k[f"kSin{tier}{q}"] * x ** q for q in sp)
    c = 1.0 + sum(k[f"kCos{tier}{q}"] * x ** q for q in cp)
    assert np.max(np.abs(s - np.sin(x))) < 1.2e-7   # below one FP32 ulp of 1 after rounding the constants
    assert np.max(np.abs(c - np.cos(x))) < 1.2e-7
    assert c[len(x) // 2] == 1.0                    # cos(0) exact: no bias of |exp(j phi)| at small phases
