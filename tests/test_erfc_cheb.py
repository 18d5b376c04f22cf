"""The Chebyshev-fitted erfc used for f_coll at R_cell (Eq. 1's erfc) by the TF32 contraction's
epilogue and the flag contraction's pencil pass, checked on the CPU: its coefficients are read from the CUDA source and the formula,
evaluated in FP64, must stay within the published fractional error bound (1.2e-7) of erfc
over the whole non-negative axis, and reduce to 1 at x = 0."""
import os
import re

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1501_06576_gb300", "csrc", "eor_internal.cuh")


def coefficients():
    text = open(SRC).read()
    body = text[text.index("float erfc_cheb(float x)"):]
    body = body[:body.index("\n}\n")]
    lits = [float(v) for v in re.findall(r"(-?\d+\.\d+)f", body)]
    # t = 1 / (1 + 0.5 x) first (the numerator, then the fmaf's 0.5 and 1), then the ten
    # polynomial coefficients from the top
    assert lits[:3] == [1.0, 0.5, 1.0]
    return lits[3:]


def erfc_cheb64(x, c):
    t = 1.0 / (1.0 + 0.5 * x)
    p = c[0]
    for a in c[1:]:
        p = p * t + a
    return t * np.exp(-x * x + p)


def test_coefficient_count():
    assert len(coefficients()) == 10


def test_within_published_bound():
    special = pytest.importorskip("scipy.special")
    c = coefficients()
    x = np.concatenate([np.linspace(0.0, 6.0, 60001), np.linspace(6.0, 12.0, 2001)])
    rel = np.abs(erfc_cheb64(x, c) / special.erfc(x) - 1.0)
    assert rel.max() < 1.2e-7


def test_zero_and_large_argument():
    c = coefficients()
    assert abs(erfc_cheb64(np.array([0.0]), c)[0] - 1.0) < 1.2e-7
    assert erfc_cheb64(np.array([30.0]), c)[0] < 1e-300
