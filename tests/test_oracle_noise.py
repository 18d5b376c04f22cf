"""Pins of the total-noise oracle (oracle/noise.py, the T+S combination of Sec. 2.4 plus the
modelling error of Sec. 2.5) against closed forms and the power-spectrum oracle's counts."""
import numpy as np
import pytest

import oracle
from oracle import noise


def test_counts_match_power_spectrum_oracle():
    n, box = 32, 60.0
    _, _, cnt = oracle.power_spectrum(np.zeros((n, n, n)) + 1.0, box, 14, 0.1, 1.5)
    _, counts = noise.total_sigma(n, box, np.ones(14), None, 0.0)
    assert np.array_equal(counts, cnt)


def test_sample_variance_limit():
    n, box = 32, 60.0
    d2 = np.geomspace(5.0, 50.0, 14)
    sig, counts = noise.total_sigma(n, box, d2, None, 0.0)
    ok = counts > 0
    assert np.allclose(sig[ok], d2[ok] / np.sqrt(counts[ok]), rtol=1e-12)
    assert np.all(np.isnan(sig[~ok]))


def test_constant_thermal_noise_and_model_term():
    n, box = 32, 60.0
    d2 = np.geomspace(5.0, 50.0, 14)
    thermal = np.full((n, n, n), 7.0)
    sig, counts = noise.total_sigma(n, box, d2, thermal, 0.0)
    ok = counts > 0
    assert np.allclose(sig[ok], (7.0 + d2[ok]) / np.sqrt(counts[ok]), rtol=1e-12)
    sig25, _ = noise.total_sigma(n, box, d2, thermal, 0.25)
    assert np.allclose(sig25[ok] ** 2, sig[ok] ** 2 + (0.25 * d2[ok]) ** 2, rtol=1e-12)


def test_noisier_modes_weigh_less():
    n, box = 16, 30.0
    d2 = np.full(14, 10.0)
    rng = np.random.default_rng(0)
    thermal = rng.uniform(0, 100, (n, n, n))
    sig, counts = noise.total_sigma(n, box, d2, thermal, 0.0)
    lo, _ = noise.total_sigma(n, box, d2, None, 0.0)
    ok = counts > 0
    assert np.all(sig[ok] >= lo[ok])   # adding noise never lowers the uncertainty
    # a single-mode bin is |N + Delta2|
    b = np.nonzero(counts == 1)[0]
    for bb in b:
        sel = noise.mode_bins(n, box, 14, 0.1, 1.5) == bb
        assert sig[bb] == pytest.approx(thermal[sel][0] + 10.0)
