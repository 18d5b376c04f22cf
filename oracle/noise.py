"""FP64 CPU oracle of the mock's total uncertainty per k bin (thermal noise, sample variance
and modelling error).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this module. It shares no code with the
CUDA library and never calls it.

Sec. 2.4 combines, for each k bin, the thermal noise of every individual mode with the
sample variance of the cosmological spectrum by an inverse-weighted sum over the bin's
modes (the T+S equation), and adds a constant fractional modelling error of 25 % in
quadrature (Sec. 2.5):

    dDelta2_TS(k_b) = ( sum_{i in b} 1 / (Delta2_N,i + Delta2_21(k_b))^2 )^(-1/2),
    sigma_b^2       = dDelta2_TS(k_b)^2 + (f_model Delta2_21(k_b))^2.

Modes are those of the full n^3 grid with k != 0 in the bin (the binning of the power
spectrum: logarithmic bins on [k_lo, k_hi), half-open). Pins
(tests/test_oracle_noise.py): with no thermal noise the T+S term is the Gaussian sample
variance Delta2 / sqrt(N_modes); with a constant thermal noise it is
(N + Delta2) / sqrt(N_modes); the modelling term adds in quadrature; mode counts equal
the power-spectrum oracle's.
"""
from __future__ import annotations

import numpy as np


def mode_bins(n: int, box_mpc: float, nbins: int, k_lo: float, k_hi: float) -> np.ndarray:
    """Bin of every mode of the full n^3 grid (-1 outside [k_lo, k_hi) and at k = 0), in
    numpy's FFT index order [kx][ky][kz]."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    kf = 2.0 * np.pi / box_mpc
    k = kf * np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
    out = np.full(k.shape, -1, dtype=np.int64)
    ok = (k >= k_lo) & (k < k_hi) & (k > 0)
    b = np.floor(nbins * np.log(k[ok] / k_lo) / np.log(k_hi / k_lo)).astype(np.int64)
    b[(b < 0) | (b >= nbins)] = -1
    out[ok] = b
    return out


def total_sigma(n: int, box_mpc: float, d2_21, thermal, model_frac: float, nbins: int = 14,
                k_lo: float = 0.1, k_hi: float = 1.5):
    """sigma_b (FP64, [nbins]) for one redshift: d2_21 [nbins] is the cosmological spectrum
    (the mock's), thermal [n][n][n] the per-mode thermal noise Delta2_N,i on the full grid
    (None: zero). Bins without modes give NaN. Also returns the mode counts."""
    bins = mode_bins(n, box_mpc, nbins, k_lo, k_hi)
    d2 = np.asarray(d2_21, dtype=np.float64)
    noise = np.zeros(bins.shape) if thermal is None else np.asarray(thermal, dtype=np.float64)
    sigma = np.full(nbins, np.nan)
    counts = np.zeros(nbins, dtype=np.int64)
    for b in range(nbins):
        sel = bins == b
        counts[b] = int(sel.sum())
        if counts[b] == 0:
            continue
        inv = np.sum(1.0 / (noise[sel] + d2[b]) ** 2)
        ts = inv ** -0.5
        sigma[b] = np.sqrt(ts * ts + (model_frac * d2[b]) ** 2)
    return sigma, counts
