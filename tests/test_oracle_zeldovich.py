"""Pins of the Zel'dovich oracle (oracle/zeldovich.py) against closed forms and invariants."""
import numpy as np
import pytest

from oracle import zeldovich as zel
from paper_1501_06576_gb300 import synth


def _plane(n, mvec, amp):
    x = np.arange(n)
    ix, iy, iz = np.meshgrid(x, x, x, indexing="ij")
    return amp * np.cos(2 * np.pi * (mvec[0] * ix + mvec[1] * iy + mvec[2] * iz) / n)


def test_zero_field_and_mass():
    n, box = 16, 40.0
    assert np.allclose(zel.evolve(np.zeros((n, n, n)), box), 0.0, atol=1e-14)
    d = synth.density_box(n, box, 9.0, seed=3).astype(np.float64)
    nl = zel.evolve(d, box)
    assert np.sum(1.0 + nl) == pytest.approx(n ** 3, rel=1e-12)
    assert nl.min() >= -1.0 - 1e-12


def test_plane_wave_displacement_closed_form():
    # delta = A cos(k . q) -> psi = -A sin(k . q) k / k^2 (div psi = -delta)
    n, box, amp = 16, 40.0, 0.2
    m = (2, 0, 1)
    d = _plane(n, m, amp)
    psi = zel.displacement(d, box)
    kf = 2 * np.pi / box
    k = kf * np.array(m, dtype=float)
    x = np.arange(n)
    ix, iy, iz = np.meshgrid(x, x, x, indexing="ij")
    s = np.sin(2 * np.pi * (m[0] * ix + m[1] * iy + m[2] * iz) / n)
    for j in range(3):
        want = -amp * s * k[j] / (k @ k) / (box / n)
        assert np.allclose(psi[j], want, atol=1e-12)


def test_first_order_limit():
    # small amplitude: delta_nl follows delta_L (sign and scale of psi: a displacement in Mpc
    # instead of cells, or of the wrong sign, fails this), CIC smoothing taking a few per cent
    n, box = 16, 40.0
    d = synth.density_box(n, box, 9.0, seed=5).astype(np.float64)
    m = np.abs(np.fft.fftfreq(n, d=1.0 / n))
    keep = (m[:, None, None] <= 2) & (m[None, :, None] <= 2) & (m[None, None, :] <= 2)
    smooth = np.fft.ifftn(np.fft.fftn(d) * keep).real   # large scales: little CIC smoothing
    lin = 0.01 * smooth / smooth.std()
    nl = zel.evolve(lin, box)
    # CIC deposit of sub-cell displacements differences psi one-sidedly: a shift of up to half
    # a cell, cos(k dx / 2) >= 0.92 of correlation for these modes (k dx <= 2 pi 2 / 16)
    assert np.corrcoef(nl.ravel(), lin.ravel())[0, 1] > 0.9
    assert 0.9 < nl.std() / lin.std() < 1.1
    # and the departure from linear order grows as the square of the amplitude
    r = [zel.evolve(2 * a * lin, box) - 2 * zel.evolve(a * lin, box) for a in (1.0, 0.5)]
    assert np.abs(r[1]).max() < 0.35 * np.abs(r[0]).max()


def test_uniform_translation_invariance():
    n, box = 16, 40.0
    d = synth.density_box(n, box, 9.0, seed=4).astype(np.float64)
    nl = zel.evolve(d, box)
    nl_shift = zel.evolve(np.roll(d, 3, axis=1), box)
    assert np.allclose(np.roll(nl, 3, axis=1), nl_shift, atol=1e-12)
