"""Pins of the oracle's velocity-gradient term of delta T_b (Sec. 2.2): the growth rate
f = d ln D / d ln a against the Einstein-de Sitter value, the numerical derivative of the
oracle's own D(z) and Linder's fit, and the line-of-sight field IDFT(k_z^2/k^2 delta_hat)
against plane waves along, across and at 45 degrees to the line of sight."""
import numpy as np
import pytest

import oracle


def test_growth_rate_einstein_de_sitter():
    o = oracle.Oracle(oracle.Cosmology(omega_m=1.0, omega_l=0.0))
    for z in (0.0, 3.0, 9.0):
        assert o.growth_rate(z) == pytest.approx(1.0, abs=1e-9)


def test_growth_rate_is_the_derivative_of_ln_d():
    o = oracle.Oracle()
    for z in (0.0, 1.0, 8.0, 10.0):
        a = 1.0 / (1.0 + z)
        h = 1e-4
        za, zb = 1.0 / (a * np.exp(h)) - 1.0, 1.0 / (a * np.exp(-h)) - 1.0
        numeric = (np.log(o.growth(za)) - np.log(o.growth(zb))) / (2 * h)
        assert o.growth_rate(z) == pytest.approx(numeric, rel=1e-6)


def test_growth_rate_linder_fit():
    o = oracle.Oracle()
    om = o.cosmo.omega_m
    for z in (0.0, 0.5, 2.0, 8.0):
        a = 1.0 / (1.0 + z)
        om_z = om / a ** 3 / (om / a ** 3 + 1.0 - om)
        assert o.growth_rate(z) == pytest.approx(om_z ** 0.55, rel=1e-2)


def _plane(n, mvec, amp=0.3):
    x = np.arange(n)
    ix, iy, iz = np.meshgrid(x, x, x, indexing="ij")
    phase = 2 * np.pi * (mvec[0] * ix + mvec[1] * iy + mvec[2] * iz) / n
    return (amp * np.cos(phase)).astype(np.float32)


def _los(o, d, box):
    g = np.empty(d.shape)
    n = d.shape[0]
    o.lib.or_los_gradient(n, box, oracle._ptr(np.ascontiguousarray(d)), oracle._ptr(g))
    return g


def test_los_gradient_plane_waves():
    o = oracle.Oracle()
    n, box = 16, 40.0
    along = _plane(n, (0, 0, 3))
    assert np.allclose(_los(o, along, box), along, atol=1e-12)
    across = _plane(n, (2, 1, 0))
    assert np.allclose(_los(o, across, box), 0.0, atol=1e-12)
    diag = _plane(n, (2, 0, 2))
    assert np.allclose(_los(o, diag, box), 0.5 * diag, atol=1e-12)


def test_rsd_weight_closed_form_and_clip():
    o = oracle.Oracle()
    n, box, z = 16, 40.0, 9.0
    d = _plane(n, (0, 0, 1), amp=0.1)
    d64 = d.astype(np.float64)
    f = o.growth_rate(z)
    w = o.rsd_weight(d, box, z, 10.0)   # no clipping at this amplitude
    assert np.allclose(w, (1 + d64) / (1 - f * d64), rtol=1e-12)
    wc = o.rsd_weight(d, box, z, 0.05)  # |f delta| up to 0.1: clipped at 0.05
    dvdr = np.clip(-f * d64, -0.05, 0.05)
    assert np.allclose(wc, (1 + d64) / (1 + dvdr), rtol=1e-12)
    assert np.abs(dvdr).max() == pytest.approx(0.05)
