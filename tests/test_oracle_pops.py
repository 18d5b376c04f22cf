"""Pins of the mass-dependent efficiency oracle (Sec. 5: sources whose ionizing efficiency is a
power law in halo mass, integrated over the extended Press-Schechter conditional mass
function) against closed forms, limits and the single-population oracle."""
import numpy as np
import pytest
from scipy.special import gamma, gammaincc

import oracle
from paper_1501_06576_gb300 import synth

DC = 1.686


@pytest.fixture(scope="module")
def o():
    return oracle.Oracle()


@pytest.fixture(scope="module")
def z9(o):
    g = o.growth(9.0)
    return g, o.var_table(g, 1e7, 1e16)


def _m_r(o, r):
    return 4.0 / 3.0 * np.pi * r ** 3 * o.rho_mean()


def test_dsigma2_dlnr_central_differences(o):
    for r in (0.8, 3.0, 15.0):
        h = 1e-3
        fd = (o.sigma2(r * np.exp(h)) - o.sigma2(r * np.exp(-h))) / (2 * h)
        assert o.dsigma2_dlnr(r) == pytest.approx(fd, rel=3e-6)


def test_variance_table_against_quadrature(o, z9):
    g, tab = z9
    for m in (2.3e7, 3.3e8, 7.7e11, 2.2e14, 9e15):
        s, ds = tab.s(m)
        r = o.mass_to_radius(m)
        assert s == pytest.approx(g * g * o.sigma2(r), rel=1e-8)
        assert ds == pytest.approx(g * g * o.dsigma2_dlnr(r) / 3.0, rel=1e-5)


def test_slope_zero_is_zeta_erfc(o, z9):
    # one population of constant efficiency above M_min: zeta erfc(nu / sqrt(2 (S_min - S_R)))
    g, tab = z9
    m_min = o.mmin(10 ** 4.7, 9.0)
    pops = np.array([[30.0, 1e10, 0.0, m_min, 0.0]])
    s_lo = g * g * o.sigma2(o.mass_to_radius(m_min))
    for r in (1.5, 5.0, 15.0):
        s_r = g * g * o.sigma2(r)
        for dr in (-1.0, 0.0, 0.7, 1.5, 1.68, 1.6859):
            want = 30.0 * o.fcoll(dr, s_lo, s_r)
            assert tab.fcoll(pops, _m_r(o, r), dr) == pytest.approx(want, rel=1e-7, abs=1e-12)


def test_split_mass_range_adds_up(o, z9):
    # [m1, m2) + [m2, inf) of the same power law is the power law on [m1, inf)
    _, tab = z9
    m1, m2 = 2e8, 3e9
    for slope in (-0.5, 0.3):
        whole = np.array([[20.0, 1e10, slope, m1, 0.0]])
        split = np.array([[20.0, 1e10, slope, m1, m2], [20.0, 1e10, slope, m2, 0.0]])
        for dr in (0.2, 1.1, 1.6):
            a = tab.fcoll(whole, _m_r(o, 6.0), dr)
            b = tab.fcoll(split, _m_r(o, 6.0), dr)
            assert b == pytest.approx(a, rel=1e-9)


def test_collapsed_region_limit(o, z9):
    # delta_R -> delta_c: all the region's mass is in one halo of mass M_R
    _, tab = z9
    m_r = _m_r(o, 4.0)
    pops = np.array([[25.0, 1e10, 0.4, 3e8, 0.0], [5.0, 1e10, -0.3, 1e9, 0.0], [7.0, 1e10, 0.0, 1e8, 1e10]])
    want = 25.0 * (m_r / 1e10) ** 0.4 + 5.0 * (m_r / 1e10) ** -0.3   # third range ends below M_R
    assert tab.fcoll(pops, m_r, DC) == pytest.approx(want, rel=1e-12)
    assert tab.fcoll(pops, m_r, DC + 0.5) == pytest.approx(want, rel=1e-12)
    assert tab.fcoll(pops, m_r, DC - 1e-7) == pytest.approx(want, rel=1e-5)
    # a population whose range starts above M_R contributes nothing
    assert tab.fcoll(np.array([[30.0, 1e10, 0.2, 2 * m_r, 0.0]]), m_r, 1.0) == 0.0


def test_power_law_spectrum_incomplete_gamma():
    # P ~ k^-2: sigma^2 ~ R^-1, S = S_p (M/M_p)^(-1/3). Without a region (S_R = 0) the
    # efficiency-weighted fraction is zeta0 S_p^b (nu^2/2)^(-b) Gamma(b + 1/2, nu^2 / (2 S_lo)) / sqrt(pi)
    # with b = 3 slope (substituting u = nu^2 / (2 S) in the first-crossing distribution)
    o = oracle.Oracle(oracle.Cosmology(n_s=-2.0, use_transfer=False))
    tab = o.var_table(1.0, 1e8, 1e18)
    mp, m_lo, nu = 1e10, 1e8, DC
    s_p = o.sigma2(o.mass_to_radius(mp))
    s_lo = o.sigma2(o.mass_to_radius(m_lo))
    # the spectrum is a power law up to the quadrature's cut at k = 1e-6 / Mpc, which leaves
    # out a relative 1e-6 R [Mpc] of sigma^2 (2e-7 here, up to 1e-5 at the masses where the
    # integrand peaks): hence the 1e-5 below; a wrong slope mapping is off by tens of per cent
    assert s_lo / s_p == pytest.approx((m_lo / mp) ** (-1.0 / 3.0), rel=1e-6)
    for slope in (0.2, -0.1, 0.0):
        b = 3.0 * slope
        want = 12.0 * s_p ** b * (nu * nu / 2) ** (-b) * gammaincc(b + 0.5, nu * nu / (2 * s_lo)) * gamma(b + 0.5)
        want /= np.sqrt(np.pi)
        got = tab.fcoll(np.array([[12.0, mp, slope, m_lo, 0.0]]), 0.0, 0.0)
        assert got == pytest.approx(want, rel=1e-5)


def test_feedback_form_mass_slopes(o):
    # Sec. 5's efficiency is a power law in T_vir; at fixed z, zeta at M = M_min(T) must be
    # zeta0 (T / T_F)^alpha below T_F and zeta0 (T / T_F)^beta above
    z, alpha, beta, logtf = 8.0, 4.0 / 3.0, -1.0 / 3.0, 4.7
    pops = o.populations(2, (70.0, 15.0, logtf), (alpha, beta, 0.0, 0.0), z)
    assert pops.shape == (2, 5)
    for t in (1.5e4, 3e4, 2e5, 1e6):
        m = o.mmin(t, z)
        p = pops[0] if t < 10 ** logtf else pops[1]
        assert p[3] <= m and (p[4] <= 0 or m < p[4])
        zeta = p[0] * (m / p[1]) ** p[2]
        want = 70.0 * (t / 10 ** logtf) ** (alpha if t < 10 ** logtf else beta)
        assert zeta == pytest.approx(want, rel=1e-10)
    # no efficiency below the atomic-cooling threshold
    assert pops[0][3] == pytest.approx(o.mmin(1e4, z), rel=1e-12)


def test_ionize_pops_reduces_to_single_population(o):
    n, box, z = 16, 40.0, 9.0
    d = synth.density_box(n, box, z, seed=7)
    ref = o.ionize(d, box, z, 30.0, 10.0, 4.7)
    pops = np.array([[30.0, 1e10, 0.0, o.mmin(10 ** 4.7, z), 0.0]])
    got = o.ionize_pops(d, box, z, pops, 10.0)
    assert got["n_radii"] == ref["n_radii"]
    assert np.array_equal(got["flag"], ref["flag"])
    assert np.abs(got["xhi"] - ref["xhi"]).max() < 1e-7
    assert got["xhi_mean"] == pytest.approx(ref["xhi_mean"], abs=1e-8)


def test_ionize_pops_monotone_in_efficiency(o):
    n, box, z = 16, 40.0, 8.0
    d = synth.density_box(n, box, z, seed=8)
    lo = o.ionize_pops(d, box, z, o.populations(1, (10.0, 8.0, 4.5), (0.3, 5.0, -0.4, 5.0), z), 8.0)
    hi = o.ionize_pops(d, box, z, o.populations(1, (20.0, 8.0, 4.5), (0.3, 5.0, -0.4, 5.0), z), 8.0)
    assert np.all(hi["xhi"] <= lo["xhi"] + 1e-12)
    assert np.all(lo["flag"] <= hi["flag"])
    assert 0.0 <= hi["xhi"].min() and lo["xhi"].max() <= 1.0


def test_feedback_form_without_faint_range(o):
    # T_F below the atomic-cooling threshold: no faint population, the bright one starts at
    # M(10^4 K) and is pivoted at M_F
    pops = o.populations(2, (40.0, 10.0, 3.8), (1.0, -0.2, 0.0, 0.0), 9.0)
    assert pops.shape == (1, 5)
    assert pops[0][3] == pytest.approx(o.mmin(1e4, 9.0), rel=1e-12)
    assert pops[0][1] == pytest.approx(o.mmin(10 ** 3.8, 9.0), rel=1e-12)
    assert pops[0][2] == pytest.approx(2.0 * -0.2 / 3.0)
    assert pops[0][4] == 0.0


def test_two_population_model_second_population_off(o, z9):
    # zeta_20 = 0 in model 1 adds nothing
    _, tab = z9
    one = o.populations(1, (25.0, 10.0, 4.6), (0.2, 0.0, 0.4, 5.0), 9.0)
    assert one.shape == (2, 5)
    m_r = _m_r(o, 5.0)
    single = one[:1]
    for dr in (0.3, 1.2):
        assert tab.fcoll(one, m_r, dr) == pytest.approx(tab.fcoll(single, m_r, dr), rel=1e-14)


def test_flat_feedback_form_is_the_step_function_at_the_cooling_threshold(o):
    # alpha = beta = 0: faint [M(10^4 K), M_F) plus bright [M_F, inf) at the same zeta0 is one
    # population of zeta0 above M(10^4 K), whatever T_F is
    n, box, z = 16, 40.0, 8.5
    d = synth.density_box(n, box, z, seed=9)
    ref = o.ionize(d, box, z, 40.0, 9.0, 4.0)
    got = o.ionize_pops(d, box, z, o.populations(2, (40.0, 9.0, 4.9), (0.0, 0.0, 0.0, 0.0), z), 9.0)
    assert np.array_equal(got["flag"], ref["flag"])
    assert np.abs(got["xhi"] - ref["xhi"]).max() < 1e-7
