"""Pins of the oracle's excursion-set ionization (Eq. 1 and partial ionization, Sec. 2.1),
brightness temperature and power spectrum (Sec. 2.2) and chi^2 (Sec. 2.5): brute force
with direct DFT sums on 8^3, closed forms for uniform and plane-wave boxes, exact
monotonicity, Parseval-type sums, and recovery of the input P(k) from random fields."""
import numpy as np
import pytest
from scipy import special

import oracle
from paper_1501_06576_gb300 import synth


def W(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x > 0
    out[nz] = 3.0 * special.spherical_jn(1, x[nz]) / x[nz]
    return out


def signed(n):
    m = np.arange(n)
    return np.where(m < n // 2, m, m - n)


def kgrid(n, box):
    m = signed(n)
    kf = 2.0 * np.pi / box
    return kf * np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)


# ------------------------------------------------------------------ ladder

@pytest.mark.parametrize("n,box,rmfp,expect", [(128, 250.0, 15.0, 28), (64, 100.0, 15.0, 30)])
def test_ladder_closed_form(n, box, rmfp, expect):
    o = oracle.Oracle()
    radii = o.radius_ladder(n, box, rmfp)
    r_cell = (3.0 / (4.0 * np.pi)) ** (1.0 / 3.0) * box / n
    j = np.arange(len(radii) - 1)
    np.testing.assert_allclose(radii[:-1], rmfp / 1.1 ** j, rtol=1e-13)
    assert radii[-1] == pytest.approx(r_cell, rel=1e-14)
    assert np.all(radii[:-1] > r_cell) and radii[-2] / 1.1 <= r_cell
    assert len(radii) == expect


def test_ladder_degenerate_rmfp_below_cell():
    o = oracle.Oracle()
    radii = o.radius_ladder(64, 100.0, 0.5)
    assert len(radii) == 1 and radii[0] == pytest.approx(0.6203504908994 * 100.0 / 64, rel=1e-12)
    o1 = oracle.Oracle(ion=oracle.IonConfig(r_cell_rule=1))
    assert o1.r_cell(64, 100.0) == pytest.approx(100.0 / 64)


# ------------------------------------------------------------------ filter

def test_filter_identity_as_r_to_zero():
    rng = np.random.default_rng(1)
    d = rng.normal(size=(16, 16, 16)).astype(np.float32)
    out = oracle.Oracle().filter_box(d, 40.0, 1e-9)
    np.testing.assert_allclose(out, d.astype(np.float64), atol=1e-12)


@pytest.mark.parametrize("m0", [(1, 0, 0), (0, 3, 2), (5, -4, 8)])
def test_filter_plane_wave_closed_form(m0):
    n, box, r, a = 16, 40.0, 3.7, 0.8
    x = np.arange(n)
    ph = 2.0 * np.pi * (m0[0] * x[:, None, None] + m0[1] * x[None, :, None] + m0[2] * x[None, None, :]) / n
    d = (a * np.cos(ph)).astype(np.float32)
    k0 = 2.0 * np.pi / box * np.sqrt(sum(v * v for v in m0))
    out = oracle.Oracle().filter_box(d, box, r)
    ref = W(k0 * r) * d.astype(np.float64)
    np.testing.assert_allclose(out, ref, atol=1e-12)


# ------------------------------------------------------------------ ionization

def brute_force_ionize(o, d, box, z, zeta, rmfp, logt):
    """The same method with every transform written as a direct DFT sum."""
    n = d.shape[0]
    f = np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n)
    spec = np.einsum("ia,jb,kc,abc->ijk", f, f, f, d.astype(np.float64))
    g = o.growth(z)
    s2_min = g * g * o.sigma2(o.mass_to_radius(o.mmin(10 ** logt, z)))
    ion = np.zeros(d.shape, bool)
    kk = kgrid(n, box)
    radii = o.radius_ladder(n, box, rmfp)
    conj = np.conj(f)
    margin = np.inf
    for j, r in enumerate(radii):
        dr = np.einsum("ia,jb,kc,abc->ijk", conj, conj, conj, spec * W(kk * r)).real / n ** 3
        s2 = s2_min - g * g * o.sigma2(r)
        if s2 <= 0:
            fcoll = np.zeros_like(dr)
        else:
            fcoll = np.where(dr >= 1.686, 1.0, special.erfc((1.686 - dr) / np.sqrt(2 * s2)))
            margin = min(margin, np.min(np.abs(zeta * fcoll - 1.0)))
        ion |= zeta * fcoll >= 1.0
    xhi = 1.0 - np.where(ion, 1.0, np.minimum(1.0, zeta * fcoll))
    return ion, xhi, margin


@pytest.mark.parametrize("seed,zeta,rmfp,logt", [(1, 30.0, 10.0, 4.48), (2, 25.0, 6.0, 4.9), (3, 12.0, 18.0, 5.2)])
def test_ionize_brute_force_8cube(seed, zeta, rmfp, logt):
    n, box, z = 8, 20.0, 9.0
    rng = np.random.default_rng(seed)
    d = np.maximum(rng.normal(scale=0.6, size=(n, n, n)), -0.99).astype(np.float32)
    o = oracle.Oracle()
    res = o.ionize(d, box, z, zeta, rmfp, logt)
    ion, xhi, margin = brute_force_ionize(o, d, box, z, zeta, rmfp, logt)
    assert margin > 1e-9
    np.testing.assert_array_equal(res["flag"].astype(bool), ion)
    np.testing.assert_allclose(res["xhi"], xhi, atol=1e-10)
    t0 = o.t0_mk(z)
    np.testing.assert_allclose(res["dtb"], t0 * xhi * (1.0 + d.astype(np.float64)), atol=1e-9)
    assert res["xhi_mean"] == pytest.approx(xhi.mean(), abs=1e-12)
    assert 0 < ion.sum() < ion.size     # both outcomes occur


def test_ionize_uniform_box_closed_form():
    n, box, z, zeta, rmfp, logt = 16, 50.0, 9.0, 30.0, 15.0, np.log10(3e4)
    o = oracle.Oracle()
    d = np.zeros((n, n, n), np.float32)
    res = o.ionize(d, box, z, zeta, rmfp, logt)
    g = o.growth(z)
    s2_min = g * g * o.sigma2(o.mass_to_radius(o.mmin(10 ** logt, z)))
    radii = o.radius_ladder(n, box, rmfp)
    f = [special.erfc(1.686 / np.sqrt(2 * (s2_min - g * g * o.sigma2(r)))) for r in radii]
    flagged = any(zeta * v >= 1.0 for v in f)
    x = 0.0 if flagged else 1.0 - min(1.0, zeta * f[-1])
    np.testing.assert_allclose(res["xhi"], x, atol=1e-12)
    assert res["xhi_mean"] == pytest.approx(x, abs=1e-12)


def test_ionize_plane_wave_flags_closed_form():
    n, box, z, zeta, rmfp, logt, a = 32, 80.0, 9.0, 30.0, 12.0, 4.4, 1.2
    x = np.arange(n)
    ph = 2.0 * np.pi * 2 * x / n
    d = np.broadcast_to((a * np.cos(ph))[:, None, None], (n, n, n)).astype(np.float32)
    o = oracle.Oracle()
    res = o.ionize(d, box, z, zeta, rmfp, logt)
    k0 = 2.0 * np.pi / box * 2
    g = o.growth(z)
    s2_min = g * g * o.sigma2(o.mass_to_radius(o.mmin(10 ** logt, z)))
    ion = np.zeros(n, bool)
    for r in o.radius_ladder(n, box, rmfp):
        dr = a * np.cos(ph).astype(np.float32).astype(np.float64) * W(k0 * r)
        s2 = s2_min - g * g * o.sigma2(r)
        fcoll = np.where(dr >= 1.686, 1.0, special.erfc((1.686 - dr) / np.sqrt(2 * s2)))
        ion |= zeta * fcoll >= 1.0
    xhi = 1.0 - np.where(ion, 1.0, np.minimum(1.0, zeta * fcoll))
    np.testing.assert_array_equal(res["flag"][:, 0, 0].astype(bool), ion)
    np.testing.assert_allclose(res["xhi"][:, 5, 7], xhi, atol=1e-9)
    assert 0 < ion.sum() < n


@pytest.fixture(scope="module")
def grf32():
    return synth.density_box(32, 80.0, 9.0, seed=11)


def test_ionize_bounds_and_monotone_in_zeta(grf32):
    o = oracle.Oracle()
    prev = None
    for zeta in [5.0, 20.0, 40.0, 100.0]:
        res = o.ionize(grf32, 80.0, 9.0, zeta, 12.0, 4.5)
        assert np.all(res["xhi"] >= 0.0) and np.all(res["xhi"] <= 1.0)
        if prev is not None:
            assert np.all(res["xhi"] <= prev)      # per cell, exactly
        prev = res["xhi"]
    assert prev.mean() < 0.5


def test_ionize_monotone_in_tvir(grf32):
    o = oracle.Oracle()
    prev = None
    for logt in [4.0, 4.5, 5.0, 5.5]:
        res = o.ionize(grf32, 80.0, 9.0, 30.0, 12.0, logt)
        if prev is not None:
            assert np.all(res["xhi"] >= prev)
        prev = res["xhi"]


# ------------------------------------------------------------------ power spectrum

def test_power_spectrum_plane_wave_single_bin():
    n, box, a = 32, 100.0, 3.0
    m0 = (2, 3, 1)
    x = np.arange(n)
    ph = 2.0 * np.pi * (m0[0] * x[:, None, None] + m0[1] * x[None, :, None] + m0[2] * x[None, None, :]) / n
    box_field = 5.0 + a * np.cos(ph)     # the mean sits at k = 0 and is excluded
    d2, km, cnt = oracle.power_spectrum(box_field, box, 14, 0.1, 1.5)
    k0 = 2.0 * np.pi / box * np.sqrt(sum(v * v for v in m0))
    b0 = int(np.floor(14 * np.log(k0 / 0.1) / np.log(15.0)))
    kk = kgrid(n, box)
    in_bin = (kk >= 0.1 * 15 ** (b0 / 14)) & (kk < 0.1 * 15 ** ((b0 + 1) / 14)) & (kk < 1.5)
    vol = box ** 3
    expect = 2.0 * k0 ** 3 * (a * vol / 2.0) ** 2 / (2.0 * np.pi ** 2 * vol) / in_bin.sum()
    assert cnt[b0] == in_bin.sum()
    assert d2[b0] == pytest.approx(expect, rel=1e-10)
    others = np.delete(d2, b0)
    assert np.all(np.abs(others[np.isfinite(others)]) < 1e-12 * expect)


def test_power_spectrum_matches_numpy_mode_sum():
    n, box = 32, 100.0
    rng = np.random.default_rng(5)
    f = rng.normal(size=(n, n, n))
    d2, km, cnt = oracle.power_spectrum(f, box, 14, 0.1, 1.5)
    x = np.fft.fftn(f) * (box / n) ** 3
    kk = kgrid(n, box)
    p = kk ** 3 * np.abs(x) ** 2 / (2 * np.pi ** 2 * box ** 3)
    edges = 0.1 * 15.0 ** (np.arange(15) / 14)
    for b in range(14):
        sel = (kk >= edges[b]) & (kk < edges[b + 1])
        assert cnt[b] == sel.sum()
        assert d2[b] == pytest.approx(p[sel].mean(), rel=1e-10)
        assert km[b] == pytest.approx(kk[sel].mean(), rel=1e-12)


def test_power_spectrum_recovers_input_pk():
    # mean Delta^2 over seeds of random fields drawn from P(k) agrees with the
    # mode-averaged k^3 P(k) D^2 / (2 pi^2) within cosmic variance (5 sigma)
    n, box, z, seeds = 32, 100.0, 9.0, 12
    cos = synth.InputCosmology()
    g = cos.growth(z)
    acc = np.zeros(14)
    for s in range(seeds):
        d = synth.density_box(n, box, z, seed=1000 + s, cosmo=cos)
        acc += oracle.power_spectrum(d.astype(np.float64), box, 14, 0.1, 1.5)[0]
    acc /= seeds
    kk = kgrid(n, box)
    pk = np.zeros_like(kk)
    pk[kk > 0] = cos.pk(kk[kk > 0]) * g * g
    t = kk ** 3 * pk / (2 * np.pi ** 2)
    edges = 0.1 * 15.0 ** (np.arange(15) / 14)
    for b in range(14):
        sel = (kk >= edges[b]) & (kk < edges[b + 1])
        if sel.sum() == 0:
            continue
        expect = t[sel].mean()
        sd = np.sqrt(2.0 * np.sum(t[sel] ** 2)) / sel.sum() / np.sqrt(seeds)
        assert abs(acc[b] - expect) < 5 * sd + 1e-3 * expect, (b, acc[b], expect, sd)


# ------------------------------------------------------------------ chi^2

def test_chi2_bin_selection_and_unit_terms():
    # geometric centres 0.1*15^((b+0.5)/14) fall in [0.15, 1.0] for b = 2..11 only
    centres = 0.1 * 15.0 ** ((np.arange(14) + 0.5) / 14)
    sel = (centres >= 0.15) & (centres <= 1.0)
    assert list(np.nonzero(sel)[0]) == list(range(2, 12))
    mock = np.linspace(1.0, 14.0, 14)
    sigma = 0.2 * mock
    assert oracle.chi2(mock, None, mock, sigma) == 0.0
    assert oracle.chi2(1.2 * mock, None, mock, sigma) == pytest.approx(10.0, rel=1e-12)
    model = mock.copy()
    model[5] += 3 * sigma[5]
    model[0] += 100.0            # outside the k range: ignored
    assert oracle.chi2(model, None, mock, sigma) == pytest.approx(9.0, rel=1e-12)
    cnt = np.ones(14, np.int64)
    cnt[5] = 0                   # empty bins are skipped
    assert oracle.chi2(model, cnt, mock, sigma) == 0.0
