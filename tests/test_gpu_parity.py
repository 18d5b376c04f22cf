"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on the same
seeded inputs. Tolerances (from the path's precision split): at most 1e-4 of cells with
a flipped ionization decision (|x_HI difference| > 1e-3), 1e-4 absolute on every other
cell's x_HI, 1e-3 relative per Delta^2 bin; transforms and filters within FP32 rounding
(1e-5 of the field's rms)."""
import numpy as np
import pytest

import oracle
from paper_1501_06576_gb300 import eor21, synth

pytestmark = pytest.mark.gpu

FLIP_TOL = 1e-4
XHI_TOL = 1e-4
PS_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


METHODS = [eor21.EOR_METHOD_BASIS, eor21.EOR_METHOD_DIRECT, eor21.EOR_METHOD_BASIS_SIMT, eor21.EOR_METHOD_BASIS_TF32]
METHOD_IDS = ["basis_fp16_tensor_cores", "direct", "basis_fp32_units", "basis_tf32_tensor_cores"]


def make_ctx(n, box, zs, max_walkers=1, method=eor21.EOR_METHOD_BASIS, **kw):
    ctx = eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=max_walkers, **kw)
    ctx.set_method(method)
    return ctx


def compare_xhi(gpu, ref):
    diff = np.abs(gpu.astype(np.float64) - ref)
    flipped = diff > 1e-3
    frac = flipped.mean()
    rest = diff[~flipped].max() if (~flipped).any() else 0.0
    return frac, rest


def compare_ps(d2, ref, cnt):
    ok = cnt > 0
    rel = np.abs(d2[ok] - ref[ok]) / np.maximum(np.abs(ref[ok]), 1e-30)
    return rel.max()


# ------------------------------------------------------------------ single kernels

@pytest.mark.parametrize("n,box", [(16, 30.0), (32, 60.0), (64, 100.0), (128, 250.0)])
def test_density_spectrum_matches_oracle(n, box):
    delta = synth.density_boxes(n, box, (9.0,), seed=21)
    with make_ctx(n, box, (9.0,)) as ctx:
        ctx.init_boxes(delta)
        got = ctx.density_spectrum(0)                         # [kz][kx][ky]
    ref = oracle.fft3d(delta[0].astype(np.float64), -1)[:, :, : n // 2 + 1].transpose(2, 0, 1)
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(got - ref)) <= 1e-5 * rms


@pytest.mark.parametrize("n,box", [(16, 30.0), (32, 60.0), (64, 100.0), (128, 250.0)])
@pytest.mark.parametrize("r", [0.0, 1.3, 4.0, 15.0])
def test_filtered_density_matches_oracle(n, box, r):
    delta = synth.density_boxes(n, box, (9.0,), seed=22)
    with make_ctx(n, box, (9.0,)) as ctx:
        ctx.init_boxes(delta)
        got = ctx.filtered_density(0, r)
    ref = oracle.Oracle().filter_box(delta[0], box, r if r > 0 else 1e-12)
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(np.std(ref), 1e-3)


def test_box_power_spectrum_matches_oracle():
    n, box = 64, 100.0
    rng = np.random.default_rng(3)
    field = (20.0 * (1.0 + 0.5 * rng.standard_normal((n, n, n)))).astype(np.float32)
    with make_ctx(n, box, (9.0,)) as ctx:
        d2, km, cnt = ctx.box_power_spectrum(field)
    rd2, rkm, rcnt = oracle.power_spectrum(field.astype(np.float64), box, 14, 0.1, 1.5)
    np.testing.assert_array_equal(cnt, rcnt)
    np.testing.assert_allclose(km, rkm, rtol=1e-12)
    assert compare_ps(d2, rd2, rcnt) <= 1e-5


# ------------------------------------------------------------------ ladder and ionization

def test_walker_ladder_bitwise():
    n, box = 64, 100.0
    params = np.array([[30.0, 15.0, 4.48], [50.0, 5.123456789, 5.0], [10.0, 0.5, 4.0], [20.0, 19.99, 4.2]])
    delta = synth.density_boxes(n, box, (9.0,), seed=1)
    orc = oracle.Oracle()
    with make_ctx(n, box, (9.0,), max_walkers=4) as ctx:
        ctx.init_boxes(delta)
        ctx.set_params(params)
        for w in range(4):
            got = ctx.walker_ladder(w)
            ref = orc.radius_ladder(n, box, params[w, 1])
            assert got.tolist() == ref.tolist()


@pytest.fixture(scope="module", params=METHODS, ids=METHOD_IDS)
def cfg1(request):
    """64^3, L = 100 Mpc, z = 9, zeta = 30, R_mfp = 15 Mpc, T_vir = 3e4 K; mock from seed + 1."""
    n, box, zs = 64, 100.0, (9.0,)
    params = np.array([[30.0, 15.0, np.log10(3e4)]])
    delta = synth.density_boxes(n, box, zs, seed=2024)
    mock_delta = synth.density_boxes(n, box, zs, seed=2025)
    orc = oracle.Oracle()
    ref = orc.ionize(delta[0], box, zs[0], *params[0])
    rd2, rkm, rcnt = oracle.power_spectrum(ref["dtb"], box, 14, 0.1, 1.5)
    mref = orc.ionize(mock_delta[0], box, zs[0], *params[0])
    mock = oracle.power_spectrum(mref["dtb"], box, 14, 0.1, 1.5)[0]
    sigma = 0.2 * mock
    with make_ctx(n, box, zs, method=request.param) as ctx:
        ctx.init_boxes(delta)
        ctx.set_params(params)
        xhi, xmean = ctx.run_ionization(want_xhi=True)
        d2, km, cnt = ctx.power_spectrum()
        chi2 = ctx.chi2(mock[None], sigma[None])
    return dict(n=n, box=box, delta=delta, params=params, ref=ref, rd2=rd2, rcnt=rcnt, rkm=rkm, mock=mock,
                sigma=sigma, xhi=xhi, xmean=xmean, d2=d2, km=km, cnt=cnt, chi2=chi2)


def test_cfg1_ionization_matches_oracle(cfg1):
    frac, rest = compare_xhi(cfg1["xhi"][0, 0], cfg1["ref"]["xhi"])
    print(f"cfg1: flipped {frac:.2e}, max |dx_HI| elsewhere {rest:.2e}")
    assert frac <= FLIP_TOL
    assert rest <= XHI_TOL
    assert abs(cfg1["xmean"][0, 0] - cfg1["ref"]["xhi_mean"]) <= 2e-4
    assert 0.05 < cfg1["ref"]["xhi_mean"] < 0.95     # a mixed, non-degenerate box


def test_cfg1_power_spectrum_matches_oracle(cfg1):
    np.testing.assert_array_equal(cfg1["cnt"][0, 0], cfg1["rcnt"])
    np.testing.assert_allclose(cfg1["km"][0, 0], cfg1["rkm"], rtol=1e-12)
    rel = compare_ps(cfg1["d2"][0, 0], cfg1["rd2"], cfg1["rcnt"])
    print(f"cfg1: max relative Delta^2 error {rel:.2e}")
    assert rel <= PS_TOL


def test_cfg1_chi2(cfg1):
    # the chi^2 kernel on the GPU's spectra equals the definition evaluated on them
    mine = oracle.chi2(cfg1["d2"][0, 0], cfg1["cnt"][0, 0], cfg1["mock"], cfg1["sigma"])
    assert cfg1["chi2"][0] == pytest.approx(mine, rel=1e-12)
    full = oracle.chi2(cfg1["rd2"], cfg1["rcnt"], cfg1["mock"], cfg1["sigma"])
    print(f"cfg1: chi2 gpu {cfg1['chi2'][0]:.6g} oracle {full:.6g}")
    assert cfg1["chi2"][0] == pytest.approx(full, rel=5e-3)


@pytest.mark.parametrize("method", METHODS, ids=METHOD_IDS)
def test_multi_walker_multi_z_edge_cases(method):
    """3 redshifts x 6 walkers (ragged against the in-flight pair count), including a
    ladder of one radius (R_mfp < R_cell), zeta < 1 (nothing flagged), a T_vir whose M_min
    exceeds the mass of the smallest spheres, and a ladder of 39 radii (R_mfp = 45 Mpc: its
    radii above R_cell span two column groups of the tensor-core contraction). Tolerances
    are the method's: at most 1e-4 of the cells flipped (at 32^3 one cell is 3e-5), x_HI
    within 1e-4 elsewhere, Delta^2 within 1e-3 per bin: end to end where no cell flipped,
    else against the oracle's spectrum of the GPU's own x_HI (a single flipped cell moves a
    32^3 bin of a few modes by about 1e-2)."""
    n, box, zs = 32, 64.0, (8.0, 9.0, 10.0)
    params = np.array([[30.0, 12.0, 4.5], [80.0, 20.0, 4.0], [25.0, 1.0, 4.7], [0.9, 10.0, 4.3],
                       [40.0, 15.0, 6.6], [20.0, 45.0, 4.6]])
    delta = synth.density_boxes(n, box, zs, seed=77)
    orc = oracle.Oracle()
    with make_ctx(n, box, zs, max_walkers=len(params), method=method, r_mfp_max=50.0) as ctx:
        ctx.init_boxes(delta)
        ctx.set_params(params)
        assert len(ctx.walker_ladder(5)) == 39
        xhi, xmean = ctx.run_ionization(want_xhi=True)
        d2, km, cnt = ctx.power_spectrum()
    for w in range(len(params)):
        for j, z in enumerate(zs):
            ref = orc.ionize(delta[j], box, z, *params[w])
            frac, rest = compare_xhi(xhi[w, j], ref["xhi"])
            assert frac <= FLIP_TOL and rest <= XHI_TOL, (w, j, frac, rest)
            if frac > 0:   # the spectrum stage alone: the oracle's spectrum of the GPU's field
                own = orc.t0_mk(z) * xhi[w, j].astype(np.float64) * (1.0 + delta[j].astype(np.float64))
                rd2, _, rcnt = oracle.power_spectrum(own, box, 14, 0.1, 1.5)
            else:
                rd2, _, rcnt = oracle.power_spectrum(ref["dtb"], box, 14, 0.1, 1.5)
            if ref["xhi_mean"] > 0.01:
                assert compare_ps(d2[w, j], rd2, rcnt) <= PS_TOL, (w, j)
            else:
                assert np.nanmax(np.abs(d2[w, j] - rd2)) <= 1e-3 * max(np.nanmax(np.abs(rd2)), 1e-6)


@pytest.mark.parametrize("method", METHODS, ids=METHOD_IDS)
def test_batched_likelihood_equals_plain_calls(method):
    n, box, zs = 32, 64.0, (8.0, 9.0)
    params = synth.walker_params(5, seed=9)
    delta = synth.density_boxes(n, box, zs, seed=10)
    mock = np.full((2, 14), 5.0)
    sigma = 0.2 * mock
    with make_ctx(n, box, zs, max_walkers=5, method=method) as ctx:
        ctx.init_boxes(delta)
        chi2_b, d2_b = ctx.likelihood(params, mock, sigma, want_d2=True)
        chi2_b2 = ctx.likelihood(params, mock, sigma)            # graph replay
        plain = []
        for w in range(5):
            ctx.set_params(params[w:w + 1])
            ctx.run_ionization()
            d2, _, _ = ctx.power_spectrum()
            plain.append((ctx.chi2(mock, sigma)[0], d2[0]))
    for w in range(5):
        assert chi2_b[w] == pytest.approx(plain[w][0], rel=1e-12)
        np.testing.assert_allclose(d2_b[w], plain[w][1], rtol=1e-12)
    np.testing.assert_allclose(chi2_b2, chi2_b, rtol=1e-12)


def test_errors_and_call_order():
    n, box = 16, 30.0
    with make_ctx(n, box, (9.0,), max_walkers=2, r_mfp_max=10.0) as ctx:
        with pytest.raises(eor21.EorError) as e:
            ctx.set_params(np.array([[30.0, 5.0, 4.5]]))
        assert e.value.code == eor21.EOR_ESTATE
        ctx.init_boxes(synth.density_boxes(n, box, (9.0,), seed=1))
        for bad in ([0.0, 5.0, 4.5], [30.0, 11.0, 4.5], [np.nan, 5.0, 4.5], [30.0, -1.0, 4.5]):
            with pytest.raises(eor21.EorError) as e:
                ctx.set_params(np.array([bad]))
            assert e.value.code == eor21.EOR_EINVAL
        with pytest.raises(eor21.EorError) as e:
            ctx.set_params(np.ones((3, 3)))
        assert e.value.code == eor21.EOR_EINVAL
        with pytest.raises(eor21.EorError) as e:
            ctx.run_ionization()
        assert e.value.code == eor21.EOR_ESTATE
        ctx.set_params(np.array([[30.0, 5.0, 4.5]]))        # still usable after errors
        _, m = ctx.run_ionization()
        assert 0.0 <= m[0, 0] <= 1.0


def test_device_pointers_and_torch_allocator():
    import torch
    n, box, zs = 32, 64.0, (9.0,)
    delta = synth.density_boxes(n, box, zs, seed=3)
    params = np.array([[30.0, 12.0, 4.5]])
    with make_ctx(n, box, zs) as ctx:
        ctx.init_boxes(delta)
        ctx.set_params(params)
        ref_xhi, ref_mean = ctx.run_ionization(want_xhi=True)
    with eor21.Context(n=n, box_mpc=box, z=zs, torch_allocator=True) as ctx:
        ctx.init_boxes(torch.from_numpy(delta).cuda())
        ctx.set_params(torch.from_numpy(params).cuda())
        xhi, mean = ctx.run_ionization(want_xhi=True, device=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(xhi.cpu().numpy(), ref_xhi)
        np.testing.assert_array_equal(mean.cpu().numpy(), ref_mean)


# ------------------------------------------------------------------ full size

@pytest.mark.parametrize("method", METHODS, ids=METHOD_IDS)
def test_full_size_128cube_one_redshift(method):
    """128^3, L = 250 Mpc, z = 9 box of the three-redshift workload, fiducial walker."""
    n, box, zs = 128, 250.0, (8.0, 9.0, 10.0)
    delta = synth.density_boxes(n, box, zs, seed=1)
    params = np.array([[30.0, 15.0, 4.7]])
    with make_ctx(n, box, zs, method=method) as ctx:
        ctx.init_boxes(delta)
        ctx.set_params(params)
        xhi, xmean = ctx.run_ionization(want_xhi=True)
        d2, km, cnt = ctx.power_spectrum()
    orc = oracle.Oracle()
    ref = orc.ionize(delta[1], box, zs[1], *params[0])
    frac, rest = compare_xhi(xhi[0, 1], ref["xhi"])
    print(f"128^3 z=9: flipped {frac:.2e}, max |dx_HI| elsewhere {rest:.2e}")
    assert frac <= FLIP_TOL and rest <= XHI_TOL
    rd2, _, rcnt = oracle.power_spectrum(ref["dtb"], box, 14, 0.1, 1.5)
    assert compare_ps(d2[0, 1], rd2, rcnt) <= PS_TOL


def test_full_size_batched_walkers_sampled():
    """Walkers of the 128-walker prior draw through the batched likelihood call; three of
    them checked against the oracle at z = 8 (the oracle runs one box per walker here)."""
    n, box, zs = 128, 250.0, (8.0, 9.0, 10.0)
    delta = synth.density_boxes(n, box, zs, seed=1)
    params = synth.walker_params(128, seed=3)
    mock = np.full((3, 14), 10.0)
    with make_ctx(n, box, zs, max_walkers=128) as ctx:
        ctx.init_boxes(delta)
        chi2, d2 = ctx.likelihood(params, mock, 0.2 * mock, want_d2=True)
    assert np.all(np.isfinite(chi2))
    orc = oracle.Oracle()
    for w in (0, 57, 127):
        ref = orc.ionize(delta[0], box, zs[0], *params[w])
        rd2, _, rcnt = oracle.power_spectrum(ref["dtb"], box, 14, 0.1, 1.5)
        if ref["xhi_mean"] > 0.01:
            assert compare_ps(d2[w, 0], rd2, rcnt) <= PS_TOL, w
        else:
            assert np.max(np.abs(d2[w, 0] - rd2)) <= 1e-3 * max(np.max(np.abs(rd2)), 1e-6), w


def test_tracing_counts_and_times_every_launch():
    n, box, zs = 32, 64.0, (8.0, 9.0)
    params = synth.walker_params(3, seed=4)
    mock = np.full((2, 14), 5.0)
    with make_ctx(n, box, zs, max_walkers=3) as ctx:
        ctx.init_boxes(synth.density_boxes(n, box, zs, seed=5))
        ref = ctx.likelihood(params, mock, 0.2 * mock)
        untraced = ctx.launch_count()
        ctx.trace(True)
        for _ in range(2):                                   # capture, then a replay
            got = ctx.likelihood(params, mock, 0.2 * mock)
            t = ctx.trace_read()
            assert sum(c for _, c in t.values()) == ctx.launch_count() == untraced
            assert t["basis_ionize"][1] > 0 and t["ps_plane"][1] > 0
            assert all(ms > 0 for ms, c in t.values() if c > 0)
        np.testing.assert_allclose(got, ref, rtol=1e-12)
        ctx.set_method(eor21.EOR_METHOD_DIRECT)
        ctx.set_params(params)                               # traced outside a graph
        ctx.run_ionization()
        t = ctx.trace_read()
        assert t["filter_plane"][1] > 0 and t["filter_plane"][0] > 0
        assert t["pencil_ionize"][1] == t["filter_plane"][1]


@pytest.mark.parametrize("n,box", [(16, 30.0), (32, 60.0), (64, 100.0), (128, 250.0)])
def test_filter_basis_reproduces_tophat(n, box):
    """The library's basis reconstruction sum_b c_b(R) phi_b(k) equals the top-hat window
    W(kR) = 3 j1(kR)/(kR) (scipy's spherical Bessel function, not the library's own table)
    on every |k| of the grid, at the radii of the ladders from R_mfp = 5 .. 20 Mpc and at
    random radii in between, to the basis's 1e-6 tolerance (plus the coefficient table's
    interpolation)."""
    from scipy import special
    with make_ctx(n, box, (9.0,)) as ctx:
        rank, resid = ctx.basis_info()
        assert 4 <= rank <= 48 and resid <= 1e-6
        kf = 2.0 * np.pi / box
        m2 = np.arange(3 * (n // 2) ** 2 + 1, dtype=np.float64)
        r_cell = (3.0 / (4.0 * np.pi)) ** (1.0 / 3.0) * box / n
        radii = [r_cell, 20.0]
        for r_mfp in (5.0, 10.0, 15.0, 20.0):
            r = r_mfp
            while r > r_cell:
                radii.append(r)
                r /= 1.1
        radii += list(np.random.default_rng(n).uniform(r_cell, 20.0, 16))
        worst = 0.0
        for r in radii:
            w = ctx.basis_window(r)
            present = ~np.isnan(w)
            assert present[0] and present.sum() > n        # k = 0 and the shells of the grid
            x = kf * np.sqrt(m2[present]) * r
            ref = np.where(x > 0, 3.0 * special.spherical_jn(1, np.maximum(x, 1e-300)) / np.maximum(x, 1e-300), 1.0)
            worst = max(worst, float(np.max(np.abs(w[present] - ref))))
    print(f"n={n} L={box}: basis rank {rank}, stated residual {resid:.1e}, max |W - basis| {worst:.1e} "
          f"over {len(radii)} radii")
    assert worst <= 2e-6


def test_basis_window_rejects_radii_outside_its_range():
    with make_ctx(32, 60.0, (9.0,)) as ctx:
        for r in (0.1, 25.0, float("nan")):
            with pytest.raises(eor21.EorError) as e:
                ctx.basis_window(r)
            assert e.value.code == eor21.EOR_EINVAL


@pytest.mark.parametrize("method", [eor21.EOR_METHOD_BASIS, eor21.EOR_METHOD_BASIS_SIMT, eor21.EOR_METHOD_BASIS_TF32],
                         ids=["basis_fp16_tensor_cores", "basis_fp32_units", "basis_tf32_tensor_cores"])
def test_basis_and_direct_methods_agree(method):
    n, box, zs = 64, 100.0, (8.0, 9.5)
    params = synth.walker_params(6, seed=12)
    delta = synth.density_boxes(n, box, zs, seed=13)
    out = {}
    for m in (method, eor21.EOR_METHOD_DIRECT):
        with make_ctx(n, box, zs, max_walkers=6, method=m) as ctx:
            ctx.init_boxes(delta)
            ctx.set_params(params)
            xhi, xm = ctx.run_ionization(want_xhi=True)
            d2, _, cnt = ctx.power_spectrum()
            out[m] = (xhi, xm, d2, cnt)
    a, b = out[method], out[eor21.EOR_METHOD_DIRECT]
    frac, rest = compare_xhi(a[0], b[0].astype(np.float64))
    assert frac <= FLIP_TOL and rest <= XHI_TOL
    np.testing.assert_allclose(a[1], b[1], atol=2e-4)
    for w in range(6):
        for j in range(2):
            if b[1][w, j] > 0.01:
                assert compare_ps(a[2][w, j], b[2][w, j], b[3][w, j]) <= PS_TOL
