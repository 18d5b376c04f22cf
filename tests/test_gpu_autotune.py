"""GPU test of the launch-schedule autotuner (eor_autotune): it picks one of its candidates,
leaves the context usable, and the likelihood depends on the schedule only through the FP32
rounding of the spectrum's transforms."""
import numpy as np
import pytest

from paper_1501_06576_gb300 import eor21, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("method", [eor21.EOR_METHOD_BASIS, eor21.EOR_METHOD_DIRECT])
def test_autotune_picks_a_candidate_and_keeps_results(method):
    n, box, zs = 64, 100.0, (9.0, 10.0)
    ctx = eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=8)
    ctx.set_method(method)
    ctx.init_boxes(synth.density_boxes(n, box, zs, seed=8))
    params = synth.walker_params(8, seed=9)
    mock = np.full((2, 14), 20.0)
    sigma = 0.2 * mock
    before, d2_before = ctx.likelihood(params, mock, sigma, want_d2=True)
    g, p, t, ms = ctx.autotune(params, mock, sigma, reps=2)
    assert p in (4, 8, 16, 32) and t == 512 and ms > 0   # 64 only with more than 32 pairs to run
    assert g in ((4, 8, 16) if method == eor21.EOR_METHOD_DIRECT else (8,))
    after, d2_after = ctx.likelihood(params, mock, sigma, want_d2=True)
    # the spectrum's tiling may change with the schedule: the same sums up to FP32 rounding
    assert np.allclose(after, before, rtol=1e-5, atol=0)
    assert np.allclose(d2_after, d2_before, rtol=1e-5, atol=0, equal_nan=True)
    ctx.close()


def test_autotune_device_buffers_and_errors():
    torch = pytest.importorskip("torch")
    ctx = eor21.Context(n=32, box_mpc=60.0, z=(9.0,), max_walkers=4)
    with pytest.raises(eor21.EorError) as ei:
        ctx.autotune(synth.walker_params(4, seed=1), np.ones((1, 14)), np.ones((1, 14)))
    assert ei.value.code == eor21.EOR_ESTATE
    ctx.init_boxes(synth.density_boxes(32, 60.0, (9.0,), seed=3))
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    g, p, t, ms = ctx.autotune(d(synth.walker_params(4, seed=1)), d(np.full((1, 14), 5.0)), d(np.ones((1, 14))))
    assert p in (4, 8, 16, 32)
    with pytest.raises(eor21.EorError) as ei:
        ctx.autotune(synth.walker_params(5, seed=1), np.ones((1, 14)), np.ones((1, 14)))   # > max_walkers
    assert ei.value.code == eor21.EOR_EINVAL
    # the context still works with the restored schedule
    chi = ctx.likelihood(synth.walker_params(4, seed=1), np.full((1, 14), 5.0), np.ones((1, 14)))
    assert np.all(np.isfinite(chi))
    ctx.close()


def test_power_spectrum_plane_tiling_does_not_change_results():
    """At 128^3 the spectrum runs as slab and x-line passes, or as a pencil pass and one CTA
    per plane or a two-CTA cluster per plane (eor_set_ps_split); the spectra agree to the
    FP32 rounding of the transforms, and the autotuner reports the tiling it kept."""
    n, box, zs = 128, 250.0, (9.0,)
    ctx = eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=4)
    ctx.init_boxes(synth.density_boxes(n, box, zs, seed=12))
    params = synth.walker_params(4, seed=13)
    mock = np.full((1, 14), 20.0)
    sigma = 0.2 * mock
    out = {}
    for split in (0, 1, 2):
        ctx.set_ps_split(split)
        assert ctx.get_tuning()["ps_split"] == split
        out[split] = ctx.likelihood(params, mock, sigma, want_d2=True)
    for split in (0, 2):
        np.testing.assert_allclose(out[split][1], out[1][1], rtol=1e-5, equal_nan=True)
        np.testing.assert_allclose(out[split][0], out[1][0], rtol=1e-4)
    # the spectrum's passes on one stream in turn, or overlapped on two: the same kernels and
    # sums (up to the order of the FP64 additions across planes)
    for streams in (1, 2):
        ctx.set_ps_streams(streams)
        assert ctx.get_tuning()["ps_streams"] == streams
        d2 = ctx.likelihood(params, mock, sigma, want_d2=True)[1]
        np.testing.assert_allclose(d2, out[2][1], rtol=1e-12, equal_nan=True)
    ctx.autotune(params, mock, sigma, reps=1)
    assert ctx.get_tuning()["ps_split"] in (0, 1, 2) and ctx.get_tuning()["ps_streams"] in (1, 2)
    ctx.close()
    small = eor21.Context(n=64, box_mpc=100.0, z=zs, max_walkers=1)
    with pytest.raises(eor21.EorError) as ei:
        small.set_ps_split(2)
    assert ei.value.code == eor21.EOR_ENOTSUP
    small.close()


@pytest.mark.parametrize("split", [0, 1])
def test_pairs_in_flight_do_not_change_results(split):
    """36 (walker, redshift) pairs at 32^3 with 1, 4, 16 and 64 pairs per spectrum launch (64:
    the autotuner's largest candidate, one ragged batch): chi^2 and every Delta^2 bin agree up
    to the order of the FP64 additions across CTAs."""
    n, box, zs = 32, 64.0, (8.0, 9.0, 10.0)
    ctx = eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=12)
    ctx.init_boxes(synth.density_boxes(n, box, zs, seed=21))
    params = synth.walker_params(12, seed=22)
    mock = np.full((3, 14), 20.0)
    sigma = 0.2 * mock
    ctx.set_ps_split(split)
    out = {}
    for pairs in (1, 4, 16, 64):
        ctx.set_tuning(8, pairs, 512)
        assert ctx.get_tuning()["pairs"] == pairs and ctx.get_tuning()["ps_split"] == split
        out[pairs] = ctx.likelihood(params, mock, sigma, want_d2=True)
    for pairs in (1, 4, 64):
        np.testing.assert_allclose(out[pairs][0], out[16][0], rtol=1e-12)
        np.testing.assert_allclose(out[pairs][1], out[16][1], rtol=1e-12, equal_nan=True)
    assert np.all(np.isfinite(out[64][0]))
    ctx.close()
