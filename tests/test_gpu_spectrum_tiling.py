"""GPU checks of the power spectrum's tilings: the slab passes (split 0: one CTA per x slab
for the real input and the z and y transforms, then x lines with the shell sums) against the
pencil and plane passes (split 1, and the two-CTA cluster at 128^3) on the same inputs, for
every grid size the slab passes serve and each input form: the flag contraction's flags with
the step-function efficiency and with the mass-dependent one (its x_HI table), and the TF32
contraction's stored delta T_b boxes. x_HI is the same per-cell arithmetic in both passes
(equal to FP32 rounding), the spectra agree to the FP32 rounding of the transforms."""
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


FORMS = [(eor21.EOR_METHOD_BASIS, 0), (eor21.EOR_METHOD_BASIS, 2), (eor21.EOR_METHOD_BASIS_TF32, 0)]
FORM_IDS = ["flags_step_efficiency", "flags_feedback_efficiency", "stored_boxes_tf32"]


def run(ctx, split):
    ctx.set_ps_split(split)
    assert ctx.get_tuning()["ps_split"] == split
    xhi, mean = ctx.run_ionization(want_xhi=True)
    d2, km, cnt = ctx.power_spectrum()
    return xhi, mean, d2, cnt


def close_spectra(a, b):
    scale = np.nanmax(np.abs(b))
    np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(b)
    assert np.all(np.abs(a[ok] - b[ok]) <= 1e-5 * np.abs(b[ok]) + 1e-6 * scale)


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
@pytest.mark.parametrize("n,box", [(16, 30.0), (32, 64.0), (64, 100.0), (128, 250.0)])
def test_slab_passes_match_plane_passes(n, box, form):
    method, model = form
    zs = (8.0, 9.5)
    params = synth.walker_params(3, seed=n + 7)
    with eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=3, efficiency_model=model) as ctx:
        ctx.set_method(method)
        ctx.init_boxes(synth.density_boxes(n, box, zs, seed=n + 3))
        if model:
            ctx.set_efficiency(np.array([[4.0 / 3.0, -1.0 / 3.0, 0.0, 0.0]] * 3))
        ctx.set_params(params)
        ref = run(ctx, 1)
        for split in ((0, 2) if n == 128 else (0,)):
            got = run(ctx, split)
            np.testing.assert_allclose(got[0], ref[0], rtol=0, atol=1e-6)
            np.testing.assert_allclose(got[1], ref[1], rtol=0, atol=1e-7)
            np.testing.assert_array_equal(got[3], ref[3])
            close_spectra(got[2], ref[2])
        assert 0.0 < float(np.mean(ref[1])) < 1.0


@pytest.mark.parametrize("pairs", [1, 4, 5])
@pytest.mark.parametrize("n,box", [(32, 64.0), (128, 250.0)])
def test_slab_pipeline_batches(n, box, pairs):
    """The slab passes over several batches of pairs (the x-line pass of one batch on the
    second stream while the slab pass of the next fills the other half of the intermediate
    buffer), a ragged last batch (7 pairs in batches of 4 or 5) and one pair per batch give the
    same x_HI and spectra as the plane passes."""
    zs = (8.0, 9.0, 10.0, 11.0, 12.0, 13.0, 14.0)[: 7 if n == 32 else 1]
    walkers = 1 if n == 32 else 7
    params = synth.walker_params(walkers, seed=pairs + n)
    with eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=walkers) as ctx:
        ctx.init_boxes(synth.density_boxes(n, box, zs, seed=n + pairs))
        ctx.set_params(params)
        ref = run(ctx, 1)
        ctx.set_tuning(8, pairs, 512)
        got = run(ctx, 0)
    np.testing.assert_allclose(got[0], ref[0], rtol=0, atol=1e-6)
    np.testing.assert_allclose(got[1], ref[1], rtol=0, atol=1e-7)
    np.testing.assert_array_equal(got[3], ref[3])
    close_spectra(got[2], ref[2])


def test_slab_passes_many_bins_and_one_walker():
    """40 bins (more than the per-thread slots of the x-line pass: its shell sums then go
    through shared-memory atomics) and a ragged batch (one pair in flight of 16)."""
    n, box, zs = 32, 64.0, (9.0,)
    with eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=1, n_bins=40) as ctx:
        ctx.init_boxes(synth.density_boxes(n, box, zs, seed=5))
        ctx.set_params(np.array([[30.0, 12.0, 4.6]]))
        ref = run(ctx, 1)
        got = run(ctx, 0)
    np.testing.assert_allclose(got[0], ref[0], rtol=0, atol=1e-6)
    np.testing.assert_array_equal(got[3], ref[3])
    close_spectra(got[2], ref[2])


def test_slab_split_errors():
    with eor21.Context(n=32, box_mpc=64.0, z=(9.0,), max_walkers=1) as ctx:
        for bad in (-1, 3):
            with pytest.raises(eor21.EorError) as ei:
                ctx.set_ps_split(bad)
            assert ei.value.code == eor21.EOR_EINVAL
        with pytest.raises(eor21.EorError) as ei:
            ctx.set_ps_split(2)
        assert ei.value.code == eor21.EOR_ENOTSUP
        assert ctx.get_tuning()["ps_split"] == 0
