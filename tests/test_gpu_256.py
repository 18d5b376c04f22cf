"""GPU checks of the 256^3 grid (the two-population workload's, L = 500 Mpc: 1.95 Mpc cells),
where every plane pass runs as a row pass and a column pass: transforms and filters against
the FP64 oracle, one excursion-set realization with the step-function efficiency cell by
cell against the oracle, and the two-population model (Sec. 5's feedback form) end to end,
every cell and every Delta^2 bin against the oracle's own realization (its own FP64 filtered
fields, crossings and partial ionization; about 5 minutes of host time)."""
import numpy as np
import pytest

import oracle
from paper_1501_06576_gb300 import eor21, synth

pytestmark = pytest.mark.gpu

N, BOX = 256, 500.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def box9():
    return synth.density_boxes(N, BOX, (9.0,), seed=61)


def test_transforms_256(box9):
    with eor21.Context(n=N, box_mpc=BOX, z=(9.0,), max_walkers=1) as ctx:
        ctx.init_boxes(box9)
        spec = ctx.density_spectrum(0)                 # [kz][kx][ky]
        filt = ctx.filtered_density(0, 4.0)
        d2, km, cnt = ctx.box_power_spectrum(box9[0])
    ref = oracle.fft3d(box9[0].astype(np.float64), -1)[:, :, : N // 2 + 1].transpose(2, 0, 1)
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(spec - ref)) <= 1e-5 * rms
    del ref, spec
    rf = oracle.Oracle().filter_box(box9[0], BOX, 4.0)
    assert np.max(np.abs(filt - rf)) <= 1e-5 * np.std(rf)
    rd2, rkm, rcnt = oracle.power_spectrum(box9[0].astype(np.float64), BOX)
    assert np.array_equal(cnt, rcnt)
    ok = rcnt > 0
    assert np.max(np.abs(d2[ok] - rd2[ok]) / rd2[ok]) <= 1e-4


STEP_PARAMS = (30.0, 5.0, 4.7)


@pytest.fixture(scope="module")
def step_ref(box9):
    return oracle.Oracle().ionize(box9[0], BOX, 9.0, *STEP_PARAMS)


@pytest.mark.parametrize("method", [eor21.EOR_METHOD_BASIS, eor21.EOR_METHOD_DIRECT, eor21.EOR_METHOD_BASIS_TF32],
                         ids=["basis_fp16_tensor_cores", "direct", "basis_tf32_tensor_cores"])
def test_step_efficiency_256_matches_oracle(box9, step_ref, method):
    params = np.array([STEP_PARAMS])
    with eor21.Context(n=N, box_mpc=BOX, z=(9.0,), max_walkers=1) as ctx:
        ctx.set_method(method)
        ctx.init_boxes(box9)
        ctx.set_params(params)
        xhi, mean = ctx.run_ionization(want_xhi=True)
        d2, _, cnt = ctx.power_spectrum()
    ref = step_ref
    diff = np.abs(xhi[0, 0].astype(np.float64) - ref["xhi"])
    flipped = diff > 1e-3
    assert flipped.mean() <= 1e-4
    assert diff[~flipped].max() <= 1e-4
    rd2, _, rcnt = oracle.power_spectrum(ref["dtb"], BOX)
    ok = rcnt > 0
    assert np.array_equal(cnt[0, 0], rcnt)
    assert np.max(np.abs(d2[0, 0][ok] - rd2[ok]) / rd2[ok]) <= 1e-3


def test_two_populations_256_end_to_end(box9):
    # Sec. 5's fiducial feedback efficiency (zeta0 = 70, T_F = 10^4.7 K, alpha = 4/3,
    # beta = -1/3), R_mfp = 6 Mpc, z = 9: every cell's x_HI and every Delta^2 bin against the
    # oracle, at the tolerances the method is held to
    p, q, z = (70.0, 6.0, 4.7), (4.0 / 3.0, -1.0 / 3.0, 0.0, 0.0), 9.0
    with eor21.Context(n=N, box_mpc=BOX, z=(z,), max_walkers=1, efficiency_model=2) as ctx:
        ctx.init_boxes(box9)
        ctx.set_efficiency(np.array([q]))
        ctx.set_params(np.array([p]))
        xhi, mean = ctx.run_ionization(want_xhi=True)
        d2, _, cnt = ctx.power_spectrum()
    o = oracle.Oracle()
    ref = o.ionize_pops(box9[0], BOX, z, o.populations(2, p, q, z), p[1])
    diff = np.abs(xhi[0, 0].astype(np.float64) - ref["xhi"])
    flipped = diff > 1e-3
    print(f"two populations 256^3: flipped {flipped.mean():.2e} ({int(flipped.sum())} cells), "
          f"max |dx_HI| elsewhere {diff[~flipped].max():.2e}, x_HI mean {mean[0, 0]:.4f} vs {ref['xhi_mean']:.4f}")
    assert flipped.mean() <= 1e-4
    assert diff[~flipped].max() <= 1e-4
    assert abs(mean[0, 0] - ref["xhi_mean"]) <= 1e-4
    rd2, _, rcnt = oracle.power_spectrum(ref["dtb"], BOX)
    ok = rcnt > 0
    assert np.array_equal(cnt[0, 0], rcnt)
    assert np.max(np.abs(d2[0, 0][ok] - rd2[ok]) / rd2[ok]) <= 1e-3


def test_two_populations_256_slope_zero_is_step_function(box9):
    params = np.array([[30.0, 5.0, 4.7]])
    with eor21.Context(n=N, box_mpc=BOX, z=(9.0,), max_walkers=1) as ctx:
        ctx.init_boxes(box9)
        ctx.set_params(params)
        x0, m0 = ctx.run_ionization(want_xhi=True)
    with eor21.Context(n=N, box_mpc=BOX, z=(9.0,), max_walkers=1, efficiency_model=1) as ctx:
        ctx.init_boxes(box9)
        ctx.set_efficiency(np.array([[0.0, 0.0, 0.0, 5.0]]))
        ctx.set_params(params)
        x1, m1 = ctx.run_ionization(want_xhi=True)
    assert (np.abs(x0 - x1) > 1e-3).mean() <= 1e-4
    assert abs(m0[0, 0] - m1[0, 0]) <= 1e-4
