"""GPU parity of the velocity-gradient factor of delta T_b (Sec. 2.2, `rsd` in eor_config)
against the FP64 oracle: Delta^2 within 1e-3 per bin (the power-spectrum tolerance of the
other parity tests), x_HI unchanged by the factor, and the factor's effect on the spectrum
larger than that tolerance (so the test sees it)."""
import numpy as np
import pytest

import oracle
from paper_1501_06576_gb300 import eor21, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("method", [eor21.EOR_METHOD_BASIS, eor21.EOR_METHOD_DIRECT])
@pytest.mark.parametrize("max_dvdr", [0.2, 0.02])
def test_velocity_factor_spectrum_matches_oracle(method, max_dvdr):
    n, box, zs = 64, 100.0, (9.0,)
    params = np.array([[30.0, 15.0, np.log10(3e4)], [60.0, 8.0, 4.3]])
    delta = synth.density_boxes(n, box, zs, seed=7)
    ctx = eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=2, rsd=1, rsd_max_dvdr=max_dvdr)
    ctx.set_method(method)
    ctx.init_boxes(delta)
    ctx.set_params(params)
    xhi, _ = ctx.run_ionization(want_xhi=True)
    d2, _, cnt = ctx.power_spectrum()
    plain = eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=2)
    plain.set_method(method)
    plain.init_boxes(delta)
    plain.set_params(params)
    xhi0, _ = plain.run_ionization(want_xhi=True)
    d2_0, _, _ = plain.power_spectrum()
    orc = oracle.Oracle()
    for w in range(2):
        ref = orc.ionize(delta[0], box, zs[0], *params[w], rsd_max_dvdr=max_dvdr)
        rd2, _, rcnt = oracle.power_spectrum(ref["dtb"], box, 14, 0.1, 1.5)
        ok = rcnt > 0
        assert np.array_equal(cnt[w, 0], rcnt)
        rel = np.abs(d2[w, 0][ok] - rd2[ok]) / np.abs(rd2[ok])
        assert rel.max() < 1e-3, rel.max()
        # the ionization field does not depend on the factor
        assert np.array_equal(xhi[w, 0], xhi0[w, 0])
        effect = np.abs(d2[w, 0][ok] / d2_0[w, 0][ok] - 1.0).max()
        assert effect > 1e-2, effect
    ctx.close()
    plain.close()


def test_velocity_factor_config_errors():
    with pytest.raises(eor21.EorError):
        eor21.Context(n=32, box_mpc=60.0, z=(9.0,), rsd=2)
    with pytest.raises(eor21.EorError):
        eor21.Context(n=32, box_mpc=60.0, z=(9.0,), rsd=1, rsd_max_dvdr=1.5)
