"""GPU parity of the mock's total uncertainty (eor_noise_sigma: Sec. 2.4's T+S mode sum and
Sec. 2.5's modelling error) against the FP64 oracle (oracle/noise.py). The thermal noise is
a seeded function of |k_x|, |k_y|, |k_z| (equal for a mode and its conjugate), given to the
oracle on the full grid and to the library in the half-spectrum layout; FP32 noise values
and FP64 sums leave relative differences of order 1e-7."""
import numpy as np
import pytest

from oracle import noise
from paper_1501_06576_gb300 import eor21, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _thermal(n, scale):
    m = np.abs(np.fft.fftfreq(n, d=1.0 / n))
    mx, my, mz = np.meshgrid(m, m, m, indexing="ij")
    return (scale * (mx ** 2 + my ** 2 + 2.0 * mz ** 2) ** 0.75 * (1.0 + 0.1 * np.cos(mx + my))).astype(np.float32)


@pytest.mark.parametrize("n,box", [(32, 60.0), (64, 100.0)])
def test_noise_sigma_matches_oracle(n, box):
    zs = (8.0, 9.0)
    ctx = eor21.Context(n=n, box_mpc=box, z=zs)
    mock = np.stack([np.geomspace(3.0, 60.0, 14) * (1 + 0.1 * j) for j in range(2)])
    full = [_thermal(n, 0.05 * (j + 1)) for j in range(2)]
    half = np.stack([np.ascontiguousarray(np.transpose(f[:, :, : n // 2 + 1], (2, 0, 1))) for f in full])
    for thermal, frac in ((None, 0.0), (half, 0.0), (half, 0.25)):
        sig = ctx.noise_sigma(mock, thermal, frac)
        for j in range(2):
            ref, cnt = noise.total_sigma(n, box, mock[j], None if thermal is None else full[j].astype(np.float64),
                                         frac)
            ok = cnt > 0
            assert np.all(np.isnan(sig[j][~ok]))
            assert np.allclose(sig[j][ok], ref[ok], rtol=1e-6, atol=0), (thermal is None, frac)
    ctx.close()
