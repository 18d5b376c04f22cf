"""GPU parity of the Zel'dovich evolution of the density boxes (`zeldovich` in eor_config,
Sec. 2.1) against the FP64 oracle (oracle/zeldovich.py): the evolved box within 2e-4 (FP32
displacements of a few cells and FP32 positions leave about 1e-5 in the CIC weights), mass
conserved, and the likelihood on the evolved boxes against the oracle's ionization of the
oracle's evolved box at the parity tolerances of the other tests."""
import numpy as np
import pytest

import oracle
from oracle import zeldovich as zel
from paper_1501_06576_gb300 import eor21, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("n,box", [(32, 60.0), (64, 100.0)])
def test_evolved_box_matches_oracle(n, box):
    zs = (8.0, 10.0)
    lin = synth.density_boxes(n, box, zs, seed=12)
    ctx = eor21.Context(n=n, box_mpc=box, z=zs, zeldovich=1)
    ctx.init_boxes(lin)
    for j in range(2):
        got = ctx.density_box(j).astype(np.float64)
        ref = zel.evolve(lin[j].astype(np.float64), box)
        assert np.abs(got - ref).max() < 2e-4, np.abs(got - ref).max()
        assert np.sum(1.0 + got) == pytest.approx(n ** 3, rel=1e-5)
        assert np.abs(got - lin[j]).max() > 1e-2   # the evolution moved the field
    ctx.close()


def test_likelihood_on_evolved_boxes():
    n, box, zs = 64, 100.0, (9.0,)
    params = np.array([[30.0, 15.0, np.log10(3e4)], [60.0, 8.0, 4.3]])
    lin = synth.density_boxes(n, box, zs, seed=13)
    ctx = eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=2, zeldovich=1)
    ctx.init_boxes(lin)
    ctx.set_params(params)
    xhi, _ = ctx.run_ionization(want_xhi=True)
    d2, _, cnt = ctx.power_spectrum()
    evolved = zel.evolve(lin[0].astype(np.float64), box).astype(np.float32)
    orc = oracle.Oracle()
    for w in range(2):
        ref = orc.ionize(evolved, box, zs[0], *params[w])
        flipped = np.mean(np.abs(xhi[w, 0] - ref["xhi"]) > 1e-3)
        assert flipped <= 1e-4, flipped
        rd2, _, rcnt = oracle.power_spectrum(ref["dtb"], box, 14, 0.1, 1.5)
        ok = rcnt > 0
        rel = np.abs(d2[w, 0][ok] - rd2[ok]) / np.abs(rd2[ok])
        assert rel.max() < 1e-3, rel.max()
    ctx.close()
