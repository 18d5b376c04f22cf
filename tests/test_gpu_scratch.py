"""GPU check of the direct method's scratch: its group x pairs half spectra are held only while
EOR_METHOD_DIRECT is chosen (eor_set_method and eor_set_tuning size them), and switching
methods back and forth leaves the likelihood unchanged."""
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


def test_direct_method_scratch_follows_the_method():
    import torch
    n, box, zs = 64, 100.0, (9.0,)
    nspec_bytes = (n // 2 + 1) * n * n * 8
    group, pairs = 8, 16
    direct_bytes = group * pairs * nspec_bytes                       # 138 MB at 64^3
    params = synth.walker_params(4, seed=31)
    mock = np.full((1, 14), 20.0)
    with eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=4) as ctx:
        ctx.init_boxes(synth.density_boxes(n, box, zs, seed=32))
        ctx.set_tuning(group, pairs, 512)
        basis = ctx.likelihood(params, mock, 0.2 * mock, want_d2=True)
        torch.cuda.synchronize()
        free_basis = torch.cuda.mem_get_info()[0]
        ctx.set_method(eor21.EOR_METHOD_DIRECT)
        free_direct = torch.cuda.mem_get_info()[0]
        direct = ctx.likelihood(params, mock, 0.2 * mock, want_d2=True)
        # the direct method's scratch is allocated on the switch (page-granular readings)
        assert free_basis - free_direct >= direct_bytes - (8 << 20)
        ctx.set_tuning(group, 4, 512)                                 # resized for the method
        assert torch.cuda.mem_get_info()[0] - free_direct >= group * 12 * nspec_bytes - (8 << 20)
        direct4 = ctx.likelihood(params, mock, 0.2 * mock, want_d2=True)
        ctx.set_method(eor21.EOR_METHOD_BASIS)
        # released again (the basis state at 4 pairs holds less than at 16)
        assert torch.cuda.mem_get_info()[0] >= free_basis - (8 << 20)
        again = ctx.likelihood(params, mock, 0.2 * mock, want_d2=True)
    for got, ref in ((direct4, direct), (again, basis)):   # pairs in flight change no result
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
        np.testing.assert_allclose(got[1], ref[1], rtol=1e-12, equal_nan=True)
    # the two methods agree to the parity tolerance per bin
    np.testing.assert_allclose(direct[1], basis[1], rtol=1e-3, equal_nan=True)
