"""The tcgen05 TF32 tensor-core path (operand layout, descriptors, tensor-memory reads)
against numpy: D = A B^T for A 128 x 32 and B n x 32."""
import numpy as np
import pytest

from paper_1501_06576_gb300 import eor21

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def tf32(x):
    """Round-to-nearest (ties away) of float32 to 10 mantissa bits, as cvt.rna.tf32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("n", [16, 64, 128, 256])
def test_tensor_core_matches_numpy(torch_cuda, n):
    torch = torch_cuda
    rng = np.random.default_rng(n)
    a = rng.standard_normal((128, 32)).astype(np.float32)
    b = rng.standard_normal((n, 32)).astype(np.float32)
    d, err = eor21.tensor_core_check(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    assert int(err.item()) == 0
    ref = tf32(a).astype(np.float64) @ tf32(b).astype(np.float64).T
    np.testing.assert_allclose(d.cpu().numpy(), ref, atol=1e-4, rtol=1e-4)


def test_tensor_core_layout_is_exact_on_integers(torch_cuda):
    # small integers are exact in TF32 and in FP32 sums: every element checks the mapping
    torch = torch_cuda
    n = 64
    a = (np.arange(128 * 32).reshape(128, 32) % 7 - 3).astype(np.float32)
    b = (np.arange(n * 32).reshape(n, 32) % 5 - 2).astype(np.float32)
    d, err = eor21.tensor_core_check(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    assert int(err.item()) == 0
    np.testing.assert_array_equal(d.cpu().numpy(), a @ b.T)
