"""The Python wrapper of the allocation-free power spectrum refuses tensors that the C entry
point would misread (it sees raw device pointers, so only the wrapper can check dtype,
element count and device). CPU-only: the tensors are stand-ins that report themselves as
CUDA tensors, so every rejection is exercised without a GPU."""
import types

import pytest

torch = pytest.importorskip("torch")

from paper_1501_06576_gb300 import eor21


class FakeCuda:
    def __init__(self, dtype, numel, device=0, contiguous=True, cuda=True):
        self.dtype, self._numel, self._contig, self.is_cuda = dtype, numel, contiguous, cuda
        self.device = types.SimpleNamespace(index=device)

    def numel(self):
        return self._numel

    def is_contiguous(self):
        return self._contig


N, BINS = 32, 14


def good():
    return dict(box=FakeCuda(torch.float32, N ** 3), d2=FakeCuda(torch.float64, BINS),
                nmodes=FakeCuda(torch.int64, BINS))


def check(**over):
    a = good()
    a.update(over)
    eor21.check_noalloc_tensors(N, BINS, a["box"], a["d2"], a["nmodes"], device=0)


def test_accepts_matching_tensors():
    check()
    check(nmodes=None)
    check(d2=FakeCuda(torch.float64, BINS + 5))          # longer outputs are fine


@pytest.mark.parametrize("over,words", [
    (dict(box=FakeCuda(torch.float32, N ** 3, cuda=False)), "CUDA"),
    (dict(box=FakeCuda(torch.float32, N ** 3, contiguous=False)), "contiguous"),
    (dict(box=FakeCuda(torch.float64, N ** 3)), "float32"),
    (dict(box=FakeCuda(torch.float32, 16 ** 3)), "elements"),         # a 16^3 box passed with n = 32
    (dict(box=FakeCuda(torch.float32, 64 ** 3)), "elements"),
    (dict(d2=FakeCuda(torch.float32, BINS)), "float64"),
    (dict(d2=FakeCuda(torch.float64, BINS - 1)), "elements"),
    (dict(nmodes=FakeCuda(torch.int32, BINS)), "int64"),
    (dict(nmodes=FakeCuda(torch.int64, 3)), "elements"),
    (dict(box=FakeCuda(torch.float32, N ** 3, device=1)), "current device"),
    (dict(d2=FakeCuda(torch.float64, BINS, device=1)), "current device"),
    (dict(nmodes=FakeCuda(torch.int64, BINS, device=2)), "current device"),
])
def test_rejects_mismatched_tensor(over, words):
    with pytest.raises(ValueError, match=words):
        check(**over)
