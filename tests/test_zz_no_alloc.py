"""The allocation-free power spectrum (eor_box_power_spectrum_noalloc).

Callers that cannot allocate GPU memory where they need a power spectrum (applications
that hand all device memory to their own pool or budget, code that must not synchronize
the device) use this entry point: it needs no context and keeps its scratch in a static
device array. This test calls it through the C ABI on two boxes in a row
(the second call reuses the array the first one filled) and checks each result against
the context-based eor_box_power_spectrum on the same box. The file is named to be
collected last; it also passes when run on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1501_06576_gb300 import eor21

pytestmark = pytest.mark.gpu


def test_noalloc_power_spectrum_matches_context_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    n, box_mpc = 64, 100.0
    rng = np.random.default_rng(2026)
    boxes = [(20.0 * (1.0 + 0.5 * rng.standard_normal((n, n, n)))).astype(np.float32) for _ in range(2)]
    with eor21.Context(n=n, box_mpc=box_mpc, z=(9.0,)) as ctx:
        refs = [ctx.box_power_spectrum(b) for b in boxes]

    stream = torch.cuda.Stream()
    d2 = torch.full((14,), float("nan"), dtype=torch.float64, device="cuda")
    nmodes = torch.zeros(14, dtype=torch.int64, device="cuda")
    dev_boxes = [torch.from_numpy(b).cuda() for b in boxes]   # every test allocation before the calls
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    free_after = []
    for dev_box, (ref_d2, _, ref_cnt) in zip(dev_boxes, refs):
        eor21.box_power_spectrum_noalloc(n, box_mpc, dev_box, d2, nmodes, stream=stream.cuda_stream)
        stream.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
        np.testing.assert_array_equal(nmodes.cpu().numpy(), ref_cnt)
        np.testing.assert_allclose(d2.cpu().numpy(), ref_d2, rtol=1e-9)
    # the scratch is the library's static array (EOR21_NOALLOC_SCRATCH_BYTES = 9 MiB): the
    # driver may place it in device memory when the entry point first needs it (in 2 MiB
    # pages), so the first call may take the array itself and nothing more; the second none
    scratch, page = 9 << 20, 2 << 20
    assert free_before - free_after[0] <= (scratch + page - 1) // page * page
    assert free_after[1] >= free_after[0]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # buffers of the size n = 256 needs, so that the C entry point itself refuses the size
    box = torch.zeros((256, 256, 256), dtype=torch.float32, device="cuda")
    d2 = torch.zeros(14, dtype=torch.float64, device="cuda")
    with pytest.raises(eor21.EorError) as e:
        eor21.box_power_spectrum_noalloc(256, 500.0, box, d2)
    assert e.value.code == eor21.EOR_EINVAL
    with pytest.raises(ValueError):   # a box that does not match n is refused before the call
        eor21.box_power_spectrum_noalloc(64, 100.0, box, d2)
