"""A bounded device wait that runs out is reported, and leaves the GPU usable.

Every wait of the tensor-core contraction is bounded in GPU time; when one gives up, the CTA
records where (role, barrier, step), stops issuing, waits for its MMAs and bulk copies in
flight, frees its tensor memory and exits, and the host sees EOR_ETIMEOUT. The test makes
that happen without a GPU fault: the test-only switch eor_debug_withhold makes the
epilogue keep back its release of the accumulator buffer of step 0 (the first coefficient
chunk against the first cell tile), so the MMA thread's wait before step 2 (the same
buffer) runs out after 1 ms. Nothing asynchronous is made to
time out. Then the context is destroyed, and a fresh context gives the same chi^2 as one
that never saw the fault.
"""
import numpy as np
import pytest

from paper_1501_06576_gb300 import eor21, synth

pytestmark = pytest.mark.gpu

N, BOX, ZS = 32, 60.0, (9.0,)
WALKERS = 12          # 12 walkers x one 32-column group each = 384 columns = 2 chunks of 256


def _inputs():
    params = synth.walker_params(WALKERS, seed=41)
    delta = synth.density_boxes(N, BOX, ZS, seed=43)
    return params, delta


def _reference():
    params, delta = _inputs()
    with eor21.Context(n=N, box_mpc=BOX, z=ZS, max_walkers=WALKERS) as ctx:
        ctx.init_boxes(delta)
        ctx.set_params(params[:1])
        ctx.run_ionization()
        mock, _, _ = ctx.power_spectrum()
        mock = mock[0]
        chi2 = ctx.likelihood(params, mock, 0.2 * mock)
    return params, delta, mock, chi2


def test_withheld_release_times_out_and_context_recovers():
    params, delta, mock, ref_chi2 = _reference()
    assert np.all(np.isfinite(ref_chi2))
    ctx = eor21.Context(n=N, box_mpc=BOX, z=ZS, max_walkers=WALKERS)
    ctx.init_boxes(delta)
    ctx.debug_withhold(0, 1.0)
    with pytest.raises(eor21.EorError) as e:
        ctx.likelihood(params, mock, 0.2 * mock)
    assert e.value.code == eor21.EOR_ETIMEOUT
    assert "role 2, barrier 7, step 2" in str(e.value), str(e.value)
    ctx.close()                                   # eor_destroy after the timeout

    with eor21.Context(n=N, box_mpc=BOX, z=ZS, max_walkers=WALKERS) as fresh:
        fresh.init_boxes(delta)
        np.testing.assert_allclose(fresh.likelihood(params, mock, 0.2 * mock), ref_chi2, rtol=1e-12)


def test_injection_switched_off_gives_the_normal_result():
    params, delta, mock, ref_chi2 = _reference()
    with eor21.Context(n=N, box_mpc=BOX, z=ZS, max_walkers=WALKERS) as ctx:
        ctx.init_boxes(delta)
        ctx.debug_withhold(0, 1.0)
        ctx.debug_withhold(-1)
        np.testing.assert_allclose(ctx.likelihood(params, mock, 0.2 * mock), ref_chi2, rtol=1e-12)


def test_injection_arguments_are_checked():
    with eor21.Context(n=N, box_mpc=BOX, z=ZS, max_walkers=WALKERS) as ctx:
        for ms in (0.0, -1.0, 5000.0):
            with pytest.raises(eor21.EorError) as e:
                ctx.debug_withhold(0, ms)
            assert e.value.code == eor21.EOR_EINVAL
