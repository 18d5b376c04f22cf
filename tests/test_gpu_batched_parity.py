"""Every walker of the batched 128-walker workload against the FP64 oracle.

The workload: 128 walkers drawn uniformly from the prior (zeta in [5, 100], R_mfp in
[5, 20] Mpc, log10 T_vir in [4, 6]) on three 128^3, 250 Mpc boxes (z = 8, 9, 10), the mock
being the fiducial model on the seed + 1 boxes with a 20 % noise term (Sec. 2.5, Sec. 3.4).
One eor_likelihood call gives every walker's chi^2 and Delta^2; the same batch through
eor_set_params / eor_run_ionization (the same kernels, not captured) gives every x_HI box
and must reproduce those spectra. Each of the 384 (walker, redshift) realizations is then
compared with the oracle's: at most 1e-4 of the cells with a flipped ionization decision
(|x_HI difference| > 1e-3), x_HI within 1e-4 on every other cell, every Delta^2 bin within
1e-3 (relative; absolute against the largest bin for a box that is nearly all ionized, where
the spectrum is close to zero), and each walker's chi^2 within 1e-3. The largest and median
errors are printed for the record.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1501_06576_gb300 import eor21, synth

pytestmark = pytest.mark.gpu

N, BOX, ZS, W = 128, 250.0, (8.0, 9.0, 10.0), 128
FLIP_TOL, XHI_TOL, PS_TOL, CHI2_TOL = 1e-4, 1e-4, 1e-3, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_every_walker_of_the_batched_workload_matches_the_oracle():
    delta = synth.density_boxes(N, BOX, ZS, seed=1)
    mock_delta = synth.density_boxes(N, BOX, ZS, seed=2)
    params = synth.walker_params(W, seed=3)
    with eor21.Context(n=N, box_mpc=BOX, z=ZS, max_walkers=W) as ctx:
        ctx.init_boxes(mock_delta)
        ctx.set_params(np.array([[30.0, 15.0, 4.7]]))
        ctx.run_ionization()
        mock = np.ascontiguousarray(ctx.power_spectrum()[0][0])
        sigma = 0.2 * mock
        ctx.init_boxes(delta)
        chi2, d2 = ctx.likelihood(params, mock, sigma, want_d2=True)
        ctx.set_params(params)
        xhi, xhi_mean = ctx.run_ionization(want_xhi=True)
        d2b, _, cnt = ctx.power_spectrum()
    np.testing.assert_allclose(d2b, d2, rtol=1e-12, equal_nan=True)   # same batch, same kernels

    orc = oracle.Oracle()
    flips, xerr, pserr, chierr = [], [], [], []
    for w in range(W):
        chi_ref = 0.0
        for j, z in enumerate(ZS):
            ref = orc.ionize(delta[j], BOX, z, *params[w])
            diff = np.abs(xhi[w, j].astype(np.float64) - ref["xhi"])
            flipped = diff > 1e-3
            flips.append(flipped.mean())
            xerr.append(diff[~flipped].max() if (~flipped).any() else 0.0)
            rd2, _, rcnt = oracle.power_spectrum(ref["dtb"], BOX, 14, 0.1, 1.5)
            assert np.array_equal(cnt[w, j], rcnt)
            ok = rcnt > 0
            if ref["xhi_mean"] > 0.01:
                e = np.max(np.abs(d2[w, j][ok] - rd2[ok]) / np.abs(rd2[ok]))
            else:
                e = np.max(np.abs(d2[w, j][ok] - rd2[ok])) / max(np.max(np.abs(rd2[ok])), 1e-6)
            pserr.append(e)
            assert abs(xhi_mean[w, j] - ref["xhi_mean"]) <= XHI_TOL, (w, j)
            chi_ref += oracle.chi2(rd2, rcnt, mock[j], sigma[j])
        chierr.append(abs(chi2[w] - chi_ref) / max(abs(chi_ref), 1e-12))
    flips, xerr, pserr, chierr = map(np.asarray, (flips, xerr, pserr, chierr))
    summary = (f"128 walkers x 3 z at 128^3: flipped fraction max {flips.max():.2e} median {np.median(flips):.2e} "
               f"(total flipped cells {int(round(flips.sum() * N ** 3))}); max |dx_HI| elsewhere "
               f"{xerr.max():.2e} median {np.median(xerr):.2e}; Delta^2 rel err max {pserr.max():.2e} "
               f"median {np.median(pserr):.2e}; chi^2 rel err max {chierr.max():.2e} median {np.median(chierr):.2e}")
    print(summary)
    out = os.environ.get("EOR_PARITY_SUMMARY")
    if out:
        with open(out, "w") as f:
            f.write(summary + "\n")
    assert flips.max() <= FLIP_TOL
    assert xerr.max() <= XHI_TOL
    assert pserr.max() <= PS_TOL
    assert chierr.max() <= CHI2_TOL
