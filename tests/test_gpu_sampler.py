"""GPU tests of the device-side ensemble sampler (eor_mcmc_*) against the FP64 stretch-move
oracle (oracle/sampler.py), which draws the same SplitMix64 numbers.

On the Gaussian test target both sides evaluate the same FP64 formula, so every Metropolis
decision and every position must agree (positions to 1e-12). On the simulation target the
mock's sigma is made so large that log p is ~0 and the decisions turn on z^2 and the
neutral-fraction prior alone; the oracle evaluates its own FP64 likelihood, and a decision
may differ only where the oracle's x_HI lies within 1e-4 of the prior's limit."""
import numpy as np
import pytest

import oracle
from oracle import sampler as sm
from paper_1501_06576_gb300 import eor21, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


MU = np.array([40.0, 12.0, 5.0])
COV = np.array([[100.0, 5.0, 0.0], [5.0, 4.0, 0.2], [0.0, 0.2, 0.1]])


def test_gaussian_target_matches_oracle():
    w, steps, seed = 16, 60, 5
    prec = np.linalg.inv(COV)
    lo, hi = [5.0, 5.0, 4.0], [100.0, 20.0, 6.0]   # tight enough that some proposals leave it
    smp = eor21.Sampler(None, n_walkers=w, seed=seed, gauss_target=1, gauss_mean=MU, gauss_precision=prec,
                        prior_lo=lo, prior_hi=hi)
    x0 = MU + synth.normals(8, 0, w * 3).reshape(w, 3) * np.sqrt(np.diag(COV)) * 0.3
    f = lambda y: -0.5 * np.einsum("ni,ij,nj->n", y - MU, prec, y - MU)
    lnp0 = smp.start(x0)
    assert np.allclose(lnp0, f(x0), rtol=1e-13, atol=1e-12)
    chain, lnp, acc = smp.run(steps)
    rc, rl, ra = sm.run(x0, f(x0), steps, 2.0, seed, f, lo, hi)
    assert np.array_equal(acc.astype(bool), ra)
    assert np.allclose(chain, rc, rtol=1e-12, atol=1e-12)
    assert np.allclose(lnp, rl, rtol=1e-12, atol=1e-12)
    assert 0.2 < ra.mean() < 0.9
    # a second call continues the same chain (the step count carries over)
    chain2, _, acc2 = smp.run(5)
    rc2, _, ra2 = sm.run(x0, f(x0), steps + 5, 2.0, seed, f, lo, hi)
    assert np.array_equal(acc2.astype(bool), ra2[steps:])
    assert np.allclose(chain2, rc2[steps:], rtol=1e-12, atol=1e-12)
    x, l = smp.walkers()
    assert np.allclose(x, rc2[-1], rtol=1e-12, atol=1e-12)
    smp.close()


def test_simulation_target_with_neutral_fraction_prior():
    n, box, zs = 32, 60.0, (9.0,)
    delta = synth.density_boxes(n, box, zs, seed=5)
    ctx = eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=4)
    ctx.init_boxes(delta)
    mock = np.full((1, 14), 10.0)
    sigma = 1e6 * mock   # chi^2 ~ 1e-10: the decisions rest on z^2 and the x_HI prior
    w, steps, seed, xmin = 8, 4, 3, 0.35
    lo, hi = [5.0, 5.0, 4.0], [100.0, 20.0, 6.0]
    smp = eor21.Sampler(ctx, n_walkers=w, seed=seed, prior_lo=lo, prior_hi=hi, xhi_prior_z=0, xhi_prior_min=xmin)
    x0 = np.array([[30.0, 12.0, 4.7], [20.0, 8.0, 5.0], [40.0, 15.0, 4.5], [25.0, 10.0, 5.3],
                   [35.0, 18.0, 4.9], [15.0, 6.0, 5.5], [50.0, 9.0, 5.8], [22.0, 14.0, 5.1]])
    orc = oracle.Oracle()
    cache = {}

    def lnp_fn(y):
        out = []
        for p in y:
            key = tuple(p)
            if key not in cache:
                ion = orc.ionize(delta[0], box, zs[0], *p)
                d2, _, cnt = oracle.power_spectrum(ion["dtb"], box, 14, 0.1, 1.5)
                chi2 = oracle.chi2(d2, cnt, mock[0], sigma[0])
                cache[key] = (-0.5 * chi2 if ion["xhi_mean"] >= xmin else -np.inf, ion["xhi_mean"])
            out.append(cache[key][0])
        return np.array(out)

    lnp0 = smp.start(x0, mock, sigma)
    ref0 = lnp_fn(x0)
    assert np.array_equal(np.isfinite(lnp0), np.isfinite(ref0))
    chain, lnp, acc = smp.run(steps)
    rc, rl, ra = sm.run(x0, ref0, steps, 2.0, seed, lnp_fn, lo, hi)
    for s in range(steps):
        if not np.array_equal(acc[s].astype(bool), ra[s]):
            # allowed only where the oracle's x_HI of the proposal sits at the prior's limit
            close = [abs(v[1] - xmin) < 1e-4 for v in cache.values()]
            assert any(close), f"step {s}: decisions differ away from the prior's limit"
            break
        assert np.allclose(chain[s], rc[s], rtol=1e-12, atol=1e-12)
        fin = np.isfinite(rl[s])
        assert np.array_equal(np.isfinite(lnp[s]), fin)
        assert np.allclose(lnp[s][fin], rl[s][fin], rtol=5e-3, atol=1e-12)
    assert ra.any() and not ra.all()
    smp.close()
    ctx.close()


def test_sampler_errors():
    ctx = eor21.Context(n=32, box_mpc=60.0, z=(9.0,), max_walkers=4)
    with pytest.raises(eor21.EorError):
        eor21.Sampler(ctx, n_walkers=7)
    with pytest.raises(eor21.EorError):
        eor21.Sampler(ctx, n_walkers=10)              # half the ensemble exceeds max_walkers
    with pytest.raises(eor21.EorError):
        eor21.Sampler(ctx, n_walkers=8, prior_hi=[100.0, 25.0, 6.0])   # R_mfp beyond r_mfp_max
    with pytest.raises(eor21.EorError):
        eor21.Sampler(None, n_walkers=8)              # no context and no test target
    smp = eor21.Sampler(ctx, n_walkers=8)
    with pytest.raises(eor21.EorError) as ei:
        smp.run(2)
    assert ei.value.code == eor21.EOR_ESTATE
    with pytest.raises(eor21.EorError) as ei:
        smp.start(synth.walker_params(8, seed=1), np.ones((1, 14)), np.ones((1, 14)))   # no boxes yet
    assert ei.value.code == eor21.EOR_ESTATE
    smp.close()
    ctx.close()
