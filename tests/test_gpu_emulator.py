"""GPU tests of the power-spectrum surrogate through the C ABI (eor_emu_*).

Parity with the FP64 oracle (oracle/emulator.py) on the same seeded weights and inputs:
forward pass, loss and gradient, Adam steps, ensemble prediction and the fallback rule.
Tolerances follow the arithmetic: weights are bf16-rounded identically on both sides, so
what remains is FP32 summation over at most a few hundred terms (relative ~1e-6) and
CUDA's erff/expf in GELU (a few ulp): 1e-4 relative on outputs, 1e-4 of a layer's largest
gradient, 1e-4 dex on predicted log10 Delta^2.

Then the surrogate against the simulation it stands in for: walkers sent to the
simulation get exactly the simulation's chi^2 and spectra, emulated walkers the chi^2 of
their predicted spectra, and a network trained on simulated spectra (64^3, 100 Mpc,
z = 9) is measured against held-out simulations: how many walkers it spares the
simulation and how many of those it gets wrong by more than 5 % in some bin.
"""
import time

import numpy as np
import pytest

import oracle
from oracle import emulator as em
from paper_1501_06576_gb300 import eor21, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def make_emu(members=3, hidden=256, n_hidden=3, n_bins=14, zs=(8.0, 9.0, 10.0), max_rows=1024, **kw):
    return eor21.Emulator(members=members, hidden=hidden, n_hidden=n_hidden, n_bins=n_bins, z=zs,
                          max_rows=max_rows, **kw)


def dims_of(emu):
    return em.layer_dims(4, emu.cfg.hidden, emu.cfg.n_hidden, emu.cfg.n_bins)


def seeded_weights(emu, seed=21):
    dims = dims_of(emu)
    return np.stack([synth.mlp_params(seed + e, dims) for e in range(emu.members)]).astype(np.float32)


def seeded_batch(n, n_bins, seed=4):
    x = (synth.uniform01(seed, 1, 4 * n).reshape(n, 4) * 2 - 1).astype(np.float32)
    t = synth.normals(seed, 2, n * n_bins).reshape(n, n_bins).astype(np.float32)
    return x, t


@pytest.mark.parametrize("hidden,n_hidden,n", [(256, 3, 150), (64, 2, 37), (96, 1, 1)])
def test_forward_matches_oracle(hidden, n_hidden, n):
    emu = make_emu(hidden=hidden, n_hidden=n_hidden)
    w = seeded_weights(emu)
    emu.set_weights(w)
    x, _ = seeded_batch(n, emu.n_bins)
    y = emu.forward(x)
    for e in range(emu.members):
        ref, _ = em.forward(w[e].astype(np.float64), dims_of(emu), x)
        assert np.all(np.abs(y[e] - ref) <= 1e-4 * (1.0 + np.abs(ref))), np.abs(y[e] - ref).max()
    # master weights come back unchanged
    assert np.array_equal(emu.get_weights(), w)
    emu.close()


@pytest.mark.parametrize("hidden,n_hidden,n", [(256, 3, 150), (48, 2, 200)])
def test_loss_grad_matches_oracle(hidden, n_hidden, n):
    emu = make_emu(hidden=hidden, n_hidden=n_hidden)
    w = seeded_weights(emu, seed=31)
    emu.set_weights(w)
    x, t = seeded_batch(n, emu.n_bins, seed=6)
    loss, grad = emu.loss_grad(x, t)
    dims = dims_of(emu)
    for e in range(emu.members):
        ref_loss, ref_grad = em.loss_and_grad(w[e].astype(np.float64), dims, x, t)
        assert loss[e] == pytest.approx(ref_loss, rel=1e-5)
        p = 0
        for fi, fo in dims:
            for size in (fi * fo, fo):   # W then b of each layer
                g, r = grad[e, p:p + size], ref_grad[p:p + size]
                assert np.abs(g - r).max() <= 1e-4 * np.abs(r).max() + 1e-12, (fi, fo, size)
                p += size
    emu.close()


def test_adam_steps_match_oracle():
    emu = make_emu(members=2, hidden=64, n_hidden=2)
    w0 = seeded_weights(emu, seed=41)
    x, t = seeded_batch(96, emu.n_bins, seed=8)
    dims = dims_of(emu)
    lr, steps = 1e-3, 4
    for run_steps in (1, steps):
        emu.set_weights(w0)
        emu.train_batch(x, t, run_steps, lr)
        got = emu.get_weights()
        for e in range(emu.members):
            th = w0[e].astype(np.float64)
            m = np.zeros_like(th)
            v = np.zeros_like(th)
            robust = np.ones(th.size, dtype=bool)
            for s in range(1, run_steps + 1):
                _, g = em.loss_and_grad(th, dims, x, t)
                # entries whose gradient sign FP32 summation cannot flip
                robust &= np.abs(g) > 1e-3 * np.abs(g).max()
                th, m, v = em.adam_step(th, g, m, v, s, lr)
            d = np.abs(got[e] - th)
            assert robust.mean() > 0.9
            assert d[robust].max() <= 2e-7 + 1e-6 * np.abs(th[robust]).max(), d[robust].max()
            assert d.max() <= 2 * lr * run_steps
    emu.close()


def test_training_is_deterministic_and_learns():
    walkers = synth.walker_params(600, seed=3)
    zs = (8.0, 9.0, 10.0)
    # a smooth stand-in spectrum (training-loop test only; the simulated ones are below)
    kc = np.geomspace(0.1, 1.5, 15)
    kc = np.sqrt(kc[:-1] * kc[1:])
    z = np.array(zs)
    d2 = (walkers[:, 0, None, None] / 30.0) ** 0.5 * (1 + 0.05 * walkers[:, 1, None, None]) \
        * (kc[None, None, :] / 0.3) ** (0.5 + 0.1 * walkers[:, 2, None, None]) * (z[None, :, None] / 9.0) ** 2
    out = []
    for _ in range(2):
        emu = make_emu(members=2, hidden=128, zs=zs, max_rows=2048, max_samples=4096, seed=7)
        emu.set_data(walkers, d2)
        first = emu.train(1, 256, 2e-3, seed=5)
        last = emu.train(600, 256, 2e-3, seed=5)
        out.append((first, last, emu.get_weights()))
        norm = emu.get_normalization()
        ref_t = em.targets(d2, emu.cfg.d2_floor).reshape(-1, 14)
        assert np.allclose(norm[0], ref_t.mean(axis=0), rtol=1e-12, atol=1e-12)
        assert np.allclose(norm[1], ref_t.std(axis=0), rtol=1e-10)
        emu.close()
    assert np.array_equal(out[0][2], out[1][2])
    assert np.all(out[0][1] < 0.05 * out[0][0]), (out[0][0], out[0][1])


# predictions on the tensor cores round every layer input to BF16; the oracle does the same
# (round_act) and what remains is FP32 summation order flipping an occasional BF16 rounding
# by one unit (2^-8 relative in one activation): 2e-3 dex bounds its effect on the outputs
TC_TOL = 2e-3


def _pred_setup(members=3, tensor_cores=False):
    emu = make_emu(members=members, max_rows=2048)
    emu.set_inference(tensor_cores)
    w = seeded_weights(emu, seed=51)
    emu.set_weights(w)
    norm = np.stack([synth.normals(9, 1, 14) + 2.0, 0.2 + synth.uniform01(9, 2, 14)])
    emu.set_normalization(norm)
    return emu, w, norm


def _oracle_predict(emu, w, norm, params):
    dims = dims_of(emu)
    zs = list(emu.cfg.z)[:emu.n_z]
    lo, hi = list(emu.cfg.prior_lo), list(emu.cfg.prior_hi)
    preds, spreads = [], []
    for z in zs:
        x = em.features(params, z, lo, hi, min(zs), max(zs))
        p, s = em.predict_log10_d2([w[e].astype(np.float64) for e in range(emu.members)], dims, x, norm[0], norm[1],
                                   round_act=emu.inference() == 1)
        preds.append(p)
        spreads.append(s)
    return np.stack(preds, axis=1), np.stack(spreads, axis=1)


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_predict_and_fallback_rule_match_oracle(tensor_cores):
    emu, w, norm = _pred_setup(tensor_cores=tensor_cores)
    assert emu.inference() == (1 if tensor_cores else 0)
    tol = TC_TOL if tensor_cores else 1e-4
    params = synth.walker_params(300, seed=12)
    params[5] = (120.0, 10.0, 5.0)   # outside the prior box
    params[6] = (50.0, 4.0, 5.0)
    pred, spread, fb = emu.predict(params)
    rp, rs = _oracle_predict(emu, w, norm, params)
    assert np.abs(pred - rp).max() <= tol, np.abs(pred - rp).max()
    assert np.abs(spread - rs).max() <= tol
    # threshold at the median score: fallback = outside | a bin below 10 x floor | score > tau
    score = rs.max(axis=1)
    tau = float(np.median(score))
    emu.set_threshold(tau)
    _, _, fb = emu.predict(params)
    outside = np.any((params < np.array(emu.cfg.prior_lo)) | (params > np.array(emu.cfg.prior_hi)), axis=1)
    low = np.any(rp < np.log10(10 * emu.cfg.d2_floor), axis=(1, 2))
    want = outside | low | (score > tau)
    clear = np.abs(score - tau) > tol
    assert fb[5] == 1 and fb[6] == 1
    assert np.array_equal(fb[clear].astype(bool), want[clear])
    assert 0.3 < fb.mean() < 0.7
    emu.close()


def test_calibration_picks_the_threshold():
    emu, w, norm = _pred_setup()
    params = synth.walker_params(400, seed=13)
    rp, rs = _oracle_predict(emu, w, norm, params)
    score = rs.max(axis=1)
    # simulated spectra that the prediction misses by 10 % on a chosen set of walkers
    bad = synth.uniform01(13, 5, 400) < 0.2
    d2 = 10.0 ** rp
    d2[bad, 0, 3] *= 1.1
    tau, frac = emu.calibrate(params, d2, recall=1.0)
    # recall 1: tau just below the smallest score of the missed walkers (all finite here)
    assert np.all(np.isfinite(score))
    smin = score[bad].min()
    assert abs(tau - smin) <= 1e-4
    _, _, fb = emu.predict(params)
    assert np.all(fb[bad] == 1)
    assert frac == pytest.approx(fb.mean())
    # recall 0.5: the median-ranked missed walker sets tau
    tau2, _ = emu.calibrate(params, d2, recall=0.5)
    sb = np.sort(score[bad])[::-1]
    k = int(np.ceil(0.5 * bad.sum()))
    assert abs(tau2 - sb[k - 1]) <= 1e-4
    emu.close()


def _sim_ctx(n=32, box=60.0, zs=(9.0,), max_walkers=64, seed=5):
    ctx = eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=max_walkers, k_lo=0.15, k_hi=1.5, n_bins=8)
    delta = synth.density_boxes(n, box, zs, seed=seed)
    ctx.init_boxes(delta)
    return ctx


def test_emulator_likelihood_routes_walkers():
    zs = (9.0,)
    ctx = _sim_ctx(zs=zs)
    emu = make_emu(members=2, hidden=64, n_hidden=2, n_bins=8, zs=zs, max_rows=512)
    w = seeded_weights(emu, seed=61)
    emu.set_weights(w)
    norm = np.stack([np.full(8, 2.0), np.full(8, 0.3)])
    emu.set_normalization(norm)
    params = synth.walker_params(150, seed=14)
    _, mock = ctx.likelihood(np.array([[30.0, 12.0, 4.7]]), np.ones((1, 8)), np.ones((1, 8)), want_d2=True)
    mock = mock[0]   # [n_z][n_bins]
    sigma = 0.2 * mock
    chi_sim, d2_sim = [], []
    for i in range(0, 150, 64):
        c, d = ctx.likelihood(params[i:i + 64], mock, sigma, want_d2=True)
        chi_sim.append(c)
        d2_sim.append(d)
    chi_sim, d2_sim = np.concatenate(chi_sim), np.concatenate(d2_sim)
    # everything to the simulation: the simulation's results, bit for bit
    emu.set_threshold(-1.0)
    chi, d2, fb = emu.likelihood(ctx, params, mock, sigma, want_d2=True)
    assert np.all(fb == 1)
    assert np.array_equal(chi, chi_sim) and np.array_equal(d2, d2_sim, equal_nan=True)
    # everything emulated: chi^2 (Sec. 2.5 bins, the oracle's chi^2 and mode counts) of the
    # oracle's prediction from the same weights; the tolerance carries 1e-4 dex of prediction
    # difference through each bin's term
    emu.set_threshold(np.inf)
    pred, _, fb_pred = emu.predict(params)
    chi, d2, fb = emu.likelihood(ctx, params, mock, sigma, want_d2=True)
    assert np.array_equal(fb, fb_pred)
    emulated = fb == 0
    assert emulated.sum() > 100
    rp, _ = _oracle_predict(emu, w, norm, params)
    box = synth.density_boxes(32, 60.0, zs, seed=5)[0].astype(np.float64)
    _, _, cnt = oracle.power_spectrum(box, 60.0, 8, 0.15, 1.5)
    for i in np.nonzero(emulated)[0]:
        d2_ref = 10.0 ** rp[i, 0]
        want = oracle.chi2(d2_ref, cnt, mock[0], sigma[0], k_lo=0.15, k_hi=1.5)
        r = (d2_ref - mock[0]) / sigma[0]
        dr = d2_ref * (10.0 ** 1e-4 - 1.0) / sigma[0]
        used = (cnt > 0) & (np.sqrt(np.geomspace(0.15, 1.5, 9)[:-1] * np.geomspace(0.15, 1.5, 9)[1:]) <= 1.0)
        tol = np.sum(((2 * np.abs(r) + dr) * dr)[used]) + 1e-12
        assert abs(chi[i] - want) <= tol, (chi[i], want, tol)
        assert np.allclose(d2[i, 0], 10.0 ** pred[i, 0], rtol=1e-12)
        assert np.allclose(d2[i, 0], d2_ref, rtol=3e-4)
    # mixed: the median spread splits the walkers
    _, spread, _ = emu.predict(params)
    emu.set_threshold(float(np.median(spread.max(axis=1))))
    chi, d2, fb = emu.likelihood(ctx, params, mock, sigma, want_d2=True)
    sim = fb == 1
    assert 0 < sim.sum() < 150
    assert np.array_equal(chi[sim], chi_sim[sim])
    assert np.array_equal(d2[sim], d2_sim[sim], equal_nan=True)
    emu.close()
    ctx.close()


def test_tensor_core_inference_matches_fp32_units():
    emu, w, norm = _pred_setup(tensor_cores=True)
    params = synth.walker_params(600, seed=15)    # 1800 rows: 15 tiles of 128, the last one ragged
    p_tc, s_tc, _ = emu.predict(params)
    emu.set_inference(False)
    p_fp, s_fp, _ = emu.predict(params)
    # BF16 activations against FP32 ones: the oracle puts this network's difference at
    # 1.3e-3 dex at most and 1.3e-4 on average on these inputs
    assert np.abs(p_tc - p_fp).max() < 5e-3
    assert np.abs(p_tc - p_fp).mean() < 5e-4
    emu.close()


def test_emulator_errors():
    emu = make_emu(members=1, hidden=32, n_hidden=1, max_rows=64)
    with pytest.raises(eor21.EorError) as ei:
        emu.set_inference(True)   # tensor-core inference serves 3 hidden layers of 256
    assert ei.value.code == eor21.EOR_ENOTSUP
    with pytest.raises(eor21.EorError) as ei:
        emu.train(10, 32, 1e-3)
    assert ei.value.code == eor21.EOR_ESTATE
    with pytest.raises(eor21.EorError) as ei:
        emu.predict(synth.walker_params(30, seed=1))   # 30 walkers x 3 z > 64 rows
    assert ei.value.code == eor21.EOR_EINVAL
    with pytest.raises(eor21.EorError):
        emu.set_normalization(np.stack([np.zeros(14), np.zeros(14)]))
    ctx = _sim_ctx()
    with pytest.raises(eor21.EorError) as ei:   # other bins and redshifts than the emulator
        emu.likelihood(ctx, synth.walker_params(2, seed=1), np.ones((1, 8)), np.ones((1, 8)))
    assert ei.value.code == eor21.EOR_EINVAL
    with pytest.raises(eor21.EorError):
        eor21.Emulator(members=9)
    ctx.close()
    emu.close()


def test_trained_surrogate_gain_over_simulation():
    """Train on simulated spectra, calibrate on held-out ones, and measure on a third set:
    the fraction of walkers the surrogate spares the simulation, how many of those miss the
    simulated spectrum by more than 5 % in some bin, and the time of a likelihood call."""
    n, box, zs = 64, 100.0, (9.0,)
    ctx = eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=512)
    ctx.init_boxes(synth.density_boxes(n, box, zs, seed=42))
    fid = np.array([[30.0, 15.0, np.log10(3e4)]])
    _, mock = ctx.likelihood(fid, np.ones((1, 14)), np.ones((1, 14)), want_d2=True)
    mock = mock[0]
    sigma = 0.2 * mock

    def simulate(params):
        chis, d2s = [], []
        for i in range(0, len(params), 512):
            c, d = ctx.likelihood(params[i:i + 512], mock, sigma, want_d2=True)
            chis.append(c)
            d2s.append(d)
        return np.concatenate(chis), np.concatenate(d2s)

    train_p = synth.walker_params(6144, seed=100)
    val_p = synth.walker_params(2048, seed=101)
    test_p = synth.walker_params(1024, seed=102)
    _, train_d2 = simulate(train_p)
    _, val_d2 = simulate(val_p)
    test_chi, test_d2 = simulate(test_p)

    emu = eor21.Emulator(z=zs, members=4, max_rows=2048, max_samples=8192, seed=3)
    emu.set_data(train_p, train_d2)
    loss = emu.train(16000, 512, 2e-3, seed=11)
    tau, val_frac = emu.calibrate(val_p, val_d2, recall=0.99)

    pred, _, fb = emu.predict(test_p)
    has_modes = np.isfinite(test_d2) & (test_d2 > emu.cfg.d2_floor)
    rel = np.abs(10.0 ** pred / np.where(has_modes, test_d2, 1.0) - 1.0)
    err = np.where(has_modes, rel, 0.0).max(axis=(1, 2))
    accepted = fb == 0
    miss = float(np.mean(err[accepted] > 0.05)) if accepted.any() else 0.0

    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    chi, _, fb2 = emu.likelihood(ctx, test_p, mock, sigma)
    t_emu = time.perf_counter() - t0
    t0 = time.perf_counter()
    simulate(test_p)
    t_sim = time.perf_counter() - t0
    print(f"\nsurrogate: loss {loss}, tau {tau:.4f}, val fallback {val_frac:.3f}, test fallback "
          f"{1 - accepted.mean():.3f}, accepted walkers over 5 %: {miss:.4f}, median error of accepted "
          f"{np.median(err[accepted]) if accepted.any() else float('nan'):.4f}, likelihood "
          f"{t_emu * 1e3:.1f} ms vs simulation {t_sim * 1e3:.1f} ms")
    assert np.array_equal(fb2, fb)
    assert np.array_equal(chi[fb == 1], test_chi[fb == 1])
    # the surrogate spares the simulation for a large share of the walkers and is rarely wrong
    # on them (at recall 0.99 the threshold is set by the few worst validation walkers, so the
    # share moves between trainings: 46-72 % measured on this workload)
    assert accepted.mean() >= 0.4
    assert miss <= 0.02
    emu.close()
    ctx.close()
