"""Pins of the FP64 surrogate oracle (oracle/emulator.py) against things other than itself:
torch's bfloat16 conversion and hand-worked ties, the normal distribution, torch float64
modules and autograd, central finite differences, Adam's closed-form first step and
torch.optim.Adam, and the prior box's corners."""
import math

import numpy as np
import pytest
import torch

from oracle import emulator as em
from paper_1501_06576_gb300 import synth

DIMS = em.layer_dims(4, 16, 3, 5)


def test_bf16_round_hand_ties():
    one = np.float32(1.0)
    ulp = 2.0 ** -7   # bfloat16 spacing at 1
    cases = {
        1.0 + 2.0 ** -8: 1.0,                       # exactly half an ulp above an even pattern -> down
        1.0 + 3 * 2.0 ** -8: 1.0 + 2 * ulp,         # half an ulp above an odd pattern -> up to even
        1.0 + 2.0 ** -8 + 2.0 ** -20: 1.0 + ulp,    # above half -> up
        1.0 + 2.0 ** -9: 1.0,                       # below half -> down
        -(1.0 + 3 * 2.0 ** -8): -(1.0 + 2 * ulp),
        3.0: 3.0,
    }
    for x, want in cases.items():
        assert float(em.bf16_round(np.float32(x))) == want, x
    assert em.bf16_round(one).dtype == np.float32


def test_bf16_round_matches_torch():
    x = (synth.normals(11, 0, 20000) * 10.0 ** synth.uniform01(11, 1, 20000, 0) * 4 - 2).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(em.bf16_round(x), want)


def test_gelu_pins():
    # Phi(1) = 0.8413447460685429 (standard normal table)
    assert em.gelu(np.array(1.0)) == pytest.approx(0.8413447460685429, abs=1e-15)
    assert em.gelu(np.array(0.0)) == 0.0
    u = np.linspace(-6, 6, 101)
    # Phi(-u) = 1 - Phi(u)  =>  GELU(u) - GELU(-u) = u
    assert np.allclose(em.gelu(u) - em.gelu(-u), u, atol=1e-14)
    assert em.gelu(np.array(40.0)) == pytest.approx(40.0)
    assert abs(em.gelu(np.array(-40.0))) < 1e-300
    h = 1e-5
    fd = (em.gelu(u + h) - em.gelu(u - h)) / (2 * h)
    assert np.allclose(em.gelu_grad(u), fd, atol=1e-9)
    assert np.allclose(em.gelu(u), torch.nn.functional.gelu(torch.from_numpy(u)).numpy(), atol=1e-15)


def _torch_net(layers):
    mods = []
    for li, (w, b) in enumerate(layers):
        lin = torch.nn.Linear(w.shape[1], w.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(w))
            lin.bias.copy_(torch.from_numpy(b))
        mods.append(lin)
        if li < len(layers) - 1:
            mods.append(torch.nn.GELU())
    return torch.nn.Sequential(*mods)


def _case(seed=3, n=37):
    theta = synth.mlp_params(seed, DIMS)
    x = synth.uniform01(seed, 7, n * 4).reshape(n, 4) * 2 - 1
    t = synth.normals(seed, 8, n * DIMS[-1][1]).reshape(n, -1)
    return theta, x, t


def test_forward_matches_torch_modules():
    theta, x, _ = _case()
    layers = em.effective_weights(theta, DIMS)
    want = _torch_net(layers)(torch.from_numpy(x)).detach().numpy()
    y, _ = em.forward(theta, DIMS, x)
    assert np.allclose(y, want, rtol=0, atol=1e-13)
    # with weight rounding off, the master weights are used as they are
    y2, _ = em.forward(theta, DIMS, x, round_weights=False)
    want2 = _torch_net(em.unpack(theta, DIMS))(torch.from_numpy(x)).detach().numpy()
    assert np.allclose(y2, want2, atol=1e-13)
    assert not np.allclose(y, y2, atol=1e-6)   # the rounding matters at this size


def test_forward_zero_weights_closed_form():
    theta = np.zeros(em.n_params(DIMS))
    layers = em.unpack(theta, DIMS)
    for li, (w, b) in enumerate(layers):
        b[:] = 0.5 + li
    y, _ = em.forward(theta, DIMS, np.ones((2, 4)))
    # all W = 0: every layer sees only its bias; the output is b_L
    assert np.allclose(y, 3.5)


def test_gradient_matches_autograd():
    theta, x, t = _case()
    layers = em.effective_weights(theta, DIMS)
    net = _torch_net(layers)
    out = net(torch.from_numpy(x))
    loss = torch.mean((out - torch.from_numpy(t)) ** 2)
    loss.backward()
    want = []
    for mod in net:
        if isinstance(mod, torch.nn.Linear):
            want += [mod.weight.grad.numpy().ravel(), mod.bias.grad.numpy()]
    want = np.concatenate(want)
    got_loss, got = em.loss_and_grad(theta, DIMS, x, t)
    assert got_loss == pytest.approx(loss.item(), rel=1e-13)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-14)


def test_gradient_finite_differences():
    theta, x, t = _case(seed=5, n=9)
    _, g = em.loss_and_grad(theta, DIMS, x, t, round_weights=False)
    rng_idx = (synth.uniform01(5, 9, 60) * theta.size).astype(int)
    h = 1e-6
    for i in rng_idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fp = em.mse_loss(em.forward(tp, DIMS, x, False)[0], t)
        fm = em.mse_loss(em.forward(tm, DIMS, x, False)[0], t)
        assert (fp - fm) / (2 * h) == pytest.approx(g[i], rel=1e-6, abs=1e-10), i


def test_adam_first_step_closed_form():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    th = np.array([1.0, 2.0, 3.0, 4.0])
    new, m, v = em.adam_step(th, g, np.zeros(4), np.zeros(4), 1, 0.01)
    # bias-corrected moments at step 1 are g and g^2: the step is -lr g / (|g| + eps)
    assert np.allclose(new, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_matches_torch():
    theta, x, t = _case(seed=8, n=20)
    p = torch.nn.Parameter(torch.from_numpy(theta.copy()))
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    th, m, v = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    for step in range(1, 6):
        _, g = em.loss_and_grad(th, DIMS, x, t)
        th, m, v = em.adam_step(th, g, m, v, step, 3e-3)
        opt.zero_grad()
        p.grad = torch.from_numpy(em.loss_and_grad(p.detach().numpy(), DIMS, x, t)[1])
        opt.step()
        assert np.allclose(th, p.detach().numpy(), rtol=0, atol=1e-12)


def test_adam_converges_on_quadratic():
    # f(th) = sum c (th - a)^2 has its minimum at a
    a = np.array([1.0, -2.0, 0.5])
    c = np.array([1.0, 10.0, 0.1])
    th, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for step in range(1, 4001):
        th, m, v = em.adam_step(th, 2 * c * (th - a), m, v, step, 0.01 * (1 - step / 4001) + 1e-4)
    assert np.allclose(th, a, atol=1e-3)


def test_features_corners_and_targets():
    lo, hi = (5.0, 5.0, 4.0), (100.0, 20.0, 6.0)
    f = em.features(np.array([lo, hi, [52.5, 12.5, 5.0]]), 9.0, lo, hi, 8.0, 10.0)
    assert np.allclose(f[:, :3], [[-1, -1, -1], [1, 1, 1], [0, 0, 0]])
    assert np.allclose(f[:, 3], 0.0)
    assert np.allclose(em.features(np.array([lo]), 8.0, lo, hi, 8.0, 10.0)[:, 3], -1.0)
    assert np.allclose(em.features(np.array([lo]), 9.0, lo, hi, 9.0, 9.0)[:, 3], 0.0)
    t = em.targets(np.array([1e-6, 1.0, 100.0, np.nan]), 1e-4)
    assert np.allclose(t, [-4.0, 0.0, 2.0, -4.0])


def test_ensemble_spread_definition():
    theta, x, _ = _case(n=6)
    mean, std = np.zeros(5), np.ones(5)
    avg, spread = em.predict_log10_d2([theta, theta], DIMS, x, mean, std)
    assert np.allclose(spread, 0.0)
    y = em.forward(theta, DIMS, x, True, True)[0]
    assert np.allclose(avg, y)
    avg2, spread2 = em.predict_log10_d2([theta, np.zeros_like(theta)], DIMS, x, mean, std)
    # two members: population standard deviation = |difference| / 2
    assert np.allclose(spread2, np.abs(y).max(axis=1) / 2)
    assert np.allclose(avg2, y / 2)
