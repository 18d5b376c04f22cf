"""Pins of the FP64 stretch-move sampler oracle (oracle/sampler.py) against things other
than itself: an independent SplitMix64 implementation and the uniformity of its outputs,
the closed-form distribution function of the stretch factor, the moments of a Gaussian
target (detailed balance with the z^(d-1) factor), affine invariance and the prior box."""
import math

import numpy as np
import pytest

from oracle import sampler as sm
from paper_1501_06576_gb300 import synth


def test_splitmix64_matches_independent_implementation():
    # the input generator keys its stream (seed 0, stream 0) by mix(1): the same sequence
    want = synth.splitmix64(0, 0, 64)
    got = [sm.draw(1, n) for n in range(64)]
    assert [int(v) for v in want] == got
    # the plain recurrence from state 0 gives mix(golden), mix(2 golden), ...
    st, out = sm.splitmix64_next(0)
    assert out == sm._mix(0x9E3779B97F4A7C15) and st == 0x9E3779B97F4A7C15


def test_uniforms_are_uniform():
    u = np.array([sm.uniform(7, n) for n in range(40000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    counts, _ = np.histogram(u, bins=20, range=(0, 1))
    chi2 = np.sum((counts - 2000) ** 2 / 2000)
    assert chi2 < 45.3   # 99.9 % point of chi^2 with 19 degrees of freedom
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.02


def test_stretch_factor_distribution():
    # g(z) ~ 1/sqrt(z) on [1/a, a] has G(z) = (sqrt z - 1/sqrt a) / (sqrt a - 1/sqrt a)
    for a in (1.5, 2.0, 3.0):
        for u in np.linspace(0, 1, 11):
            z = sm.stretch_z(u, a)
            g = (math.sqrt(z) - 1 / math.sqrt(a)) / (math.sqrt(a) - 1 / math.sqrt(a))
            assert g == pytest.approx(u, abs=1e-12)
        assert sm.stretch_z(0.0, a) == pytest.approx(1 / a) and sm.stretch_z(1.0, a) == pytest.approx(a)


MU = np.array([1.0, -2.0, 0.5])
COV = np.array([[1.0, 0.6, 0.0], [0.6, 2.0, -0.3], [0.0, -0.3, 0.5]])


def _gauss(mu, cov):
    inv = np.linalg.inv(cov)
    return lambda y: -0.5 * np.einsum("ni,ij,nj->n", y - mu, inv, y - mu)


def test_gaussian_target_moments():
    w, steps = 32, 3000
    x0 = MU + 0.1 * synth.normals(3, 0, w * 3).reshape(w, 3)
    f = _gauss(MU, COV)
    chain, lnp, acc = sm.run(x0, f(x0), steps, 2.0, 11, f, [-50] * 3, [50] * 3)
    s = chain[500:].reshape(-1, 3)
    assert np.allclose(s.mean(axis=0), MU, atol=0.15)
    assert np.allclose(np.cov(s.T), COV, atol=0.25)
    assert 0.3 < acc.mean() < 0.9
    assert np.allclose(lnp, f(chain.reshape(-1, 3)).reshape(steps, w))


def test_affine_invariance():
    w, steps = 16, 40
    x0 = MU + synth.normals(4, 0, w * 3).reshape(w, 3)
    f = _gauss(MU, COV)
    A = np.array([[2.0, 0.5, 0.0], [0.0, 1.0, 0.3], [0.1, 0.0, 3.0]])
    b = np.array([5.0, -1.0, 2.0])
    g = _gauss(A @ MU + b, A @ COV @ A.T)
    c1, l1, a1 = sm.run(x0, f(x0), steps, 2.0, 5, f, [-1e3] * 3, [1e3] * 3)
    x0b = x0 @ A.T + b
    c2, l2, a2 = sm.run(x0b, g(x0b), steps, 2.0, 5, g, [-1e3] * 3, [1e3] * 3)
    assert np.array_equal(a1, a2)
    assert np.allclose(c2, c1 @ A.T + b, rtol=1e-9, atol=1e-9)
    assert np.allclose(l1, l2, atol=1e-9)


def test_prior_box_is_never_left():
    w = 12
    lo, hi = np.array([0.0, 0.0, 0.0]), np.array([1.0, 1.0, 1.0])
    x0 = 0.4 + 0.2 * synth.uniform01(6, 0, w * 3).reshape(w, 3)
    f = lambda y: -0.5 * np.sum((y - 0.5) ** 2, axis=1) / 4.0   # broad: most proposals hit the walls
    chain, lnp, acc = sm.run(x0, f(x0), 200, 2.0, 9, f, lo, hi)
    assert np.all(chain >= lo) and np.all(chain <= hi)
    assert acc.any() and not acc.all()
