"""FP64 CPU oracle of the affine-invariant ensemble sampler (stretch move).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this module. It shares no code with
the CUDA library and never calls it.

The paper samples its likelihood with the affine-invariant ensemble sampler of
Goodman & Weare (2010) as packaged by Foreman-Mackey et al. (2013) (Sec. 2.4),
with an optional prior on the neutral fraction at the end of reionization
(Sec. 3.3). One step of the parallel form updates the two halves of the ensemble
in turn; walker k of the active half

    picks a partner j uniformly from the other half,
    draws z from g(z) ~ 1/sqrt(z) on [1/a, a]  (z = ((a - 1) u + 1)^2 / a),
    proposes Y = X_j + z (X_k - X_j),
    accepts with probability min(1, z^(d - 1) p(Y) / p(X_k)), d = 3 parameters.

The random numbers come from SplitMix64 (Steele, Lea & Flood 2014), written here
from its published definition and keyed like the CUDA side: for step s, half h,
walker k and draw c in {partner, stretch, accept}, output number
((2 s + h) W + k) 3 + c of the stream keyed by the seed; a uniform in [0, 1) is
its top 53 bits over 2^53. Pins (tests/test_oracle_sampler.py): the generator's
first outputs against published SplitMix64 reference values, the z law's
distribution function, detailed balance of the move on a Gaussian target (mean
and covariance recovered), affine invariance (an affine map of the start and the
target maps the chain), and rejection outside the prior.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = 0x9E3779B97F4A7C15
_MASK = 0xFFFFFFFFFFFFFFFF


def splitmix64_next(state: int) -> tuple[int, int]:
    """One step of SplitMix64: returns (new state, output)."""
    state = (state + _GOLDEN) & _MASK
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return state, z ^ (z >> 31)


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def draw(seed: int, n: int) -> int:
    """Output n (from 0) of the SplitMix64 stream whose state starts at mix(seed)."""
    return _mix((_mix(seed & _MASK) + _GOLDEN * (n + 1)) & _MASK)


def uniform(seed: int, n: int) -> float:
    return (draw(seed, n) >> 11) * (1.0 / 9007199254740992.0)


def stretch_z(u: float, a: float) -> float:
    """Inverse distribution function of g(z) ~ 1/sqrt(z) on [1/a, a]."""
    return ((a - 1.0) * u + 1.0) ** 2 / a


def run(x0, lnp0, steps: int, a: float, seed: int, lnp_fn, prior_lo, prior_hi):
    """Steps of the two-half stretch move from walkers x0 [W][3] with log-posteriors
    lnp0 [W]; lnp_fn(Y [n][3]) gives the log-likelihood of proposals inside the prior
    box (outside it the log-posterior is -inf). Returns (chain [steps][W][3],
    lnp [steps][W], accepted [steps][W] booleans)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    lnp = np.array(lnp0, dtype=np.float64, copy=True)
    w = x.shape[0]
    half = w // 2
    lo = np.asarray(prior_lo, dtype=np.float64)
    hi = np.asarray(prior_hi, dtype=np.float64)
    d = x.shape[1]
    chain = np.empty((steps, w, d))
    lnps = np.empty((steps, w))
    acc = np.zeros((steps, w), dtype=bool)
    for s in range(steps):
        for h in range(2):
            active = np.arange(h * half, (h + 1) * half)
            other = np.arange((1 - h) * half, (2 - h) * half)
            y = np.empty((half, d))
            zs = np.empty(half)
            us = np.empty(half)
            for i, k in enumerate(active):
                base = ((2 * s + h) * w + int(k)) * 3
                j = other[int(uniform(seed, base) * half)]
                zs[i] = stretch_z(uniform(seed, base + 1), a)
                us[i] = uniform(seed, base + 2)
                y[i] = x[j] + zs[i] * (x[k] - x[j])
            inside = np.all((y >= lo) & (y <= hi), axis=1)
            lny = np.full(half, -np.inf)
            if inside.any():
                lny[inside] = lnp_fn(y[inside])
            for i, k in enumerate(active):
                # accept with probability min(1, z^(d-1) p(Y) / p(X_k)): u < exp(q), never
                # outside the prior (q = -inf)
                if not np.isfinite(lny[i]):
                    continue
                q = (d - 1) * math.log(zs[i]) + lny[i] - lnp[k]
                if us[i] == 0.0 or math.log(us[i]) < q:
                    x[k] = y[i]
                    lnp[k] = lny[i]
                    acc[s, k] = True
        chain[s] = x
        lnps[s] = lnp
    return chain, lnps, acc
