"""FP64 CPU oracle of the learned surrogate of the 21-cm power spectrum.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this module. It shares no code with
the CUDA library and never calls it.

The surrogate is not in the paper: it replaces, for parameter sets where it is
trusted, the simulation whose Delta^2(k) (Sec. 2.2, the 21-cm power spectrum in
logarithmic k bins) enters the chi^2 of Sec. 2.5. It is a multilayer perceptron

    inputs  x = the walker's (zeta, R_mfp, log10 T_vir) and the redshift z, each
            mapped linearly from its prior interval onto [-1, 1];
    hidden  h_l = GELU(W_l h_{l-1} + b_l), l = 0 .. L-1, GELU(u) = u Phi(u)
            (Hendrycks & Gimpel 2016; Phi the standard normal distribution);
    output  y = W_L h_{L-1} + b_L, the standardised log10 Delta^2 per bin:
            log10 Delta^2_b = mean_b + std_b y_b,

with weights rounded to bfloat16 (round to nearest, ties to even) wherever they
multiply, and biases, activations and sums kept in higher precision. Training
minimises the mean squared error over samples and bins with Adam (Kingma & Ba
2015: beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected moments); the
gradient passes the weight rounding unchanged (its derivative is taken as 1), so
the master weights receive the gradient of the rounded ones.

Everything here is FP64 numpy, step by step in that order. Pins
(tests/test_oracle_emulator.py): bf16 rounding against torch's conversion and
hand-worked ties; GELU against the normal distribution's printed value at 1, its
odd-part identity and its limits; forward and gradient against torch float64
modules and autograd and against central finite differences; Adam against its
closed-form first step and torch.optim.Adam in float64; the feature map against
the prior box's corners.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def layer_dims(n_in: int, hidden: int, n_hidden: int, n_out: int) -> list[tuple[int, int]]:
    """(fan_in, fan_out) of every layer: n_in -> hidden (x n_hidden) -> n_out."""
    dims = [(n_in, hidden)] + [(hidden, hidden)] * (n_hidden - 1) + [(hidden, n_out)]
    return dims


def n_params(dims) -> int:
    return sum(i * o + o for i, o in dims)


def unpack(theta: np.ndarray, dims) -> list[tuple[np.ndarray, np.ndarray]]:
    """Flat parameter vector -> [(W_l [out][in], b_l [out])], layer by layer, W before b."""
    out, p = [], 0
    for i, o in dims:
        w = theta[p:p + i * o].reshape(o, i)
        p += i * o
        b = theta[p:p + o]
        p += o
        out.append((w, b))
    assert p == theta.size
    return out


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (8-bit significand), ties to even.

    bfloat16 keeps the top 16 bits of the IEEE binary32 pattern; the discarded low
    half decides the rounding: above half -> up, below -> down, exactly half -> to the
    kept pattern with an even last bit. Finite inputs only.
    """
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    low = u & np.uint64(0xFFFF)
    keep = u >> np.uint64(16)
    half = np.uint64(0x8000)
    up = (low > half) | ((low == half) & ((keep & np.uint64(1)) == np.uint64(1)))
    keep = keep + up.astype(np.uint64)
    return (keep << np.uint64(16)).astype(np.uint32).view(np.float32)


def gelu(u: np.ndarray) -> np.ndarray:
    """GELU(u) = u Phi(u) = u (1 + erf(u / sqrt 2)) / 2."""
    return 0.5 * u * (1.0 + erf(u / math.sqrt(2.0)))


def gelu_grad(u: np.ndarray) -> np.ndarray:
    """d GELU / du = Phi(u) + u phi(u), phi the standard normal density."""
    return 0.5 * (1.0 + erf(u / math.sqrt(2.0))) + u * np.exp(-0.5 * u * u) / math.sqrt(2.0 * math.pi)


def effective_weights(theta: np.ndarray, dims, round_weights: bool = True):
    """Layers with each W replaced by its bfloat16 rounding (biases unchanged), in FP64."""
    layers = []
    for w, b in unpack(np.asarray(theta, dtype=np.float64), dims):
        wq = bf16_round(w.astype(np.float32)).astype(np.float64) if round_weights else w
        layers.append((wq, b.astype(np.float64)))
    return layers


def forward(theta, dims, x, round_weights: bool = True, round_act: bool = False):
    """Network outputs y [n][n_out] for inputs x [n][n_in], FP64.

    round_act rounds every layer's input to bfloat16 before it multiplies (what a
    bf16 x bf16 tensor-core product sees); the default keeps activations exact.
    Returns (y, cache) with cache = [(layer input, pre-activation)] for backward().
    """
    layers = effective_weights(theta, dims, round_weights)
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for li, (w, b) in enumerate(layers):
        a = bf16_round(h.astype(np.float32)).astype(np.float64) if round_act else h
        z = a @ w.T + b
        cache.append((a, z))
        h = gelu(z) if li < len(layers) - 1 else z
    return h, cache


def mse_loss(y: np.ndarray, t: np.ndarray) -> float:
    """Mean over samples and bins of (y - t)^2."""
    return float(np.mean((np.asarray(y, np.float64) - np.asarray(t, np.float64)) ** 2))


def loss_and_grad(theta, dims, x, t, round_weights: bool = True):
    """MSE loss and its gradient with respect to the flat parameter vector (FP64).

    Backpropagation by the chain rule: dL/dy = 2 (y - t) / (n n_out); for each layer
    from the last, dW = delta^T a, db = sum over samples of delta, and the error
    passed down is (delta W) * GELU'(z) of the layer below. The weight rounding is
    passed through unchanged.
    """
    layers = effective_weights(theta, dims, round_weights)
    y, cache = forward(theta, dims, x, round_weights)
    t = np.asarray(t, dtype=np.float64)
    loss = mse_loss(y, t)
    delta = 2.0 * (y - t) / y.size
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        a, _ = cache[li]
        w, _ = layers[li]
        grads[li] = (delta.T @ a, delta.sum(axis=0))
        if li > 0:
            delta = (delta @ w) * gelu_grad(cache[li - 1][1])
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, flat


def adam_step(theta, grad, m, v, step: int, lr: float):
    """One Adam update (step counts from 1). Returns new (theta, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * grad
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * grad * grad
    mh = m / (1.0 - ADAM_B1 ** step)
    vh = v / (1.0 - ADAM_B2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def features(params: np.ndarray, z: float, prior_lo, prior_hi, z_lo: float, z_hi: float) -> np.ndarray:
    """Network inputs of walkers params [n][3] at redshift z: each coordinate mapped
    linearly from its interval onto [-1, 1] (z from [z_lo, z_hi]; a single redshift
    maps to 0)."""
    p = np.asarray(params, dtype=np.float64)
    lo = np.asarray(prior_lo, dtype=np.float64)
    hi = np.asarray(prior_hi, dtype=np.float64)
    f = np.empty((p.shape[0], 4))
    f[:, :3] = 2.0 * (p - lo) / (hi - lo) - 1.0
    f[:, 3] = 0.0 if z_hi <= z_lo else 2.0 * (z - z_lo) / (z_hi - z_lo) - 1.0
    return f


def targets(d2: np.ndarray, floor: float) -> np.ndarray:
    """log10 of Delta^2 floored at `floor` (empty bins, NaN, also map to the floor)."""
    d = np.asarray(d2, dtype=np.float64)
    d = np.where(np.isfinite(d), d, floor)
    return np.log10(np.maximum(d, floor))


def predict_log10_d2(thetas, dims, x, mean, std, round_act: bool = True):
    """Ensemble prediction: per member log10 Delta^2 = mean + std y; returns the
    members' average [n][n_out] and the spread max_b (standard deviation over members)
    [n], both FP64."""
    preds = np.stack([mean + std * forward(th, dims, x, True, round_act)[0] for th in thetas])
    return preds.mean(axis=0), preds.std(axis=0).max(axis=1)
