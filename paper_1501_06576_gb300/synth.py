"""Seeded synthetic inputs for the excursion-set 21-cm likelihood path.

This module makes the INPUTS that the CUDA library and the CPU oracle both
consume, and nothing else: it holds no step of the method (no filtering,
collapsed fraction, ionization, brightness temperature, power spectrum or
chi^2). Neither the library nor the oracle imports it for any of their own
arithmetic.

What it makes (the workloads stand in for the paper's Zel'dovich-evolved
21CMFAST density boxes of Sec. 2.5, which need the 768^3 initial-condition
pipeline and are not reproduced here):

* density boxes: a Gaussian random field with a BBKS LCDM spectrum, normalised
  to sigma_8, grown linearly to redshift z and clipped at delta > -1, stored as
  FP32 in row-major (x, y, z) order;
* walker parameters: (zeta, R_mfp, log10 T_vir) drawn uniformly in a box;
* parameter vectors of the surrogate network (test inputs).

All random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea & Flood 2014, "Fast splittable pseudorandom number generators"), with
Box-Muller for normal deviates, so a (seed, stream) pair gives the same box on
every machine and numpy version.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 sequence keyed by (seed, stream)."""
    key = _mix64(np.array([(seed * 0x100000001B3 + stream * 0x9E3779B1 + 1) & 0xFFFFFFFFFFFFFFFF],
                          dtype=np.uint64))[0]
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + idx * _GOLDEN)


def uniform01(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits."""
    u = splitmix64(seed, stream, count, offset)
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normals(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normal deviates by Box-Muller on consecutive pairs."""
    m = (count + 1) // 2
    u = splitmix64(seed, stream, 2 * m)
    u1 = ((u[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)  # (0, 1]
    u2 = (u[1::2] >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2.0 * np.pi * u2)
    out[1::2] = r * np.sin(2.0 * np.pi * u2)
    return out[:count]


# ---------------------------------------------------------------- input spectrum

def _bbks(q: np.ndarray) -> np.ndarray:
    q = np.maximum(q, 1e-30)
    poly = 1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4
    return np.log1p(2.34 * q) / (2.34 * q) * poly ** -0.25


class InputCosmology:
    """The spectrum the synthetic density boxes are drawn from (BBKS, sigma_8 normalised)."""

    def __init__(self, h=0.68, omega_m=0.31, n_s=0.96, sigma8=0.82):
        self.h, self.omega_m, self.n_s, self.sigma8 = h, omega_m, n_s, sigma8
        lnk = np.linspace(np.log(1e-6), np.log(1e4), 400001)
        k = np.exp(lnk)
        x = k * 8.0 / h
        w = np.where(x < 1e-3, 1.0 - x * x / 10.0, 3.0 * (np.sin(x) - x * np.cos(x)) / np.maximum(x, 1e-3) ** 3)
        integrand = k ** 3 * self._shape(k) * w * w / (2.0 * np.pi ** 2)
        self.amp = sigma8 ** 2 / np.trapezoid(integrand, lnk)

    def _shape(self, k):
        return k ** self.n_s * _bbks(k / (self.omega_m * self.h ** 2)) ** 2

    def pk(self, k):
        return self.amp * self._shape(np.asarray(k, dtype=np.float64))

    def growth(self, z: float) -> float:
        def unnorm(a):
            ap = np.linspace(0.0, a, 200001)[1:]
            e = np.sqrt(self.omega_m / ap ** 3 + 1.0 - self.omega_m)
            integ = np.concatenate([[0.0], 1.0 / (ap * e) ** 3])
            grid = np.concatenate([[0.0], ap])
            return np.sqrt(self.omega_m / a ** 3 + 1.0 - self.omega_m) * np.trapezoid(integ, grid)
        return unnorm(1.0 / (1.0 + z)) / unnorm(1.0)


def density_box(n: int, box_mpc: float, z: float, seed: int, stream: int = 0,
                cosmo: InputCosmology | None = None) -> np.ndarray:
    """Seeded Gaussian random field at redshift z, FP32 (n, n, n), clipped at delta > -1."""
    cosmo = cosmo or InputCosmology()
    w = normals(seed, stream, n ** 3).reshape(n, n, n)
    wk = np.fft.rfftn(w)
    m = np.fft.fftfreq(n, d=1.0 / n)
    mz = np.arange(n // 2 + 1, dtype=np.float64)
    kf = 2.0 * np.pi / box_mpc
    k = kf * np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2)
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = np.sqrt(n ** 3 * cosmo.pk(k[nz]) / box_mpc ** 3)
    delta = np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2)) * cosmo.growth(z)
    return np.maximum(delta, -1.0 + 1e-6).astype(np.float32)


def density_boxes(n: int, box_mpc: float, zs, seed: int) -> np.ndarray:
    """One independent box per redshift, keyed (seed, redshift index): (n_z, n, n, n) FP32."""
    cosmo = InputCosmology()
    return np.stack([density_box(n, box_mpc, z, seed, j, cosmo) for j, z in enumerate(zs)])


def walker_params(count: int, seed: int, zeta=(5.0, 100.0), r_mfp=(5.0, 20.0),
                  log10_tvir=(4.0, 6.0)) -> np.ndarray:
    """(count, 3) float64 rows (zeta, R_mfp [Mpc], log10 T_vir [K]) drawn uniformly."""
    u = uniform01(seed, 1000, 3 * count).reshape(count, 3)
    lo = np.array([zeta[0], r_mfp[0], log10_tvir[0]])
    hi = np.array([zeta[1], r_mfp[1], log10_tvir[1]])
    return lo + (hi - lo) * u


def mlp_params(seed: int, dims) -> np.ndarray:
    """Flat FP64 parameter vector of a multilayer perceptron with layers dims = [(fan_in,
    fan_out), ...], laid out layer by layer as W [fan_out][fan_in] then b [fan_out]: weights
    uniform on +-sqrt(3 / fan_in) (unit-variance pre-activations for unit inputs), biases
    normal with standard deviation 0.1. Test and initialisation inputs only."""
    parts = []
    for li, (fi, fo) in enumerate(dims):
        a = np.sqrt(3.0 / fi)
        parts.append((uniform01(seed, 2000 + 2 * li, fi * fo) * 2.0 - 1.0) * a)
        parts.append(0.1 * normals(seed, 2001 + 2 * li, fo))
    return np.concatenate(parts)


# Workloads (sizes and parameters of the hot path's configurations).
WORKLOADS = {
    "64cube_L100_z9": dict(n=64, box_mpc=100.0, zs=(9.0,), params=(30.0, 15.0, np.log10(3e4))),
    "128cube_L250_z8-9-10": dict(n=128, box_mpc=250.0, zs=(8.0, 9.0, 10.0), params=(30.0, 15.0, 4.7)),
}
