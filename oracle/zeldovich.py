"""FP64 CPU oracle of the Zel'dovich evolution of a density box.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this module. It shares no code with the
CUDA library and never calls it.

Sec. 2.1: the density field is a linear realization evolved with the Zel'dovich
approximation (Zel'dovich 1970). Every cell q of the n^3 grid carries one particle of
unit mass, displaced to x = q + psi(q) with the linear displacement

    psi(k) = i k / k^2 delta_L(k)        (so that delta = -div psi to first order),

and the particles are deposited back on the grid by cloud-in-cell weights with periodic
wrap: 1 + delta_nl(x) = sum over particles of the CIC weight. Readings (the paper is
silent): one particle per cell of the same grid (the paper's coarser smoothing grid is
not built); the displacement's Nyquist component along its own axis is set to zero (an
odd derivative has no Nyquist value). Pins (tests/test_oracle_zeldovich.py): zero field
-> zero; mass conservation; the displacement of a plane wave in closed form; the first-
order limit delta_nl -> delta_L for small amplitudes with an O(A^2) remainder; a uniform
translation leaves the field unchanged.
"""
from __future__ import annotations

import numpy as np


def displacement(delta_l: np.ndarray, box_mpc: float) -> np.ndarray:
    """psi [3][n][n][n] in grid units (cells) of the linear field delta_l [n][n][n]."""
    d = np.asarray(delta_l, dtype=np.float64)
    n = d.shape[0]
    dk = np.fft.fftn(d)
    m = np.fft.fftfreq(n, d=1.0 / n)
    mx, my, mz = np.meshgrid(m, m, m, indexing="ij")
    m2 = mx ** 2 + my ** 2 + mz ** 2
    m2[0, 0, 0] = 1.0
    kf = 2.0 * np.pi / box_mpc
    dx = box_mpc / n
    out = np.empty((3,) + d.shape)
    for j, mj in enumerate((mx, my, mz)):
        w = np.where(mj == -n // 2, 0.0, mj) / (kf * m2)   # k_j / k^2 [Mpc], Nyquist of the axis -> 0
        w[0, 0, 0] = 0.0
        out[j] = np.fft.ifftn(1j * w * dk).real / dx
    return out


def evolve(delta_l: np.ndarray, box_mpc: float) -> np.ndarray:
    """delta_nl [n][n][n] (FP64): CIC density of the Zel'dovich-displaced grid particles."""
    d = np.asarray(delta_l, dtype=np.float64)
    n = d.shape[0]
    psi = displacement(d, box_mpc)
    q = np.indices(d.shape).astype(np.float64)
    pos = (q + psi).reshape(3, -1)
    i0 = np.floor(pos).astype(np.int64)
    f = pos - i0
    rho = np.zeros(n ** 3)
    for cx in (0, 1):
        wx = f[0] if cx else 1.0 - f[0]
        for cy in (0, 1):
            wy = f[1] if cy else 1.0 - f[1]
            for cz in (0, 1):
                wz = f[2] if cz else 1.0 - f[2]
                idx = (((i0[0] + cx) % n) * n + (i0[1] + cy) % n) * n + (i0[2] + cz) % n
                np.add.at(rho, idx, wx * wy * wz)
    return rho.reshape(d.shape) - 1.0
