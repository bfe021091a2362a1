"""Seeded synthetic void fraction for the 3-D channel workload.

``channel3d_fields(n)`` returns (phi, g) for an n^3 porous channel, the 3-D form of
the 2-D channel recipe: a periodic Gaussian random field (white noise filtered in
Fourier space by exp(-|k|^2 l^2 / 2), l = 16 cells) mapped affinely onto
[0.35, 1.0], a cube block [0.4 n, 0.6 n)^3 holding 0.4 with two ramp layers
(0.8, 0.6) and an 8-cell collar of 1.0 around it, and the body acceleration
g = 1e-6 along x. Fields are shaped [nz, ny, nx]. This module holds none of the
lattice Boltzmann arithmetic.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 2409


def gaussian_random_field3d(n: int, corr: float = 16.0, seed: int = DEFAULT_SEED) -> np.ndarray:
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n, n, n)).astype(np.float32)
    k = 2.0 * np.pi * np.fft.fftfreq(n)
    kr = 2.0 * np.pi * np.fft.rfftfreq(n)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + kr[None, None, :] ** 2
    spec = np.fft.rfftn(noise) * np.exp(-0.5 * k2 * corr * corr)
    return np.fft.irfftn(spec, s=(n, n, n), axes=(0, 1, 2))


def channel3d_fields(n: int, seed: int = DEFAULT_SEED, lo: float = 0.35, hi: float = 1.0, g: float = 1e-6):
    f = gaussian_random_field3d(n, seed=seed)
    phi = lo + (hi - lo) * (f - f.min()) / (f.max() - f.min())
    a, b = int(round(0.4 * n)), int(round(0.6 * n))
    idx = np.arange(n)
    d1 = np.minimum(idx - a, b - 1 - idx)          # depth inside the block along one axis
    depth = np.minimum(np.minimum(d1[:, None, None], d1[None, :, None]), d1[None, None, :])
    phi[(depth < 0) & (depth >= -8)] = hi
    for d in range(2):
        phi[depth == d] = hi - (hi - 0.4) * (d + 1) / 3
    phi[depth >= 2] = 0.4
    return np.ascontiguousarray(phi, dtype=np.float64), g
