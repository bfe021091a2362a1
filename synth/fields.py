"""Seeded synthetic void-fraction fields for the channel workloads.

``channel_phi(nx, ny, seed)`` builds the porous channel field: a periodic
Gaussian random field (white noise filtered in Fourier space by
exp(-|k|^2 l^2 / 2), correlation length l = 32 cells), mapped affinely onto
[0.35, 1.0], with a sharp block embedded after Eq. (24): the block
[0.4 nx, 0.6 nx) x [0.4 ny, 0.6 ny) holds 0.4, its two outer layers ramp
1.0 -> 0.4 (values 0.8, 0.6), and a 16-cell collar around it is set to 1.0.
Because the filter is applied spectrally, the field is periodic at every size.

This module holds none of the lattice Boltzmann arithmetic.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 2409


def gaussian_random_field(nx: int, ny: int, corr: float = 32.0, seed: int = DEFAULT_SEED) -> np.ndarray:
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((ny, nx))
    kx = 2.0 * np.pi * np.fft.rfftfreq(nx)
    ky = 2.0 * np.pi * np.fft.fftfreq(ny)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    spec = np.fft.rfft2(noise) * np.exp(-0.5 * k2 * corr * corr)
    return np.fft.irfft2(spec, s=(ny, nx))


def embed_block(phi: np.ndarray, inner: float = 0.4, outer: float = 1.0, collar: int = 16,
                ramp: int = 2) -> np.ndarray:
    ny, nx = phi.shape
    x0, x1 = int(round(0.4 * nx)), int(round(0.6 * nx))
    y0, y1 = int(round(0.4 * ny)), int(round(0.6 * ny))
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    # Chebyshev depth inside the block (0 on its outer layer), negative outside
    dx = np.minimum(xx - x0, x1 - 1 - xx)
    dy = np.minimum(yy - y0, y1 - 1 - yy)
    depth = np.minimum(dx, dy)
    out = phi.copy()
    out[(depth < 0) & (depth >= -collar)] = outer
    for d in range(ramp):
        out[depth == d] = outer - (outer - inner) * (d + 1) / (ramp + 1)
    out[depth >= ramp] = inner
    return out


def channel_phi(nx: int, ny: int, seed: int = DEFAULT_SEED, lo: float = 0.35, hi: float = 1.0,
                corr: float = 32.0, block: bool = True) -> np.ndarray:
    g = gaussian_random_field(nx, ny, corr, seed)
    g = lo + (hi - lo) * (g - g.min()) / (g.max() - g.min())
    return embed_block(g) if block else g


def rest_fields(nx: int, ny: int, rho0: float = 1.0):
    """rho = rho0, u = 0 everywhere (a channel starting from rest)."""
    return (np.full((ny, nx), rho0), np.zeros((ny, nx)), np.zeros((ny, nx)))


def batch_lattices(count: int = 512, seed: int = DEFAULT_SEED):
    """The batched workload's lattices: n uniform over {32, 48, ..., 1024}, tau ~
    U[0.55, 1.5], amplitude A ~ U[0.05, 0.3] of the spatiotemporal manufactured
    solution, with the diffusive scaling T = 1000 (n/64)^2, U0 = 0.01 (64/n).
    Returns (n, tau, A, T, U0) per lattice."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(np.arange(32, 1025, 16), size=count)
    taus = rng.uniform(0.55, 1.5, size=count)
    amps = rng.uniform(0.05, 0.3, size=count)
    return [(int(n), float(t), float(a), 1000.0 * (n / 64) ** 2, 0.01 * 64 / n)
            for n, t, a in zip(sizes, taus, amps)]
