"""Shared set-ups for the GPU parity tests: the same seeded inputs go to the CUDA
library (through its C ABI binding) and to the FP64 oracle."""
from __future__ import annotations

import numpy as np

from synth import fields, mms

REST_W = np.array([0.0] + [1 / 9] * 4 + [1 / 36] * 4)


def rest_populations(phi, kappa=0.5, rho0=1.0):
    """f^rest of Eq. (14) at u = 0, rho = rho0 (used to scale population errors)."""
    f = np.empty((9,) + phi.shape)
    f[0] = (phi - 5 * kappa / 9) * rho0
    for i in range(1, 9):
        f[i] = REST_W[i] * kappa * rho0
    return f


def random_case(nx, ny, seed, wall_y=False, unsteady=False, field=False, g=(0.0, 0.0)):
    """Smooth random rho, u, phi fields (and phi(t+1), F^B field) on nx x ny."""
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    a = rng.uniform(0, 2 * np.pi, size=8)
    phi = 0.7 + 0.15 * np.sin(kx * x + a[0]) * np.cos(ky * y + a[1]) + 0.05 * rng.uniform(-1, 1, size=(ny, nx))
    rho = 1 + 0.01 * np.cos(kx * x + a[2]) * np.sin(ky * y + a[3])
    ux = 0.03 * np.sin(ky * y + a[4]) + 0.005 * rng.uniform(-1, 1, size=(ny, nx))
    uy = 0.02 * np.cos(kx * x + a[5]) + 0.005 * rng.uniform(-1, 1, size=(ny, nx))
    if wall_y:
        ux = ux * np.sin(np.pi * (y + 0.5) / ny)
        uy = uy * np.sin(np.pi * (y + 0.5) / ny)
    phin = phi + 0.01 * np.sin(kx * x + a[6]) if unsteady else None
    fb = rng.normal(size=(2, ny, nx)) * 1e-4 if field else None
    return dict(phi=phi, phin=phin, rho=rho, ux=ux, uy=uy, fb=fb, g=g)


def total_force(case):
    """F^B(x) = phi(x) g + field(x) as the oracle takes it."""
    phi = case["phi"]
    fb = np.stack([phi * case["g"][0], phi * case["g"][1]])
    if case["fb"] is not None:
        fb = fb + case["fb"]
    return fb


def config1(n=64):
    return mms.Config1(n=n)


# non-shear relaxation rates of the porous-channel workload
CHANNEL_RATES = dict(s_e=1.2, s_eps=1.2, s_q=1.2)


def channel_case(nx, ny, seed=fields.DEFAULT_SEED, g=1e-6):
    phi = fields.channel_phi(nx, ny, seed)
    rho, ux, uy = fields.rest_fields(nx, ny)
    return dict(phi=phi, phin=None, rho=rho, ux=ux, uy=uy, fb=None, g=(g, 0.0))
