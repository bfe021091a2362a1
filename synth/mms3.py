"""A 3-D manufactured solution for the D3Q19 extension of the VANSE scheme.

phi(x, t) = phi0 + A sin(kx) sin(ky) sin(kz) cos(wt), k = 2 pi / n, w = 2 pi / T, and
phi u = grad psi + v with lap psi = -d_t phi, so the continuity equation of Eq. (1)
holds with rho = rho0:

    psi = -(A w sin(wt)) / (3 k^2) sin(kx) sin(ky) sin(kz),
    v   = U0 (sin(ky), sin(kz), sin(kx))        (divergence-free, steady).

The body force is the momentum residual at these fields with constant density and
no pressure term (as Sec. 3.4 does in 2-D), for the viscous stress the 3-D scheme
recovers, tau = nu (grad u + grad u^T - 2/3 div u I) + 2/3 nu_e div u I,
evaluated exactly with Taylor jets. Lattice units: x, y, z are node indices, t is
the step count. This module holds none of the lattice Boltzmann arithmetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import jet3 as J


def _fields(n, T, A, U0, phi0, t, ops, coords):
    x, y, z = coords
    k = 2.0 * math.pi / n
    w = 2.0 * math.pi / T
    sx, sy, sz = ops.sin(k * x), ops.sin(k * y), ops.sin(k * z)
    cx, cy, cz = ops.cos(k * x), ops.cos(k * y), ops.cos(k * z)
    phi = phi0 + A * (sx * sy * sz) * math.cos(w * t)
    a = -(A * w * math.sin(w * t)) / (3.0 * k * k)
    # grad psi, written out
    gpx = a * k * (cx * sy * sz)
    gpy = a * k * (sx * cy * sz)
    gpz = a * k * (sx * sy * cz)
    px = gpx + U0 * sy
    py = gpy + U0 * sz
    pz = gpz + U0 * sx
    return phi, px / phi, py / phi, pz / phi


class _NpOps:
    sin = staticmethod(np.sin)
    cos = staticmethod(np.cos)


class _JetOps:
    sin = staticmethod(J.sin)
    cos = staticmethod(J.cos)


@dataclass
class Config3:
    n: int = 32
    T: float = 400.0
    A: float = 0.2
    U0: float = 0.01
    phi0: float = 0.7

    def _grid(self):
        zz, yy, xx = np.meshgrid(*(np.arange(self.n, dtype=np.float64),) * 3, indexing="ij")
        return xx, yy, zz

    def phi(self, t: float) -> np.ndarray:
        return _fields(self.n, self.T, self.A, self.U0, self.phi0, t, _NpOps, self._grid())[0]

    def velocity(self, t: float) -> np.ndarray:
        _, ux, uy, uz = _fields(self.n, self.T, self.A, self.U0, self.phi0, t, _NpOps, self._grid())
        return np.stack([ux, uy, uz])

    def _jets(self, t: float):
        x, y, z, tt = J.coordinates(self.n, self.n, self.n, t)
        # time enters through jets too, so d_t of every field is exact
        k = 2.0 * math.pi / self.n
        w = 2.0 * math.pi / self.T
        sx, sy, sz = J.sin(k * x), J.sin(k * y), J.sin(k * z)
        cx, cy, cz = J.cos(k * x), J.cos(k * y), J.cos(k * z)
        ct, st = J.cos(w * tt), J.sin(w * tt)
        phi = (sx * sy * sz) * ct * self.A + self.phi0
        a = st * (-(self.A * w) / (3.0 * k * k))
        px = a * (cx * sy * sz) * k + sy * self.U0
        py = a * (sx * cy * sz) * k + sz * self.U0
        pz = a * (sx * sy * cz) * k + sx * self.U0
        return phi, [px / phi, py / phi, pz / phi]

    def force(self, t: float, nu: float, nu_e: float = 0.0, rho0: float = 1.0) -> np.ndarray:
        """F = rho0 [d_t(phi u) + div(phi u u) - div(phi tau)], shaped [3, n, n, n]."""
        phi, u = self._jets(t)
        pu = [phi * ua for ua in u]
        div = u[0].g[0] + u[1].g[1] + u[2].g[2]
        out = []
        for a in range(3):
            conv = pu[a].g[3] + sum((pu[a] * u[b]).g[b] for b in range(3))
            # tau_ab = nu (d_b u_a + d_a u_b) + (2/3)(nu_e - nu) div u delta_ab
            lam = (2.0 / 3.0) * (nu_e - nu)
            vis = np.zeros_like(phi.v)
            for b in range(3):
                tab = nu * (u[a].g[b] + u[b].g[a]) + (lam * div if a == b else 0.0)
                # d_b tau_ab
                dtab = nu * (u[a].h[b][b] + u[b].h[a][b])
                if a == b:
                    dtab = dtab + lam * (u[0].h[0][b] + u[1].h[1][b] + u[2].h[2][b])
                vis = vis + phi.g[b] * tab + phi.v * dtab
            out.append(rho0 * (conv - vis))
        return np.stack(out)

    def continuity_residual(self, t: float) -> np.ndarray:
        phi, u = self._jets(t)
        return phi.g[3] + sum((phi * u[b]).g[b] for b in range(3))
