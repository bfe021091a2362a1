"""Manufactured solutions for the VANSE convergence workloads (Sec. 3.4).

Each manufactured setting gives phi(x, y, t) and u(x, y, t) at lattice nodes and
the body force of Eq. (25), the momentum residual of Eq. (1) at those fields,
evaluated exactly with Taylor jets (``synth.jet``). As in Sec. 3.4 the density
is the constant rho0 and the pressure-gradient term is left out of the force.
Lattice units throughout: x, y are node indices, t is the step count.

Settings:
  * ``Config1``  phi = 0.7 + A sin(kx) sin(ky) cos(wt), k = 2 pi/n, w = 2 pi/T,
                 with phi u = grad psi + rot Psi (psi solves lap psi = -d_t phi, so
                 the continuity equation of Eq. (1) holds with rho = rho0) and a
                 steady solenoidal part Psi = (U0/k) sin(kx) sin(ky).
  * ``CaseI``    Eq. (27)        * ``CaseII``   Eq. (28)
  * ``CaseIII``  Eq. (29)-(30)

This module holds none of the lattice Boltzmann arithmetic: the oracle and the
CUDA library both take its arrays as inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from types import SimpleNamespace

import numpy as np

from . import jet as J

_JET_OPS = SimpleNamespace(sin=J.sin, cos=J.cos, exp=J.exp)
_NP_OPS = SimpleNamespace(sin=np.sin, cos=np.cos, exp=np.exp)


def _viscous_divergence(phi: J.Jet, ux: J.Jet, uy: J.Jet):
    """sum_beta d_beta(phi tau_ab), tau_ab = d_b u_a + d_a u_b - 2/3 delta_ab div u
    (Eq. 2 without rho), returned for a = x, y."""
    div = ux.g[0] + uy.g[1]
    txx = 2.0 * ux.g[0] - (2.0 / 3.0) * div
    tyy = 2.0 * uy.g[1] - (2.0 / 3.0) * div
    txy = ux.g[1] + uy.g[0]
    # d_b tau_ab = lap u_a + (1/3) d_a div u
    ddiv_x = ux.h[0][0] + uy.h[1][0]
    ddiv_y = ux.h[0][1] + uy.h[1][1]
    dtx = ux.h[0][0] + ux.h[1][1] + ddiv_x / 3.0
    dty = uy.h[0][0] + uy.h[1][1] + ddiv_y / 3.0
    vx = phi.g[0] * txx + phi.g[1] * txy + phi.v * dtx
    vy = phi.g[0] * txy + phi.g[1] * tyy + phi.v * dty
    return vx, vy


def residual_force(phi: J.Jet, ux: J.Jet, uy: J.Jet, nu: float, rho0: float = 1.0):
    """Eq. (25) with constant density rho0 and the pressure term dropped:
    F = rho0 [d_t(phi u) + div(phi u u) - nu div(phi tau)]."""
    pux = phi * ux
    puy = phi * uy
    fx = pux.g[2] + (pux * ux).g[0] + (pux * uy).g[1]
    fy = puy.g[2] + (puy * ux).g[0] + (puy * uy).g[1]
    vx, vy = _viscous_divergence(phi, ux, uy)
    return rho0 * (fx - nu * vx), rho0 * (fy - nu * vy)


def continuity_residual(phi: J.Jet, ux: J.Jet, uy: J.Jet):
    """d_t phi + div(phi u) (zero for a valid manufactured setting with rho const)."""
    return phi.g[2] + (phi * ux).g[0] + (phi * uy).g[1]


def _grid(nx: int, ny: int):
    yy, xx = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                         indexing="ij")
    return xx, yy


class Manufactured:
    """Base class: subclasses define ``_build(x, y, t, ops) -> (phi, ux, uy)``, written
    once and evaluated either on Taylor jets or on plain arrays."""
    n: int

    @property
    def nx(self):
        return self.n

    @property
    def ny(self):
        return self.n

    def _build(self, x, y, t, ops):  # pragma: no cover - abstract
        raise NotImplementedError

    def jets(self, t: float):
        x, y, tt = J.coordinates(self.nx, self.ny, t)
        return self._build(x, y, tt, _JET_OPS)

    def values(self, t: float):
        x, y = _grid(self.nx, self.ny)
        phi, ux, uy = self._build(x, y, float(t), _NP_OPS)
        shp = (self.ny, self.nx)
        return (np.broadcast_to(phi, shp).astype(np.float64),
                np.broadcast_to(ux, shp).astype(np.float64),
                np.broadcast_to(uy, shp).astype(np.float64))

    def phi(self, t: float) -> np.ndarray:
        return self.values(t)[0]

    def velocity(self, t: float):
        _, ux, uy = self.values(t)
        return ux, uy

    def force(self, t: float, nu: float, rho0: float = 1.0) -> np.ndarray:
        phi, ux, uy = self.jets(t)
        fx, fy = residual_force(phi, ux, uy, nu, rho0)
        return np.stack([fx, fy])


@dataclass
class Config1(Manufactured):
    """The spatiotemporal void-fraction workload: phi = phi0 + A sin sin cos(wt) on
    an n x n periodic lattice with period T steps."""
    n: int = 64
    T: float = 1000.0
    A: float = 0.2
    phi0: float = 0.7
    U0: float = 0.01

    @staticmethod
    def refined(n: int, n_ref: int = 64, T_ref: float = 1000.0, U0_ref: float = 0.01,
                A: float = 0.2):
        """Diffusive scaling: T ~ n^2, U0 ~ 1/n (so the Mach number falls with dx)."""
        s = n / n_ref
        return Config1(n=n, T=T_ref * s * s, A=A, U0=U0_ref / s)

    def _build(self, x, y, t, ops):
        k = 2.0 * math.pi / self.n
        w = 2.0 * math.pi / self.T
        sx, sy = ops.sin(k * x), ops.sin(k * y)
        cx, cy = ops.cos(k * x), ops.cos(k * y)
        phi = self.phi0 + self.A * sx * sy * ops.cos(w * t)
        a = -(self.A * w / (2.0 * k)) * ops.sin(w * t)
        qx = a * cx * sy + self.U0 * sx * cy
        qy = a * sx * cy - self.U0 * cx * sy
        return phi, qx / phi, qy / phi


def _star(x, n: int):
    return (2.0 * x - (n - 1)) / n


@dataclass
class CaseI(Manufactured):
    """Eq. (27): divergence-free velocity, steady void fraction."""
    n: int = 64
    a: float = 0.5
    b: float = 0.4
    us: float = 0.8

    def _build(self, x, y, t, ops):
        n = self.n
        X, Y = _star(x, n), _star(y, n)
        sx, sy = ops.sin(math.pi * X), ops.sin(math.pi * Y)
        cx, cy = ops.cos(math.pi * X), ops.cos(math.pi * Y)
        phi = self.a + self.b * sx * sy
        s = self.us / n
        return phi, -s * sx * sx * sy * cy, s * sy * sy * sx * cx


@dataclass
class CaseII(Manufactured):
    """Eq. (28): divergent velocity, steady void fraction."""
    n: int = 64
    a: float = 0.5
    b: float = 0.3
    us: float = 0.8

    def _build(self, x, y, t, ops):
        n = self.n
        X, Y = _star(x, n), _star(y, n)
        ss = ops.sin(math.pi * X) * ops.sin(math.pi * Y)
        phi = self.a * ops.exp(-self.b * ss)
        u = (self.us / n) * ops.exp(self.b * ss)
        return phi, u, u


@dataclass
class CaseIII(Manufactured):
    """Eq. (29)-(30): void fraction travelling diagonally at 4 u_s t / n^2."""
    n: int = 64
    a: float = 0.5
    b: float = 0.25
    us: float = 0.08

    def _build(self, x, y, t, ops):
        n = self.n
        shift = (4.0 * self.us / (n * n)) * t
        X, Y = _star(x, n) + shift, _star(y, n) + shift
        phi = self.a + self.b * ops.sin(math.pi * X) * ops.sin(math.pi * Y)
        u = (self.us / n) * (1.0 / phi - 2.0)
        return phi, u, u


def relative_l2(ux, uy, ux_ref, uy_ref) -> float:
    """Eq. (26): sqrt(sum |u - u_ref|^2 / sum |u_ref|^2) over all nodes."""
    num = np.sum((ux - ux_ref) ** 2 + (uy - uy_ref) ** 2)
    den = np.sum(ux_ref ** 2 + uy_ref ** 2)
    return float(np.sqrt(num / den))
