"""Taylor jets in (x, y, z, t) over numpy arrays (the 3-D counterpart of ``synth.jet``).

A jet carries a value, its gradient with respect to (x, y, z, t) and its Hessian
with respect to (x, y, z): enough to evaluate a momentum residual with a viscous
term exactly (up to rounding) at lattice nodes. Plain forward-mode automatic
differentiation; no lattice Boltzmann arithmetic.
"""
from __future__ import annotations

import numpy as np

NV = 4  # x, y, z, t
NH = 3  # x, y, z


class Jet:
    __slots__ = ("v", "g", "h")

    def __init__(self, v, g=None, h=None):
        v = np.asarray(v, dtype=np.float64)
        self.v = v
        self.g = g if g is not None else [np.zeros_like(v) for _ in range(NV)]
        self.h = h if h is not None else [[np.zeros_like(v) for _ in range(NH)] for _ in range(NH)]

    @staticmethod
    def var(v, k):
        v = np.asarray(v, dtype=np.float64)
        g = [np.zeros_like(v) for _ in range(NV)]
        g[k] = np.ones_like(v)
        return Jet(v, g)

    def _lift(self, o):
        return o if isinstance(o, Jet) else Jet(np.broadcast_to(np.asarray(o, dtype=np.float64),
                                                                 self.v.shape).copy())

    def _chain(self, f0, f1, f2):
        g = [f1 * gi for gi in self.g]
        h = [[f2 * self.g[i] * self.g[j] + f1 * self.h[i][j] for j in range(NH)] for i in range(NH)]
        return Jet(f0, g, h)

    def __add__(self, o):
        if not isinstance(o, Jet):
            return Jet(self.v + o, list(self.g), [list(r) for r in self.h])
        return Jet(self.v + o.v, [a + b for a, b in zip(self.g, o.g)],
                   [[self.h[i][j] + o.h[i][j] for j in range(NH)] for i in range(NH)])

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.v, [-a for a in self.g], [[-self.h[i][j] for j in range(NH)] for i in range(NH)])

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return self._lift(o) - self

    def __mul__(self, o):
        if not isinstance(o, Jet):
            return Jet(self.v * o, [a * o for a in self.g], [[a * o for a in r] for r in self.h])
        g = [self.g[i] * o.v + self.v * o.g[i] for i in range(NV)]
        h = [[self.h[i][j] * o.v + self.g[i] * o.g[j] + self.g[j] * o.g[i] + self.v * o.h[i][j]
              for j in range(NH)] for i in range(NH)]
        return Jet(self.v * o.v, g, h)

    __rmul__ = __mul__

    def recip(self):
        v = self.v
        return self._chain(1.0 / v, -1.0 / v ** 2, 2.0 / v ** 3)

    def __truediv__(self, o):
        return self * self._lift(o).recip()


def sin(a: Jet) -> Jet:
    return a._chain(np.sin(a.v), np.cos(a.v), -np.sin(a.v))


def cos(a: Jet) -> Jet:
    return a._chain(np.cos(a.v), -np.sin(a.v), -np.cos(a.v))


def coordinates(nx: int, ny: int, nz: int, t: float):
    """Jets for the node coordinates (indices) x, y, z, shaped [nz, ny, nx], and time t."""
    zz, yy, xx = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                             np.arange(nx, dtype=np.float64), indexing="ij")
    return Jet.var(xx, 0), Jet.var(yy, 1), Jet.var(zz, 2), Jet.var(np.full_like(xx, float(t)), 3)
