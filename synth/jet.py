"""Taylor jets in (x, y, t) over numpy arrays.

A jet carries a value, its gradient with respect to (x, y, t) and its Hessian
with respect to (x, y), so
that analytic manufactured fields can be differentiated exactly (up to rounding)
when the momentum residual of Eq. (25) is evaluated at lattice nodes. This is
plain forward-mode automatic differentiation; it holds none of the lattice
Boltzmann arithmetic.
"""
from __future__ import annotations

import numpy as np

NV = 3  # gradient variables: x, y, t
NH = 2  # Hessian variables: x, y (Eq. (25) needs only first time derivatives)


class Jet:
    __slots__ = ("v", "g", "h")

    def __init__(self, v, g=None, h=None):
        v = np.asarray(v, dtype=np.float64)
        self.v = v
        self.g = g if g is not None else [np.zeros_like(v) for _ in range(NV)]
        self.h = h if h is not None else [[np.zeros_like(v) for _ in range(NH)] for _ in range(NH)]

    # -- constructors
    @staticmethod
    def var(v, k):
        v = np.asarray(v, dtype=np.float64)
        g = [np.zeros_like(v) for _ in range(NV)]
        g[k] = np.ones_like(v)
        return Jet(v, g)

    @staticmethod
    def const(c, like):
        return Jet(np.broadcast_to(np.asarray(c, dtype=np.float64), like.v.shape).copy())

    def _lift(self, o):
        return o if isinstance(o, Jet) else Jet.const(o, self)

    # -- a function f applied to the jet, given f, f', f'' at the value
    def _chain(self, f0, f1, f2):
        g = [f1 * gi for gi in self.g]
        h = [[f2 * self.g[i] * self.g[j] + f1 * self.h[i][j] for j in range(NH)]
             for i in range(NH)]
        return Jet(f0, g, h)

    # -- arithmetic
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

    def __rtruediv__(self, o):
        return self._lift(o) * self.recip()

    def __pow__(self, n: int):
        v = self.v
        return self._chain(v ** n, n * v ** (n - 1), n * (n - 1) * v ** (n - 2) if n >= 2 else 0.0 * v)

    # -- derivatives as plain arrays
    def dx(self):
        return self.g[0]

    def dy(self):
        return self.g[1]

    def dt(self):
        return self.g[2]


def sin(a: Jet) -> Jet:
    return a._chain(np.sin(a.v), np.cos(a.v), -np.sin(a.v))


def cos(a: Jet) -> Jet:
    return a._chain(np.cos(a.v), -np.sin(a.v), -np.cos(a.v))


def exp(a: Jet) -> Jet:
    e = np.exp(a.v)
    return a._chain(e, e, e)


def coordinates(nx: int, ny: int, t: float):
    """Jets for the lattice-node coordinates x, y (node indices) and time t."""
    yy, xx = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                         indexing="ij")
    return Jet.var(xx, 0), Jet.var(yy, 1), Jet.var(np.full_like(xx, float(t)), 2)


def grad_of_product_derivative(a: Jet, b: Jet, i: int, j: int):
    """d_i (a * d_j b) as a plain array (needs only second-order jets)."""
    return a.g[i] * b.g[j] + a.v * b.h[i][j]
