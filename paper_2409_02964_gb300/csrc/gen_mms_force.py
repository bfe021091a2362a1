#!/usr/bin/env python3
"""Generate mms_force.cuh: the body force of Eq. (25) for the spatiotemporal
manufactured solution, evaluated inside the batched kernel.

Fields (lattice units, n x n periodic lattice, k = 2 pi / n, w = 2 pi / T):
    phi = phi0 + A sin(kx) sin(ky) cos(wt)
    q = phi u = grad psi + rot Psi,  psi = -(A w sin(wt) / (2 k^2)) sin(kx) sin(ky),
                                     Psi = (U0 / k) sin(kx) sin(ky)
so that d_t phi + div q = 0 with rho = rho0; the force is Eq. (25) with the pressure
term dropped (constant density):
    F / rho0 = d_t q + div(q u) - nu div(phi tau),  tau = grad u + grad u^T - (2/3) div u I.

The emitted code evaluates this in a structured way rather than as one expanded
rational expression: phi and q with their first and second derivatives are short
products of sin/cos of kx, ky (the arguments sx, cx, sy, cy) with step constants;
u = q / phi and its derivatives follow from the quotient rule with one reciprocal;
the force is then assembled from those. At generation time the structured result
is checked against the direct symbolic derivation (sympy) at random points.

Run from this directory:  python gen_mms_force.py  (needs sympy; the generated
header is committed, so building the library does not).
"""
import os
import random

import sympy as sp


def direct_force():
    """Eq. (25) by symbolic differentiation of the fields (the reference form)."""
    x, y, t = sp.symbols("x y t", real=True)
    k, w, A, U0, phi0, nu = sp.symbols("k w A U0 phi0 nu", positive=True)
    s_x, s_y, c_x, c_y = sp.sin(k * x), sp.sin(k * y), sp.cos(k * x), sp.cos(k * y)
    phi = phi0 + A * s_x * s_y * sp.cos(w * t)
    b = -(A * w / (2 * k)) * sp.sin(w * t)
    qx = b * c_x * s_y + U0 * s_x * c_y
    qy = b * s_x * c_y - U0 * c_x * s_y
    ux, uy = qx / phi, qy / phi
    div = sp.diff(ux, x) + sp.diff(uy, y)
    txx = 2 * sp.diff(ux, x) - sp.Rational(2, 3) * div
    tyy = 2 * sp.diff(uy, y) - sp.Rational(2, 3) * div
    txy = sp.diff(ux, y) + sp.diff(uy, x)
    Fx = sp.diff(qx, t) + sp.diff(qx * ux, x) + sp.diff(qx * uy, y) - nu * (sp.diff(phi * txx, x) + sp.diff(phi * txy, y))
    Fy = sp.diff(qy, t) + sp.diff(qy * ux, x) + sp.diff(qy * uy, y) - nu * (sp.diff(phi * txy, x) + sp.diff(phi * tyy, y))
    return (x, y, t, k, w, A, U0, phi0, nu), Fx, Fy


# The structured evaluation: (name, kind, expression text). kind "s" = float scalar
# (uniform per lattice and step), "v" = per-cell value of type T. Expressions use the
# inputs sx, cx, sy, cy (T), ct, st, k, w, A, U0, phi0, nu (float) and earlier names.
STEPS = [
    # step constants
    ("a", "s", "A * ct"),                        # phi = phi0 + a sx sy
    ("b", "s", "-(A * w * st) / (2 * k)"),       # q_x = b cx sy + U0 sx cy, q_y = b sx cy - U0 cx sy
    ("bt", "s", "-(A * w * w * ct) / (2 * k)"),  # d_t b
    ("ak", "s", "a * k"),
    ("akk", "s", "a * k * k"),
    ("bk", "s", "b * k"),
    ("uk", "s", "U0 * k"),
    ("kk", "s", "k * k"),
    # products of the trig arguments
    ("ss", "v", "sx * sy"),
    ("cc", "v", "cx * cy"),
    ("cs", "v", "cx * sy"),
    ("sc", "v", "sx * cy"),
    # phi and its derivatives
    ("ph", "v", "phi0 + a * ss"),
    ("phx", "v", "ak * cs"),
    ("phy", "v", "ak * sc"),
    ("phxx", "v", "-akk * ss"),                 # = phi_yy
    ("phxy", "v", "akk * cc"),
    # q and its derivatives
    ("qx", "v", "b * cs + U0 * sc"),
    ("qy", "v", "b * sc - U0 * cs"),
    ("qxt", "v", "bt * cs"),
    ("qyt", "v", "bt * sc"),
    ("qxx", "v", "uk * cc - bk * ss"),          # d_x q_x
    ("qxy", "v", "bk * cc - uk * ss"),          # d_y q_x
    ("qyx", "v", "bk * cc + uk * ss"),          # d_x q_y
    ("qyy", "v", "-bk * ss - uk * cc"),         # d_y q_y
    ("qmx", "v", "-kk * (b * sc + U0 * cs)"),   # d_x d_y q_x
    ("qmy", "v", "kk * (U0 * sc - b * cs)"),    # d_x d_y q_y  (d_xx q = d_yy q = -k^2 q)
    # u = q / phi and its derivatives (quotient rule)
    ("ip", "v", "1 / ph"),
    ("ux", "v", "qx * ip"),
    ("uy", "v", "qy * ip"),
    ("uxx", "v", "(qxx - ux * phx) * ip"),
    ("uxy", "v", "(qxy - ux * phy) * ip"),
    ("uyx", "v", "(qyx - uy * phx) * ip"),
    ("uyy", "v", "(qyy - uy * phy) * ip"),
    ("uxXX", "v", "(-kk * qx - 2 * uxx * phx - ux * phxx) * ip"),
    ("uxYY", "v", "(-kk * qx - 2 * uxy * phy - ux * phxx) * ip"),
    ("uxXY", "v", "(qmx - uxx * phy - uxy * phx - ux * phxy) * ip"),
    ("uyXX", "v", "(-kk * qy - 2 * uyx * phx - uy * phxx) * ip"),
    ("uyYY", "v", "(-kk * qy - 2 * uyy * phy - uy * phxx) * ip"),
    ("uyXY", "v", "(qmy - uyx * phy - uyy * phx - uy * phxy) * ip"),
    # viscous stress and its divergence terms
    ("dv", "v", "uxx + uyy"),
    ("txx", "v", "2 * uxx - (2.0 / 3.0) * dv"),
    ("tyy", "v", "2 * uyy - (2.0 / 3.0) * dv"),
    ("txy", "v", "uxy + uyx"),
    ("dxtxx", "v", "(4.0 / 3.0) * uxXX - (2.0 / 3.0) * uyXY"),
    ("dytyy", "v", "(4.0 / 3.0) * uyYY - (2.0 / 3.0) * uxXY"),
    ("dytxy", "v", "uxYY + uyXY"),
    ("dxtxy", "v", "uxXY + uyXX"),
    ("vx", "v", "phx * txx + ph * dxtxx + phy * txy + ph * dytxy"),
    ("vy", "v", "phx * txy + ph * dxtxy + phy * tyy + ph * dytyy"),
    # Eq. (25) without the pressure term, per unit rho0
    ("fx", "out", "qxt + qxx * ux + qx * uxx + qxy * uy + qx * uyy - nu * vx"),
    ("fy", "out", "qyt + qyx * ux + qy * uxx + qyy * uy + qy * uyy - nu * vy"),
]

INPUTS_V = ("sx", "cx", "sy", "cy")
INPUTS_S = ("ct", "st", "k", "w", "A", "U0", "phi0", "nu")


def check_against_direct(trials: int = 12) -> float:
    """Largest relative difference between the structured and the direct force."""
    syms, Fx, Fy = direct_force()
    x, y, t, k, w, A, U0, phi0, nu = syms
    rng = random.Random(2409)
    worst = 0.0
    for _ in range(trials):
        vals = {k: 2 * 3.141592653589793 / rng.choice([16, 32, 48, 64]), w: 2 * 3.141592653589793 / rng.uniform(200, 3000),
                A: rng.uniform(0.05, 0.3), U0: rng.uniform(0.0, 0.02), phi0: 0.7, nu: rng.uniform(0.02, 0.3),
                x: rng.uniform(0, 64), y: rng.uniform(0, 64), t: rng.uniform(0, 5000)}
        ref = [sp.N(F.subs(vals), 30) for F in (Fx, Fy)]
        env = {"sx": sp.sin(vals[k] * vals[x]), "cx": sp.cos(vals[k] * vals[x]), "sy": sp.sin(vals[k] * vals[y]),
               "cy": sp.cos(vals[k] * vals[y]), "ct": sp.cos(vals[w] * vals[t]), "st": sp.sin(vals[w] * vals[t]),
               "k": vals[k], "w": vals[w], "A": vals[A], "U0": vals[U0], "phi0": vals[phi0], "nu": vals[nu]}
        for name, _, expr in STEPS:
            env[name] = sp.N(sp.sympify(expr, locals=dict(env)), 30)
        scale = max(abs(r) for r in ref) or 1
        for got, want in zip((env["fx"], env["fy"]), ref):
            worst = max(worst, float(abs(got - want) / scale))
    return worst


def emit(expr: str, kind: str) -> str:
    """C++ text: numbers as float literals, 1 / T as mms_rcp(T)."""
    import re
    text = expr.replace("1 / ph", "mms_rcp(ph)")
    text = re.sub(r"(?<![\w.])(\d+\.\d+|\d+)(?![\w.])", lambda m: f"{float(m.group(1))!r}f", text)
    return text


def main() -> None:
    err = check_against_direct()
    assert err < 1e-12, f"structured force differs from the direct derivation by {err}"
    lines = []
    for name, kind, expr in STEPS:
        if kind == "s":
            lines.append(f"    const float {name} = {emit(expr, kind)};")
        elif kind == "v":
            lines.append(f"    const T {name} = {emit(expr, kind)};")
        else:
            lines.append(f"    {name} = {emit(expr, kind)};")
    body = "\n".join(lines)
    text = f'''// mms_force.cuh -- GENERATED by gen_mms_force.py; do not edit by hand.
//
// Body force of Eq. (25) (constant density, pressure term dropped) for the
// spatiotemporal manufactured solution phi = phi0 + A sin(kx) sin(ky) cos(wt),
// phi u = grad psi + rot Psi (see the generator for the definitions), per unit rho0.
// Arguments: sx, cx = sin, cos of k x; sy, cy = sin, cos of k y; ct, st = cos, sin
// of w t. Evaluated from phi, q = phi u and their derivatives, u by the quotient rule.
// T is the arithmetic type (float or a packed pair); it must provide + - * between
// T values and with a float on either side, unary -, and mms_rcp(T).
#pragma once

namespace lbmv {{

template <typename T>
__device__ __forceinline__ void mms_force(T sx, T cx, T sy, T cy, float ct, float st, float k, float w, float A,
                                          float U0, float phi0, float nu, T& fx, T& fy) {{
{body}
}}

}}  // namespace lbmv
'''
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mms_force.cuh")
    with open(out, "w") as fh:
        fh.write(text)
    print(out, f"{len(STEPS)} steps, structured vs direct: {err:.1e}")


if __name__ == "__main__":
    main()
