#!/usr/bin/env python3
"""Generate mms_force.cuh: the body force of Eq. (25) for the spatiotemporal
manufactured solution, in closed form, for the batched kernel's in-kernel source.

Fields (lattice units, n x n periodic lattice, k = 2 pi / n, w = 2 pi / T):
    phi = phi0 + A sin(kx) sin(ky) cos(wt)
    phi u = grad psi + rot Psi,  psi = -(A w sin(wt) / (2 k^2)) sin(kx) sin(ky),
                                 Psi = (U0 / k) sin(kx) sin(ky)
so that d_t phi + div(phi u) = 0 with rho = rho0; the force is Eq. (25) with the
pressure term dropped (constant density). The derivatives are taken symbolically,
then sin/cos of kx, ky, wt are replaced by the arguments sx, cx, sy, cy, ct, st and
common subexpressions are shared. The emitted function is a template over the
arithmetic type, so the same code serves scalars and packed pairs.

Run from this directory:  python gen_mms_force.py  (needs sympy; the generated
header is committed, so building the library does not).
"""
import os

import sympy as sp


def main() -> None:
    x, y, t = sp.symbols("x y t", real=True)
    k, w, A, U0, phi0, nu = sp.symbols("k w A U0 phi0 nu", positive=True)
    sx, sy, cx, cy = sp.sin(k * x), sp.sin(k * y), sp.cos(k * x), sp.cos(k * y)
    phi = phi0 + A * sx * sy * sp.cos(w * t)
    a = -(A * w / (2 * k)) * sp.sin(w * t)
    qx = a * cx * sy + U0 * sx * cy
    qy = a * sx * cy - U0 * cx * sy
    ux, uy = qx / phi, qy / phi
    div = sp.diff(ux, x) + sp.diff(uy, y)
    txx = 2 * sp.diff(ux, x) - sp.Rational(2, 3) * div
    tyy = 2 * sp.diff(uy, y) - sp.Rational(2, 3) * div
    txy = sp.diff(ux, y) + sp.diff(uy, x)
    Fx = sp.diff(qx, t) + sp.diff(qx * ux, x) + sp.diff(qx * uy, y) - nu * (sp.diff(phi * txx, x) + sp.diff(phi * txy, y))
    Fy = sp.diff(qy, t) + sp.diff(qy * ux, x) + sp.diff(qy * uy, y) - nu * (sp.diff(phi * txy, x) + sp.diff(phi * tyy, y))
    Sx, Sy, Cx, Cy, Ct, St = sp.symbols("sx sy cx cy ct st")
    rep = {sp.sin(k * x): Sx, sp.sin(k * y): Sy, sp.cos(k * x): Cx, sp.cos(k * y): Cy,
           sp.cos(w * t): Ct, sp.sin(w * t): St}
    Fx = sp.together(Fx.subs(rep))
    Fy = sp.together(Fy.subs(rep))
    reps, (ex, ey) = sp.cse([Fx, Fy], symbols=sp.numbered_symbols("e"), optimizations="basic")

    scalars = {"k", "w", "A", "U0", "phi0", "nu", "ct", "st"}
    fields = {"sx", "sy", "cx", "cy"}

    def emit(expr) -> str:
        return _emit(sp.expand_power_base(expr), scalars, fields)

    lines = []
    for sym, e in reps:
        if _is_scalar(e, scalars):
            scalars.add(str(sym))
            lines.append(f"    const float {sym} = {emit(e)};")
        else:
            lines.append(f"    const T {sym} = {emit(e)};")
    lines.append(f"    fx = {emit(ex)};")
    lines.append(f"    fy = {emit(ey)};")
    body = "\n".join(lines)
    text = f'''// mms_force.cuh -- GENERATED by gen_mms_force.py; do not edit by hand.
//
// Body force of Eq. (25) (constant density, pressure term dropped) for the
// spatiotemporal manufactured solution phi = phi0 + A sin(kx) sin(ky) cos(wt),
// phi u = grad psi + rot Psi (see the generator for the definitions). Arguments:
// sx, cx = sin, cos of k x; sy, cy = sin, cos of k y; ct, st = cos, sin of w t.
// T is the arithmetic type (float or a packed pair); it must provide + and *
// between T values and with a float on either side, and mms_rcp(T).
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
    print(out, len(reps), "subexpressions")


def _emit(e, scalars, fields) -> str:
    """C++ text of a sympy expression over T (field symbols / subexpressions) and
    float scalars; divisions become multiplications by mms_rcp."""
    if e.is_Symbol:
        return str(e)
    if e.is_Number:
        return f"{float(e)!r}f"
    if e.is_Add:
        terms = [_emit(a, scalars, fields) for a in e.args]
        return "(" + " + ".join(terms) + ")"
    if e.is_Mul:
        num, den = [], []
        for a in e.args:
            if a.is_Pow and a.exp.is_Number and a.exp < 0:
                den.append(sp.Pow(a.base, -a.exp))
            else:
                num.append(a)
        # scalar factors first so that float * T products come out
        num.sort(key=lambda a: 0 if _is_scalar(a, scalars) else 1)
        parts = [_emit(a, scalars, fields) for a in num] or ["1.0f"]
        s = " * ".join(parts)
        if den:
            d = " * ".join(_emit(a, scalars, fields) for a in den)
            s = f"({s}) * mms_rcp({d})"
        return "(" + s + ")"
    if e.is_Pow:
        b, p = e.base, e.exp
        if p.is_Integer and p > 0:
            return "(" + " * ".join([_emit(b, scalars, fields)] * int(p)) + ")"
        if p.is_Integer and p < 0:
            return f"mms_rcp({_emit(sp.Pow(b, -p), scalars, fields)})"
        raise ValueError(f"unsupported power {e}")
    raise ValueError(f"unsupported expression {e} ({type(e)})")


def _is_scalar(e, scalars) -> bool:
    return all(str(s) in scalars for s in e.free_symbols) if e.free_symbols else True


if __name__ == "__main__":
    main()
