"""The oracle's x walls against its y walls by symmetry. Swapping x and y maps D2Q9
onto itself (E <-> N, W <-> S, NW <-> SE, the others fixed) and the scheme onto itself:
the rates of j_x, j_y and of q_x, q_y are equal, p_xx changes sign and p_xy does not,
both relaxed with s_nu, and Eq. (10), (13), (20) treat the axes alike. A lattice with
walls in x (and periodic or walled y) therefore steps exactly like the transposed
lattice with walls in y, cell by cell and population by population, up to rounding
(with a moving phi, a force field, App. B and model B; with walls on all four sides
the corners too). Pins the x-wall streaming and Eq. (10) ghost rule of the oracle
against its y-wall code."""
import numpy as np
import pytest

from gpu_cases import random_case, total_force

# population index after swapping x and y (order of Eq. 5: rest, E, N, W, S, NE, NW, SW, SE)
SWAP = [0, 2, 1, 4, 3, 5, 8, 7, 6]


def _transpose_case(case):
    t = lambda a: None if a is None else np.ascontiguousarray(a.T)  # noqa: E731
    fb = case["fb"]
    return dict(phi=t(case["phi"]), phin=t(case["phin"]), rho=t(case["rho"]), ux=t(case["uy"]), uy=t(case["ux"]),
                fb=None if fb is None else np.stack([fb[1].T, fb[0].T]), g=(case["g"][1], case["g"][0]))


def _run(O, prm, case, steps):
    fb = total_force(case)
    f = O.init(prm, case["rho"], case["ux"], case["uy"], case["phi"], fb)
    for k in range(steps):
        phin = case["phin"] if k == 0 else None
        if k == 1 and case["phin"] is not None:
            case = dict(case, phi=case["phin"], phin=None)
            fb = total_force(case)
        f = O.step(prm, f, case["phi"], phin, fb)
    return f


@pytest.mark.parametrize("nx,ny,walls_y,eq_order,model_b", [(17, 11, False, 3, False), (14, 9, True, 3, False),
                                                           (12, 13, True, 2, False), (10, 7, False, 3, True)])
def test_x_walls_equal_transposed_y_walls(oracle_mod, nx, ny, walls_y, eq_order, model_b):
    O = oracle_mod
    case = random_case(nx, ny, seed=nx * ny, wall_y=True, unsteady=True, field=True, g=(1e-5, 3e-5))
    x = np.arange(nx)[None, :]
    case = dict(case, ux=case["ux"] * np.sin(np.pi * (x + 0.5) / nx), uy=case["uy"] * np.sin(np.pi * (x + 0.5) / nx))
    rates = O.rates_from_tau(0.7, s_eps=1.2, s_q=1.4)
    pa = O.Params(nx=nx, ny=ny, **rates, kappa=0.5, bc_x=1, bc_y=int(walls_y), eq_order=eq_order, model_b=int(model_b))
    pb = O.Params(nx=ny, ny=nx, **rates, kappa=0.5, bc_x=int(walls_y), bc_y=1, eq_order=eq_order, model_b=int(model_b))
    fa = _run(O, pa, case, 8)
    fb = _run(O, pb, _transpose_case(case), 8)
    fb_back = np.stack([fb[SWAP[i]].T for i in range(9)])
    dev = np.abs(fa - fa.mean(axis=(1, 2), keepdims=True)).max()
    assert np.abs(fa - fb_back).max() <= 1e-13 * dev
    # and the walls matter: the same run with periodic x differs
    pp = O.Params(nx=nx, ny=ny, **rates, kappa=0.5, bc_x=0, bc_y=int(walls_y), eq_order=eq_order, model_b=int(model_b))
    assert np.abs(_run(O, pp, case, 8) - fa).max() > 1e-6 * dev
