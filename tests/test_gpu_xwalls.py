"""Half-way bounce-back walls in x (bc_x = bounce-back, step kernel 1) against the
FP64 oracle, which applies the rule of the y walls to x (Sec. 3.1; the paper is
silent on the Eq. (10) stencil at a wall: the ghost cell mirrors the cell next to the
wall, vector components negated once, also past two walls at a corner).

Lattices with x walls alone and with walls on all four sides (corners), ragged
against kernel 1's 124-column tiles, one to three columns wide, with a moving phi and
per-cell force fields; the Eq. (14) and App. B equilibria and model B; a closed box
that conserves its mass to round-off; argument checks. Tolerances as in
test_gpu_parity: FP64 1e-12 of the largest deviation from rest, FP32 (kernel 1 collides
full populations) 32 * 2^-24 * max|f| per step.
"""
import numpy as np
import pytest

from gpu_cases import random_case, rest_populations, total_force

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_02964_gb300 as pkg
    pkg.capi.load()
    return pkg


def _case(nx, ny, seed, wall_y, unsteady, field, g):
    case = random_case(nx, ny, seed, wall_y=wall_y, unsteady=unsteady, field=field, g=g)
    x = np.arange(nx)[None, :]
    damp = np.sin(np.pi * (x + 0.5) / nx)   # velocities that vanish towards the x walls
    return dict(case, ux=case["ux"] * damp, uy=case["uy"] * damp)


def _run(P, O, nx, ny, case, steps, storage, wall_y, eq_order=3, model_b=False, tau=0.8):
    lat = P.Lattice(nx, ny, tau, s_eps=1.2, s_q=1.4, bc_x="bounceback", bc_y="bounceback" if wall_y else "periodic",
                    storage=storage, eq_order=eq_order, model_b=model_b)
    assert lat.launch_shape()["threads"] == 128   # kernel 1
    lat.set_void_fraction(case["phi"], case["phin"])
    lat.set_body_force(case["g"][0], case["g"][1], case["fb"])
    lat.init_fields(case["rho"], case["ux"], case["uy"])
    prm = O.Params(nx=nx, ny=ny, **O.rates_from_tau(tau, s_eps=1.2, s_q=1.4), kappa=0.5, bc_x=1, bc_y=int(wall_y),
                   eq_order=eq_order, model_b=int(model_b))
    fb = total_force(case)
    f = O.init(prm, case["rho"], case["ux"], case["uy"], case["phi"], fb)
    f0g = lat.get_populations().cpu().numpy()
    init_err = np.abs(f0g - f).max() / np.abs(f).max()
    for k in range(steps):
        phin = case["phin"] if k == 0 else None
        if k == 1 and case["phin"] is not None:
            case = dict(case, phi=case["phin"], phin=None)
            fb = total_force(case)
        f = O.step(prm, f, case["phi"], phin, fb)
    lat.step(steps)
    lat.sync()
    fg = lat.get_populations().cpu().numpy()
    lat.close()
    return init_err, fg, f, case


CASES = [
    # nx, ny, wall_y, unsteady, field, g
    (40, 23, False, True, True, (0.0, 2e-5)),
    (33, 17, True, False, False, (1e-5, -1e-5)),    # a closed box: four corners
    (130, 9, True, True, True, (0.0, 1e-5)),        # two CTAs in x, ragged tail
    (3, 12, True, False, True, (0.0, 0.0)),
    (1, 8, False, False, False, (0.0, 3e-5)),
    (2, 5, True, True, False, (0.0, 0.0)),
]


@pytest.mark.parametrize("nx,ny,wall_y,unsteady,field,g", CASES)
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_x_walls_match_oracle(P, oracle_mod, nx, ny, wall_y, unsteady, field, g, storage):
    steps = 6
    case = _case(nx, ny, 5 * nx + ny, wall_y, unsteady, field, g)
    init_err, fg, fo, case = _run(P, oracle_mod, nx, ny, case, steps, storage, wall_y)
    if storage == "fp64":
        assert init_err < 1e-14
        assert np.abs(fg - fo).max() / np.abs(fo - rest_populations(case["phi"])).max() <= 1e-12
    else:
        assert np.abs(fg - fo).max() <= steps * 32 * EPS32 * np.abs(fo).max()


@pytest.mark.parametrize("eq_order,model_b", [(2, False), (3, True)])
def test_x_walls_variants_match_oracle(P, oracle_mod, eq_order, model_b):
    nx, ny = 45, 21
    case = _case(nx, ny, 71, True, True, True, (1e-5, 1e-5))
    _, fg, fo, case = _run(P, oracle_mod, nx, ny, case, 5, "fp64", True, eq_order=eq_order, model_b=model_b)
    assert np.abs(fg - fo).max() / np.abs(fo - rest_populations(case["phi"])).max() <= 1e-12


def test_closed_box_conserves_mass_and_stays_at_rest(P):
    """Walls on four sides: the mass is conserved to round-off over 300 steps with a
    moving flow; a uniform rest state (phi not equal to kappa) stays at rest to
    round-off (the FP64 initial state and read-back leave |u| ~ 1e-19)."""
    nx, ny = 50, 30
    case = _case(nx, ny, 3, True, False, False, (0.0, 0.0))
    lat = P.Lattice(nx, ny, 0.7, bc_x="bounceback", bc_y="bounceback", storage="fp64")
    lat.set_void_fraction(case["phi"])
    lat.init_fields(case["rho"], case["ux"], case["uy"])
    m0, _, _ = lat.reduce()
    lat.step(300)
    m1, _, _ = lat.reduce()
    lat.close()
    assert abs(m1 - m0) <= 1e-13 * m0
    lat = P.Lattice(nx, ny, 0.7, bc_x="bounceback", bc_y="bounceback", storage="fp64")
    lat.set_void_fraction(np.full((ny, nx), 0.6))
    lat.init_fields(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    lat.step(50)
    m = lat.macros()
    lat.close()
    assert float(m["ux"].abs().max()) < 1e-15 and float(m["uy"].abs().max()) < 1e-15


def test_x_wall_argument_checks(P):
    for k in (2, 5):
        with pytest.raises(P.LbmError):
            P.Lattice(16, 8, 0.8, bc_x="bounceback", kernel=k)
    lat = P.Lattice(16, 8, 0.8, bc_x="bounceback", bc_y="bounceback")
    with pytest.raises(P.LbmError):
        lat.set_solid_cells()
    with pytest.raises(P.LbmError):
        lat.set_moving_wall(0.01, 0.0)
    lat.close()
