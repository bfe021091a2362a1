"""FP16 / BF16 storage with the momentum base (lbm_dev_base LBM_BASE_MOMENTUM, step
kernel 5): each slot holds its deviation from f_i^rest + 3 w_i e_i . J, the linear term
of the Eq. (14) equilibrium with J the post-collision momentum of the cell holding the
slot, and J itself is stored (rounded) in two more planes of the buffer.

* against the FP64 oracle on random lattices (walls or periodic, ragged against the
  60-column tiles, moving phi, force fields, App. B, the drag, the moving wall), from
  the device's initial populations with the inputs rounded to FP32: the kernel-5
  bound of test_gpu_parity, K5 = 8 units of 2^-24 D per step, plus the storage's
  stochastic rounding, 2 spacings (2^-11 FP16, 2^-8 BF16) of D per step, D = max|f -
  f_rest| (the stored remainders are smaller than D, so the bound holds a fortiori);
* on a smooth flow the BF16 remainders, and so the error against the oracle, are
  several times smaller than with the rest base (measured ratio printed);
* macros, sums and checkpoints see the same populations; argument checks.
"""
import numpy as np
import pytest

from gpu_cases import random_case, rest_populations, total_force

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
K5 = 8
SPACING = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_02964_gb300 as pkg
    pkg.capi.load()
    return pkg


def _f32(case):
    r = lambda a: None if a is None else a.astype(np.float32).astype(np.float64)  # noqa: E731
    return dict(case, phi=r(case["phi"]), phin=r(case["phin"]), fb=r(case["fb"]))


def _run(P, O, nx, ny, case, steps, storage, wall_y, dev_base="momentum", eq_order=3, drag=None, uw=None,
         tau=0.8):
    case = _f32(case)
    lat = P.Lattice(nx, ny, tau, s_eps=1.2, s_q=1.4, bc_y="bounceback" if wall_y else "periodic", storage=storage,
                    eq_order=eq_order, dev_base=dev_base)
    assert lat.launch_shape()["threads"] == 32
    kw = {}
    if drag:
        lat.set_drag(*drag)
        kw.update(drag_d0=drag[0], drag_d1=drag[1], us_x=drag[2], us_y=drag[3])
    if uw:
        lat.set_moving_wall(*uw)
        kw.update(nee_top=1, uw_x=uw[0], uw_y=uw[1])
    lat.set_void_fraction(case["phi"], case["phin"])
    lat.set_body_force(case["g"][0], case["g"][1], case["fb"])
    lat.init_fields(case["rho"], case["ux"], case["uy"])
    prm = O.Params(nx=nx, ny=ny, **O.rates_from_tau(tau, s_eps=1.2, s_q=1.4), kappa=0.5, bc_y=int(wall_y),
                   eq_order=eq_order, **kw)
    f = lat.get_populations().cpu().numpy().astype(np.float64)
    fb = total_force(case)
    for k in range(steps):
        phin = case["phin"] if k == 0 else None
        if k == 1 and case["phin"] is not None:
            case = dict(case, phi=case["phin"], phin=None)
            fb = total_force(case)
        f = O.step(prm, f, case["phi"], phin, fb)
    lat.step(steps)
    lat.sync()
    fg = lat.get_populations().cpu().numpy()
    m = {k: v.cpu().numpy() for k, v in lat.macros().items()}
    mo = O.macros(prm, fg.astype(np.float64), case["phi"], fb)
    lat.close()
    return fg, f, case, m, mo


def _bound(fo, case, steps, storage):
    D = np.abs(fo - rest_populations(case["phi"])).max()
    return D, steps * (K5 * EPS32 + 2 * SPACING[storage]) * D


CASES = [
    # nx, ny, wall_y, unsteady, field, g
    (130, 40, True, True, True, (2e-5, -1e-5)),
    (61, 33, False, False, True, (0.0, 0.0)),
    (200, 70, True, False, False, (1e-5, 0.0)),
    (9, 5, False, True, False, (0.0, 3e-5)),
]


@pytest.mark.parametrize("nx,ny,wall_y,unsteady,field,g", CASES)
@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_momentum_base_matches_oracle(P, oracle_mod, nx, ny, wall_y, unsteady, field, g, storage):
    steps = 6
    case = random_case(nx, ny, seed=11 * nx + ny, wall_y=wall_y, unsteady=unsteady, field=field, g=g)
    fg, fo, case, m, mo = _run(P, oracle_mod, nx, ny, case, steps, storage, wall_y)
    D, tol = _bound(fo, case, steps, storage)
    err = np.abs(fg - fo).max()
    print(f"{storage} momentum base: {err / (steps * D):.2e} D per step (bound {tol / (steps * D):.2e})")
    assert err <= tol
    # the macroscopic fields of the same populations
    for k in ("rho", "ux", "uy"):
        assert np.abs(m[k] - mo[k]).max() <= 1e-12 * max(1.0, np.abs(mo[k]).max()), k


@pytest.mark.parametrize("variant", ["appb", "drag", "moving_wall"])
def test_momentum_base_variants_match_oracle(P, oracle_mod, variant):
    nx, ny, steps = 70, 29, 6
    case = random_case(nx, ny, seed=3, wall_y=True, unsteady=True, field=True, g=(1e-5, 0.0))
    kw = {"appb": dict(eq_order=2), "drag": dict(drag=(0.03, 0.4, 2e-3, -1e-3)),
          "moving_wall": dict(uw=(2e-3, 0.0))}[variant]
    fg, fo, case, _, _ = _run(P, oracle_mod, nx, ny, case, steps, "bf16", True, **kw)
    _, tol = _bound(fo, case, steps, "bf16")
    assert np.abs(fg - fo).max() <= tol


def _smooth_case(nx, ny):
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    phi = 0.7 + 0.1 * np.sin(kx * x) * np.cos(ky * y)
    return dict(phi=phi, phin=None, rho=np.ones((ny, nx)), ux=0.04 + 0.01 * np.sin(ky * y),
                uy=0.01 * np.cos(kx * x), fb=None, g=(0.0, 0.0))


def test_momentum_base_shrinks_the_bf16_rounding(P, oracle_mod):
    """A smooth periodic flow with a mean velocity, 200 steps: with the momentum base
    the BF16 populations stay several times closer to the oracle's than with the rest
    base (the stored remainders are the higher-order and non-equilibrium parts)."""
    nx, ny, steps = 128, 96, 200
    errs = {}
    for base in ("rest", "momentum"):
        fg, fo, case, _, _ = _run(P, oracle_mod, nx, ny, _smooth_case(nx, ny), steps, "bf16", False, dev_base=base)
        errs[base] = np.abs(fg - fo).max()
    print(f"BF16 after {steps} steps: rest base {errs['rest']:.3e}, momentum base {errs['momentum']:.3e} "
          f"(ratio {errs['rest'] / errs['momentum']:.1f})")
    assert errs["momentum"] * 3 < errs["rest"]


def test_momentum_base_sums_and_checkpoint(P):
    """lbm_vanse_step_sums of the momentum-base kernel: from the same populations
    (set_populations encodes against J = 0, the rest base's own values) its sums of
    the post-collision m_0, j equal the rest-base kernel's to FP32 rounding; a saved
    state continues bit for bit (the J planes are part of it); a rest-base lattice
    refuses it."""
    import torch
    nx, ny = 150, 50
    # periodic: the post-streaming populations carry the post-collision momentum
    case = _f32(random_case(nx, ny, seed=8, wall_y=False, unsteady=False, field=True, g=(1e-5, 0.0)))

    def make(base="momentum"):
        lat = P.Lattice(nx, ny, 0.7, s_eps=1.2, s_q=1.4, storage="bf16", dev_base=base)
        lat.set_void_fraction(case["phi"])
        lat.set_body_force(case["g"][0], case["g"][1], case["fb"])
        lat.init_fields(case["rho"], case["ux"], case["uy"])
        return lat

    lat = make()
    ref = make("rest")
    ref.step(5)
    f0 = ref.get_populations()
    outs = []
    for L in (lat, ref):
        L.set_populations(f0)
        out = torch.zeros(3, dtype=torch.float64, device="cuda")
        L.step_sums(out)
        outs.append(out.cpu().numpy())
    ref.close()
    assert abs(outs[0][0] - outs[1][0]) <= 1e-12 * abs(outs[1][0])
    assert np.abs(outs[0][1:] - outs[1][1:]).max() <= 1e-9 * abs(outs[1][0])
    lat.step(5)
    state = lat.save_state()
    lat.step(40)
    want = lat.get_populations().cpu().numpy()
    lat.close()
    other = make()
    other.load_state(state)
    other.step(40)
    got = other.get_populations().cpu().numpy()
    other.close()
    assert np.array_equal(got, want)
    rest = make("rest")
    with pytest.raises(P.LbmError):
        rest.load_state(state)
    rest.close()


def test_momentum_base_argument_checks(P):
    for kw in (dict(storage="fp32"), dict(storage="fp64"), dict(storage="bf16", kernel=1),
               dict(storage="bf16", kernel=2), dict(storage="fp16", bc_x="bounceback", bc_y="bounceback")):
        with pytest.raises(P.LbmError):
            P.Lattice(16, 8, 0.8, dev_base="momentum", **kw)
    lat = P.Lattice(16, 8, 0.8, storage="bf16", dev_base="momentum")
    with pytest.raises(P.LbmError):
        lat.set_solid_cells()
    lat.close()
