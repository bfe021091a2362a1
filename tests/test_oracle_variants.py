"""Pins of the oracle's physics variants:

App. B (eq_order = 2): the 2nd-order equilibrium (B1) against its printed moments
(B2); the exact reduction to a textbook BGK with Guo forcing at phi = kappa (where
(B3) vanishes and (B1) is the textbook equilibrium of density kappa rho); the bulk
viscosity nu_e = nu/3 through sound damping at uniform phi != kappa (sensitive to
the div(phi rho u) coefficient of C_a); second-order convergence on the
spatiotemporal manufactured solution (sensitive to C_b and C_c).

Linear drag F^B = phi G - beta (u - u_s), beta = phi^2 (d0 + d1 (1 - phi)), with u
solved implicitly (reading c8): the Darcy-Brinkman channel of Eq. (21)-(22 I)
against its analytic profile, converging at second order; the nonuniform particle
flow of Eq. (23) (steady, u_s = 0) against u = G / (a phi); the momentum balance
sum j(t+1) - sum j(t) = sum F(t) with the drag inside F.
"""
import numpy as np
import pytest

from synth import mms

from test_oracle_step import _textbook_bgk_guo_step

E = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])


def test_appb_equilibrium_has_the_printed_moments(oracle_mod):
    M = oracle_mod.M()
    rng = np.random.default_rng(21)
    for _ in range(50):
        kappa, phi = rng.uniform(0.3, 1.0), rng.uniform(0.2, 1.0)
        rho, ux, uy = rng.uniform(0.8, 1.2), rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1)
        f = oracle_mod.feq(kappa, phi, rho, ux, uy, order=2)
        m = oracle_mod.meq(kappa, phi, rho, ux, uy, order=2)
        pr, X, uu = phi * rho, kappa / phi, ux * ux + uy * uy
        printed = pr * np.array([1, -4 + 3 * uu + 2 * X, 4 - 3 * uu - 3 * X, ux, -ux, uy, -uy, ux * ux - uy * uy,
                                 ux * uy])
        assert np.abs(M @ f - m).max() < 1e-14
        assert np.abs(m - printed).max() < 1e-14


@pytest.mark.parametrize("wall_y", [0, 1])
def test_appb_reduces_to_textbook_bgk_when_phi_equals_kappa(oracle_mod, wall_y):
    ny, nx = 9, 11
    kappa = 0.5
    s = 1 / 0.7
    p = oracle_mod.Params(nx=nx, ny=ny, s_nu=s, s_e=s, s_eps=s, s_q=s, s_c=s, kappa=kappa, bc_y=wall_y,
                          eq_order=2)
    rng = np.random.default_rng(12)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    phi = np.full((ny, nx), kappa)
    rho = 1 + 0.01 * np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * y / ny)
    ux = 0.03 * np.cos(2 * np.pi * y / ny)
    uy = 0.02 * np.sin(2 * np.pi * x / nx)
    fb = rng.normal(size=(2, ny, nx)) * 1e-4
    f = oracle_mod.init(p, rho, ux, uy, phi, fb)
    g = f.copy()
    for _ in range(25):
        f = oracle_mod.step(p, f, phi, None, fb)
        g = _textbook_bgk_guo_step(g, s, fb, wall_y)
    assert np.abs(f - g).max() < 1e-14


@pytest.mark.parametrize("phi0", [0.8, 0.35])
def test_appb_sound_wave_damping_pins_bulk_viscosity(oracle_mod, phi0):
    n, tau = 64, 0.8
    nu = (tau - 0.5) / 3
    p = oracle_mod.Params(nx=n, ny=1, **oracle_mod.rates_from_tau(tau), kappa=0.5, eq_order=2)
    x = np.arange(n, dtype=float)[None, :]
    k = 2 * np.pi / n
    phi = np.full((1, n), phi0)
    f = oracle_mod.init(p, 1 + 1e-4 * np.cos(k * x), np.zeros((1, n)), np.zeros((1, n)), phi)
    amps, steps = [], [0, 400, 800, 1200]
    for t in range(steps[-1] + 1):
        if t in steps:
            m = oracle_mod.macros(p, f, phi)
            a_rho = 2 / n * np.sum((m["rho"] - 1) * np.cos(k * x))
            a_u = 2 / n * np.sum(m["ux"] * np.sin(k * x))
            amps.append(np.sqrt(a_rho ** 2 + 3 * a_u ** 2))
        f = oracle_mod.step(p, f, phi)
    rate = -np.polyfit(steps, np.log(amps), 1)[0]
    assert abs(rate / ((2.0 / 3.0) * nu * k * k) - 1) < 0.05


def _mms_error(oracle_mod, n, order):
    M = mms.Config1.refined(n)
    tau = 0.8
    nu = (tau - 0.5) / 3
    p = oracle_mod.Params(nx=n, ny=n, **oracle_mod.rates_from_tau(tau, s_eps=1.2, s_q=1.2), kappa=0.5,
                          eq_order=order)
    ux, uy = M.velocity(0)
    f = oracle_mod.init(p, np.ones((n, n)), ux, uy, M.phi(0), M.force(0, nu))
    nsteps = int(round(M.T))
    phi_next = M.phi(0)
    for t in range(nsteps):
        phi_t, phi_next = phi_next, M.phi(t + 1)
        f = oracle_mod.step(p, f, phi_t, phi_next, M.force(t, nu))
    mac = oracle_mod.macros(p, f, M.phi(nsteps), M.force(nsteps, nu))
    return mms.relative_l2(mac["ux"], mac["uy"], *M.velocity(nsteps))


def test_appb_manufactured_solution_second_order_convergence(oracle_mod):
    errs = [_mms_error(oracle_mod, n, 2) for n in (16, 32, 64)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 1.85) and np.all(slopes < 2.15), (errs, slopes)
    assert errs[-1] < 5e-3


def _darcy_brinkman(oracle_mod, ny, phi0=0.5, tau=0.8, G=1e-6, da=1e-2, steps=8000):
    nx = 3
    nu = (tau - 0.5) / 3
    k0 = da * ny * ny
    p = oracle_mod.Params(nx=nx, ny=ny, **oracle_mod.rates_from_tau(tau, s_eps=1.2, s_q=1.2), kappa=0.5, bc_y=1,
                          drag_d0=nu / k0)
    phi = np.full((ny, nx), phi0)
    fb = np.stack([phi * G, 0 * phi])
    f = oracle_mod.init(p, np.ones((ny, nx)), 0 * phi, 0 * phi, phi, fb)
    for _ in range(steps):
        f = oracle_mod.step(p, f, phi, None, fb)
    u = oracle_mod.macros(p, f, phi, fb)["ux"][:, 0]
    y = np.arange(ny) + 0.5          # walls half-way: at y = 0 and y = H = ny
    r = np.sqrt(phi0 / k0)
    ua = G * k0 / (phi0 * nu) * (1 - np.cosh(r * (y - ny / 2)) / np.cosh(r * ny / 2))
    return np.sqrt(np.sum((u - ua) ** 2) / np.sum(ua ** 2))


def test_drag_darcy_brinkman_channel_matches_eq22(oracle_mod):
    e16, e32 = _darcy_brinkman(oracle_mod, 16), _darcy_brinkman(oracle_mod, 32)
    assert e32 < 2e-3
    assert 3.3 < e16 / e32 < 4.7, (e16, e32)


def _particle_flow(oracle_mod, L, a=0.3, G=1e-6, tau=0.8, steps=20000):
    nx, ny = L, 3
    p = oracle_mod.Params(nx=nx, ny=ny, **oracle_mod.rates_from_tau(tau, s_eps=1.2, s_q=1.2), kappa=0.5, drag_d1=1.0)
    phi = np.tile(1 + a * (np.sin(2 * np.pi * np.arange(nx) / L) - 1), (ny, 1))
    fb = np.stack([phi * G, 0 * phi])
    f = oracle_mod.init(p, np.ones((ny, nx)), 0 * phi, 0 * phi, phi, fb)
    for _ in range(steps):
        f = oracle_mod.step(p, f, phi, None, fb)
    u = oracle_mod.macros(p, f, phi, fb)["ux"][0]
    ua = G / (a * phi[0])
    return np.sqrt(np.sum((u - ua) ** 2) / np.sum(ua ** 2))


def test_drag_nonuniform_particle_flow_matches_eq23(oracle_mod):
    e50, e100 = _particle_flow(oracle_mod, 50), _particle_flow(oracle_mod, 100)
    assert e100 < 5e-4
    assert 3.3 < e50 / e100 < 4.7, (e50, e100)


def test_drag_momentum_balance(oracle_mod):
    nx, ny = 12, 9
    rng = np.random.default_rng(31)
    p = oracle_mod.Params(nx=nx, ny=ny, **oracle_mod.rates_from_tau(0.7), kappa=0.5, drag_d0=0.02, drag_d1=0.5,
                          us_x=3e-3, us_y=-1e-3)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    phi = 0.6 + 0.2 * np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * y / ny)
    fb = rng.normal(size=(2, ny, nx)) * 1e-4
    f = oracle_mod.init(p, 1 + 0.01 * np.cos(2 * np.pi * y / ny), 0.02 * np.cos(2 * np.pi * y / ny),
                        0.01 * np.sin(2 * np.pi * x / nx), phi, fb)
    for _ in range(5):
        m = oracle_mod.macros(p, f, phi, fb)
        j0 = np.array([np.sum(E[:, 0][:, None, None] * f), np.sum(E[:, 1][:, None, None] * f)])
        f = oracle_mod.step(p, f, phi, None, fb)
        j1 = np.array([np.sum(E[:, 0][:, None, None] * f), np.sum(E[:, 1][:, None, None] * f)])
        dF = np.array([m["Fx"].sum(), m["Fy"].sum()])
        assert np.abs(j1 - j0 - dF).max() < 1e-14
    # the drag is inside F: u solves u sum f = j + F/2 with F evaluated at that u
    m = oracle_mod.macros(p, f, phi, fb)
    jx = np.einsum("i,iyx->yx", E[:, 0].astype(float), f)
    assert np.abs(m["ux"] * f.sum(0) - (jx + 0.5 * m["Fx"])).max() < 1e-15


def _db(oracle_mod, ny, phi0, da, kappa, tau=0.8, G=1e-6, steps=15000):
    nx = 3
    nu = (tau - 0.5) / 3
    k0 = da * ny * ny
    p = oracle_mod.Params(nx=nx, ny=ny, **oracle_mod.rates_from_tau(tau, s_eps=1.2, s_q=1.2), kappa=kappa, bc_y=1,
                          drag_d0=nu / k0)
    phi = np.full((ny, nx), phi0)
    fb = np.stack([phi * G, 0 * phi])
    f = oracle_mod.init(p, np.ones((ny, nx)), 0 * phi, 0 * phi, phi, fb)
    for _ in range(steps):
        f = oracle_mod.step(p, f, phi, None, fb)
    u = oracle_mod.macros(p, f, phi, fb)["ux"][:, 0]
    y = np.arange(ny) + 0.5
    r = np.sqrt(phi0 / k0)
    ua = G * k0 / (phi0 * nu) * (1 - np.cosh(r * (y - ny / 2)) / np.cosh(r * ny / 2))
    return np.sqrt(np.sum((u - ua) ** 2) / np.sum(ua ** 2))


@pytest.mark.parametrize("phi0,da,kappa,bound", [(0.3, 1e-3, 0.5, 1e-3), (0.1, 1e-4, 0.25, 4e-3)])
def test_x1_porous_poiseuille_across_darcy_numbers(oracle_mod, phi0, da, kappa, bound):
    """Eq. (22 I) at smaller Da and phi (the thin Brinkman layer, sqrt(k0 / phi) = 0.06 H
    and 0.03 H, needs ny >= 64 to be resolved): the error falls towards second order
    under refinement. phi = 0.1 runs kappa = 0.25 (reading c23: X = kappa / phi <= 2.5)."""
    e64, e128 = _db(oracle_mod, 64, phi0, da, kappa), _db(oracle_mod, 128, phi0, da, kappa)
    assert e128 < bound
    assert e64 / e128 > 2.9, (e64, e128)


def test_x3_transient_particle_flow(oracle_mod):
    """Eq. (23) with a moving void fraction (a = 0.45, u_s = 1e-3; phi down to 0.1, so
    kappa = 0.25): the velocity follows u_s + G / (a phi) with the same small
    deviation at every sampled time (periodic in the frame of the void fraction)."""
    L, ny, a, us, G, tau = 100, 3, 0.45, 1e-3, 1e-6, 0.8
    p = oracle_mod.Params(nx=L, ny=ny, **oracle_mod.rates_from_tau(tau, s_eps=1.2, s_q=1.2), kappa=0.25,
                          drag_d1=1.0, us_x=us)
    x = np.arange(L)

    def phi_of(t):
        return np.tile(1 + a * (np.sin(2 * np.pi * (x - us * t) / L) - 1), (ny, 1))

    def fb(ph):
        return np.stack([ph * G, 0 * ph])

    ph0 = phi_of(0)
    f = oracle_mod.init(p, np.ones((ny, L)), us + G / (a * ph0), 0 * ph0, ph0, fb(ph0))
    errs = []
    for t in range(6000):
        f = oracle_mod.step(p, f, phi_of(t), phi_of(t + 1), fb(phi_of(t)))
        if (t + 1) % 2000 == 0:
            ph = phi_of(t + 1)
            u = oracle_mod.macros(p, f, ph, fb(ph))["ux"][0]
            ua = us + G / (a * ph[0])
            errs.append(np.sqrt(np.sum((u - ua) ** 2) / np.sum((ua - us) ** 2)))
    assert max(errs) < 0.04, errs
    assert max(errs) - min(errs) < 1e-3 * max(errs)


@pytest.mark.parametrize("kappa,stable", [(0.25, True), (0.31, False)])
def test_provisional_eos_stability_limit(oracle_mod, kappa, stable):
    """Reading c23: the provisional equation of state gives an effective sound speed
    sqrt(X / 3), X = kappa / phi, which must stay below the lattice speed: a decaying
    shear wave at uniform phi = 0.1 stays bounded at X = 2.5 and blows up at X = 3.1."""
    nx, ny = 4, 32
    p = oracle_mod.Params(nx=nx, ny=ny, **oracle_mod.rates_from_tau(0.8, s_eps=1.2, s_q=1.2), kappa=kappa)
    phi = np.full((ny, nx), 0.1)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    f = oracle_mod.init(p, np.ones((ny, nx)), 1e-3 * np.sin(2 * np.pi * y / ny), 0 * phi, phi)
    with np.errstate(all="ignore"):
        for _ in range(3000):
            f = oracle_mod.step(p, f, phi)
    finite = bool(np.isfinite(f).all() and np.abs(f).max() < 10)
    assert finite == stable


def _couette(oracle_mod, ny, da, kappa, phi0=0.5, tau=0.8, uh=1e-3):
    """Eq. (22 II): half-way bounce-back at the bottom (y = 0), the moving wall by
    non-equilibrium extrapolation on row ny-1 (y = H = ny - 1/2), G = 0; relative L2
    error of u on the fluid rows against the analytic profile."""
    nx = 3
    nu = (tau - 0.5) / 3
    H = ny - 0.5
    drag = {}
    if da:
        k0 = da * H * H
        drag = dict(drag_d0=nu / k0)
    p = oracle_mod.Params(nx=nx, ny=ny, **oracle_mod.rates_from_tau(tau, s_eps=1.2, s_q=1.2), kappa=kappa, bc_y=1,
                          nee_top=1, uw_x=uh, **drag)
    phi = np.full((ny, nx), phi0)
    f = oracle_mod.init(p, np.ones((ny, nx)), 0 * phi, 0 * phi, phi)
    steps = int(30 * min(H * H / nu, k0 / (phi0 * nu)) + 2000) if da else int(6 * H * H / nu)
    for _ in range(steps):
        f = oracle_mod.step(p, f, phi)
    u = oracle_mod.macros(p, f, phi)["ux"][:-1, 0]
    y = np.arange(ny - 1) + 0.5
    if da:
        r = np.sqrt(phi0 / k0)
        ua = uh * np.sinh(r * y) / np.sinh(r * H)
    else:
        ua = uh * y / H
    return np.sqrt(np.sum((u - ua) ** 2) / np.sum(ua ** 2))


def test_x2_plain_couette_is_linear(oracle_mod):
    """Without the Darcy term the moving-wall channel converges to the linear Couette
    profile u_H y / H exactly (to the convergence of the run)."""
    assert _couette(oracle_mod, 16, None, 0.5) < 1e-9


@pytest.mark.parametrize("kappa", [0.5, 0.3])
def test_x2_porous_couette_matches_eq22(oracle_mod, kappa):
    """Eq. (22 II) with phi = 0.5, Da = 1e-2, u_H = 1e-3: second-order convergence of
    the profile to u_H sinh(r y) / sinh(r H), r = sqrt(phi / k0) (kappa = 0.3: phi !=
    kappa, so F^p and C are active next to the wall)."""
    e16, e32 = _couette(oracle_mod, 16, 1e-2, kappa), _couette(oracle_mod, 32, 1e-2, kappa)
    assert e32 < 8e-3
    assert 3.0 < e16 / e32 < 4.7, (e16, e32)
