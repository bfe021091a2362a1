"""Pins for the oracle's full step: reductions to textbook schemes, invariants,
analytic flows and second-order convergence on manufactured solutions."""
import math

import numpy as np
import pytest

from synth import fields, mms

E = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]


def _textbook_bgk_guo_step(f, s, F, wall_y):
    """Standard D2Q9 BGK with Guo forcing, written from the textbook (not from the
    paper): f+ = f - s (f - f^eq) + (1 - s/2) F_i, then streaming."""
    rho = f.sum(0)
    jx = np.einsum("i,iyx->yx", E[:, 0].astype(float), f)
    jy = np.einsum("i,iyx->yx", E[:, 1].astype(float), f)
    ux = (jx + 0.5 * F[0]) / rho
    uy = (jy + 0.5 * F[1]) / rho
    post = np.empty_like(f)
    for i in range(9):
        eu = E[i, 0] * ux + E[i, 1] * uy
        uu = ux * ux + uy * uy
        feq = W[i] * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * uu)
        Fi = W[i] * ((3 * (E[i, 0] - ux) + 9 * eu * E[i, 0]) * F[0]
                     + (3 * (E[i, 1] - uy) + 9 * eu * E[i, 1]) * F[1])
        post[i] = f[i] - s * (f[i] - feq) + (1 - 0.5 * s) * Fi
    out = np.empty_like(f)
    ny = f.shape[1]
    for i in range(9):
        out[i] = np.roll(post[i], shift=(E[i, 1], E[i, 0]), axis=(0, 1))
    if wall_y:
        for i in range(9):
            if E[i, 1] == 1:    # leaves through the top wall: returns opposite at y = ny-1
                out[OPP[i], ny - 1] = post[i, ny - 1]
            if E[i, 1] == -1:   # leaves through the bottom wall
                out[OPP[i], 0] = post[i, 0]
    return out


@pytest.mark.parametrize("wall_y", [0, 1])
def test_reduces_to_textbook_bgk_when_phi_equals_kappa(oracle_mod, wall_y):
    """phi = kappa gives X = 1, F^p = 0, C = 0 and the textbook equilibrium of density
    kappa rho; with every rate equal the MRT step is then BGK with Guo forcing."""
    ny, nx = 9, 11
    kappa = 0.5
    s = 1 / 0.7
    p = oracle_mod.Params(nx=nx, ny=ny, s_nu=s, s_e=s, s_eps=s, s_q=s, s_c=s, kappa=kappa,
                          bc_y=wall_y)
    rng = np.random.default_rng(10)
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


def test_rest_state_is_a_fixed_point(oracle_mod):
    """Uniform phi != kappa, rho uniform, u = 0, F = 0: the populations do not move."""
    n = 8
    p = oracle_mod.Params(nx=n, ny=n, **oracle_mod.rates_from_tau(0.8), kappa=0.5, bc_y=1)
    phi = np.full((n, n), 0.8)
    f0 = oracle_mod.init(p, np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)), phi)
    f = f0
    for _ in range(10):
        f = oracle_mod.step(p, f, phi)
    assert np.abs(f - f0).max() < 1e-15


def test_no_flow_discontinuous_block_stays_at_rest(oracle_mod):
    """Sec. 3.3, Eq. (24): with F^B = 0 and a discontinuous phi block the exact
    solution is u = 0. The populations of Eq. (14) for i != 0 do not depend on phi,
    so the rest state streams onto itself and no spurious velocity appears."""
    n = 20
    p = oracle_mod.Params(nx=n, ny=n, **oracle_mod.rates_from_tau(0.8), kappa=0.5)
    phi = np.ones((n, n))
    phi[8:12, 8:12] = 0.3
    f = oracle_mod.init(p, np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)), phi)
    for _ in range(50):
        f = oracle_mod.step(p, f, phi)
    m = oracle_mod.macros(p, f, phi)
    assert np.abs(m["ux"]).max() < 1e-15 and np.abs(m["uy"]).max() < 1e-15
    assert np.abs(m["rho"] - 1).max() < 1e-14


@pytest.mark.parametrize("bc_y", [0, 1])
def test_mass_is_conserved_with_moving_void_fraction(oracle_mod, bc_y):
    n = 16
    p = oracle_mod.Params(nx=n, ny=n, **oracle_mod.rates_from_tau(0.7), kappa=0.4, bc_y=bc_y)
    rng = np.random.default_rng(11)
    M = mms.Config1(n=n, T=200.0)
    ux, uy = M.velocity(0)
    f = oracle_mod.init(p, 1 + 0.01 * rng.normal(size=(n, n)), ux, uy, M.phi(0))
    m0 = f.sum()
    for t in range(20):
        fb = rng.normal(size=(2, n, n)) * 1e-5
        f = oracle_mod.step(p, f, M.phi(t), M.phi(t + 1), fb)
        assert abs(f.sum() - m0) < 1e-13 * m0


def test_long_run_has_no_steady_mass_or_momentum_drift(oracle_mod):
    """3000 steps: the mass of a walled, forced lattice with a steady void fraction and
    the momentum of an unforced periodic lattice at phi = kappa (F^p = 0) stay within
    round-off of their start. A back-transform that multiplies by rounded fractions
    of M^-1 (4/36, 6/36, ...) scales both by a fixed factor 1 - 5.6e-17 every step,
    1.7e-13 over these steps."""
    nx, ny, steps = 10, 8, 3000
    rng = np.random.default_rng(13)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    p = oracle_mod.Params(nx=nx, ny=ny, **oracle_mod.rates_from_tau(0.7), kappa=0.5, bc_y=1)
    phi = rng.uniform(0.4, 1.0, (ny, nx))
    fb = np.stack([phi * 1e-5, phi * 0.0])
    f = oracle_mod.init(p, 1 + 0.01 * rng.normal(size=(ny, nx)), 0 * phi, 0 * phi, phi, fb)
    m0 = f.sum()
    for _ in range(steps):
        f = oracle_mod.step(p, f, phi, None, fb)
    assert abs(f.sum() - m0) < 2e-14 * m0

    p = oracle_mod.Params(nx=nx, ny=ny, **oracle_mod.rates_from_tau(0.7), kappa=0.5)
    phi = np.full((ny, nx), 0.5)
    f = oracle_mod.init(p, 1 + 0.01 * np.cos(2 * np.pi * y / ny), 0.02 + 0.01 * np.sin(2 * np.pi * y / ny),
                        -0.01 + 0.01 * np.cos(2 * np.pi * x / nx), phi)
    j0 = np.array([np.einsum("i,iyx->", E[:, a].astype(float), f) for a in range(2)])
    for _ in range(steps):
        f = oracle_mod.step(p, f, phi)
    j1 = np.array([np.einsum("i,iyx->", E[:, a].astype(float), f) for a in range(2)])
    assert np.all(np.abs(j1 - j0) < 3e-14 * np.abs(j0)), (j0, j1)


def test_momentum_balance_periodic(oracle_mod):
    """Periodic domain: sum_x j(t+1) = sum_x j(t) + sum_x F(t), F = F^p + F^B, because
    the collision maps j to j + F (Eq. 16 with S_3 = F_x, s_c arbitrary)."""
    n = 12
    p = oracle_mod.Params(nx=n, ny=n, **oracle_mod.rates_from_tau(0.9), kappa=0.5, s_c=0.7)
    rng = np.random.default_rng(12)
    M = mms.Config1(n=n, T=300.0)
    ux, uy = M.velocity(0)
    f = oracle_mod.init(p, 1 + 0.01 * rng.normal(size=(n, n)), ux, uy, M.phi(0))
    for t in range(10):
        fb = rng.normal(size=(2, n, n)) * 1e-4
        mac = oracle_mod.macros(p, f, M.phi(t), fb)
        j0 = np.array([np.einsum("i,iyx->", E[:, a].astype(float), f) for a in range(2)])
        f = oracle_mod.step(p, f, M.phi(t), M.phi(t + 1), fb)
        j1 = np.array([np.einsum("i,iyx->", E[:, a].astype(float), f) for a in range(2)])
        Fsum = np.array([mac["Fx"].sum(), mac["Fy"].sum()])
        assert np.abs(j1 - j0 - Fsum).max() < 1e-12  # |F sum| ~ 1e-3; round-off ~ 1e-15


def test_poiseuille_exact_at_magic_rates(oracle_mod):
    """Force-driven channel with half-way bounce-back walls at y = -1/2 and ny - 1/2,
    phi = kappa = 1 (plain MRT): with (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16 the steady
    profile is the parabola G (y + 1/2)(ny - 1/2 - y) / (2 nu) to round-off."""
    ny, nx = 16, 4
    tau = 0.8
    s_nu, nu = 1 / tau, (tau - 0.5) / 3
    s_q = 1 / (0.5 + (3 / 16) / (tau - 0.5))
    p = oracle_mod.Params(nx=nx, ny=ny, s_nu=s_nu, s_e=1.1, s_eps=1.2, s_q=s_q, kappa=1.0, bc_y=1)
    phi = np.ones((ny, nx))
    G = 1e-5
    fb = np.zeros((2, ny, nx))
    fb[0] = G
    f = oracle_mod.init(p, np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), phi, fb)
    for _ in range(12000):
        f = oracle_mod.step(p, f, phi, None, fb)
    m = oracle_mod.macros(p, f, phi, fb)
    y = np.arange(ny)
    ua = G / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(m["ux"][:, 0] - ua).max() / ua.max() < 1e-7
    assert np.abs(m["uy"]).max() < 1e-14


def test_poiseuille_with_uniform_void_fraction(oracle_mod):
    """Uniform phi != kappa, F^B = phi G (Sec. 3.1 without drag): VANSE gives the same
    parabola; here the penalty term C_c and the wall ghost rule are active, so the
    match is second order rather than exact."""
    errs = []
    for ny in (8, 16):
        nx = 2
        tau = 0.8
        nu = (tau - 0.5) / 3
        p = oracle_mod.Params(nx=nx, ny=ny, **oracle_mod.rates_from_tau(tau), kappa=0.5, bc_y=1)
        phi = np.full((ny, nx), 0.8)
        G = 1e-5
        fb = np.zeros((2, ny, nx))
        fb[0] = phi * G
        f = oracle_mod.init(p, np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), phi, fb)
        for _ in range(int(60 * ny * ny)):
            f = oracle_mod.step(p, f, phi, None, fb)
        m = oracle_mod.macros(p, f, phi, fb)
        y = np.arange(ny)
        ua = G / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
        errs.append(np.abs(m["ux"][:, 0] - ua).max() / ua.max())
    assert errs[1] < 0.02
    assert errs[0] / errs[1] > 3.0, errs


def test_hydrostatic_balance_pins_pressure_correction(oracle_mod):
    """Periodic box with phi(x, y) varying and F^B = phi G, G = g (sin kx, sin ky):
    VANSE's steady state has u = 0 and grad p = G, i.e.
    rho = rho0 - 3 g (cos kx + cos ky) / k. The lattice pressure is kappa rho cs^2,
    so this balance only holds when F^p = (kappa - phi) cs^2 grad rho (Eq. 13) is
    applied with the right sign and size in both directions."""
    n = 24
    p = oracle_mod.Params(nx=n, ny=n, **oracle_mod.rates_from_tau(0.8), kappa=0.5)
    y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    k = 2 * np.pi / n
    phi = 0.7 + 0.2 * np.sin(k * x + 0.5) * np.sin(k * y + 0.3)
    g = 1e-5
    fb = np.stack([phi * g * np.sin(k * x), phi * g * np.sin(k * y)])
    f = oracle_mod.init(p, np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)), phi, fb)
    for _ in range(6000):
        f = oracle_mod.step(p, f, phi, None, fb)
    m = oracle_mod.macros(p, f, phi, fb)
    rho_a = -3 * g / k * (np.cos(k * x) + np.cos(k * y))
    r = m["rho"] - m["rho"].mean()
    # with the opposite sign of F^p the lattice would settle at
    # grad rho = 3 phi G / (phi - 2 kappa), more than twice off
    assert np.abs(r - rho_a).max() / np.abs(rho_a).max() < 0.03
    # the remaining flow is a small discretisation error against the viscous
    # velocity scale g / (k^2 nu)
    nu = 0.1
    assert max(np.abs(m["ux"]).max(), np.abs(m["uy"]).max()) < 0.05 * g / (k * k * nu)


@pytest.mark.parametrize("phi0", [0.5, 0.8])
def test_sound_wave_damping_pins_bulk_viscosity(oracle_mod, phi0):
    """App. A, Eq. (A11)-(A12): the recovered stress is rho nu (grad u + grad u^T)
    + rho (nu_e - nu)(div u) I, and VANSE's (Eq. 2) needs nu_e = nu/3. A standing
    sound wave then decays at rate (nu + nu_e) k^2 / 2 = (2/3) nu k^2 (uniform phi,
    kappa = 0.5)."""
    n = 64
    tau = 0.8
    nu = (tau - 0.5) / 3
    p = oracle_mod.Params(nx=n, ny=1, **oracle_mod.rates_from_tau(tau), kappa=0.5)
    x = np.arange(n, dtype=float)[None, :]
    k = 2 * np.pi / n
    eps = 1e-4
    phi = np.full((1, n), phi0)
    f = oracle_mod.init(p, 1 + eps * np.cos(k * x), np.zeros((1, n)), np.zeros((1, n)), phi)
    amps = []
    steps = [0, 400, 800, 1200]
    for t in range(steps[-1] + 1):
        if t in steps:
            m = oracle_mod.macros(p, f, phi)
            a_rho = 2 / n * np.sum((m["rho"] - 1) * np.cos(k * x))
            a_u = 2 / n * np.sum(m["ux"] * np.sin(k * x))
            amps.append(np.sqrt(a_rho ** 2 + 3 * a_u ** 2))
        f = oracle_mod.step(p, f, phi)
    rate = -np.polyfit(steps, np.log(amps), 1)[0]
    expect = (2.0 / 3.0) * nu * k * k
    assert abs(rate / expect - 1) < 0.05, (rate, expect)


def _mms_error(oracle_mod, n):
    M = mms.Config1.refined(n)
    tau = 0.8
    nu = (tau - 0.5) / 3
    p = oracle_mod.Params(nx=n, ny=n, **oracle_mod.rates_from_tau(tau, s_eps=1.2, s_q=1.2), kappa=0.5)
    ux, uy = M.velocity(0)
    f = oracle_mod.init(p, np.ones((n, n)), ux, uy, M.phi(0), M.force(0, nu))
    nsteps = int(round(M.T))
    phi_next = M.phi(0)
    for t in range(nsteps):
        phi_t, phi_next = phi_next, M.phi(t + 1)
        f = oracle_mod.step(p, f, phi_t, phi_next, M.force(t, nu))
    mac = oracle_mod.macros(p, f, M.phi(nsteps), M.force(nsteps, nu))
    uxr, uyr = M.velocity(nsteps)
    return mms.relative_l2(mac["ux"], mac["uy"], uxr, uyr)


def test_manufactured_solution_second_order_convergence(oracle_mod):
    """Sec. 3.4: E_u (Eq. 26) on the spatiotemporal manufactured solution falls with
    slope ~2 under refinement (diffusive scaling: T ~ n^2, U0 ~ 1/n)."""
    errs = [_mms_error(oracle_mod, n) for n in (16, 32, 64)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 1.85) and np.all(slopes < 2.15), (errs, slopes)
    assert errs[-1] < 5e-3


def test_printed_mms_forces_match_eq25():
    """App. C prints the body forces of cases I-III; the Eq. (25) residual evaluated
    with Taylor jets (synth.mms) must reproduce them."""
    n, nu = 48, 0.1
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    X, Y = (2 * xx - n + 1) / n, (2 * yy - n + 1) / n
    pi = math.pi
    # case I (C1)
    a, b, us = 0.5, 0.49, 0.8
    sx, sy, cx, cy = np.sin(pi * X), np.sin(pi * Y), np.cos(pi * X), np.cos(pi * Y)
    phi = a + b * sx * sy
    Fx = (2 * pi * us ** 2 * phi / n ** 3 * sx ** 3 * cx * sy ** 2
          + 4 * nu * pi ** 2 * us * b / n ** 3 * sx ** 3 * cy ** 3
          + 4 * nu * pi ** 2 * us / n ** 3 * sy * cy
          * (-6 * phi * sx ** 2 + 2 * a * cx ** 2 + 5 * b * sx * cx ** 2 * sy))
    Fy = (2 * pi * us ** 2 * phi / n ** 3 * sx ** 2 * sy ** 3 * cy
          - 4 * nu * pi ** 2 * us / n ** 3 * sx * cx * cy ** 2 * (2 * a + 5 * b * sx * sy)
          + 4 * nu * pi ** 2 * us / n ** 3 * cx * sy ** 2
          * (6 * a * sx + 6 * b * sx ** 2 * sy - b * cx ** 2 * sy))
    F = mms.CaseI(n, a, b, us).force(0, nu)
    scale = np.abs(F).max()
    assert np.abs(F[0] - Fx).max() < 1e-12 * scale and np.abs(F[1] - Fy).max() < 1e-12 * scale
    # case II (C2)
    a, b = 0.5, 0.5
    F = mms.CaseII(n, a, b, us).force(0, nu)
    C2 = (2 * pi * us ** 2 * a * b / n ** 3 * np.exp(b * sx * sy) * np.sin(pi * (X + Y))
          - 4 * nu * pi ** 2 * us * a * b / (3 * n ** 3) * (cx * cy - 7 * sx * sy))
    scale = np.abs(F).max()
    assert np.abs(F[0] - C2).max() < 1e-12 * scale and np.abs(F[1] - C2).max() < 1e-12 * scale
    # case III (C3)
    a, b, us, t = 0.5, 0.45, 0.08, 333.0
    F = mms.CaseIII(n, a, b, us).force(t, nu)
    Xt, Yt = X + 4 * us * t / n ** 2, Y + 4 * us * t / n ** 2
    phi = a + b * np.sin(pi * Xt) * np.sin(pi * Yt)
    s = np.sin(pi * (Xt + Yt))
    base = -8 * pi * us ** 2 * b / n ** 3 * s + 2 * pi * us ** 2 * b / (n ** 3 * phi ** 2) * s * (4 * phi ** 2 - 1)
    c = 2 * nu * pi ** 2 * us * b / (3 * n ** 3 * phi ** 2)
    common = -7 * b + 8 * a * np.cos(pi * (Xt + Yt)) - 6 * a * np.cos(pi * (Xt - Yt))
    F3x = base + c * (3 * b * np.cos(2 * pi * Xt) + 4 * b * np.cos(2 * pi * Yt) + common)
    F3y = base + c * (4 * b * np.cos(2 * pi * Xt) + 3 * b * np.cos(2 * pi * Yt) + common)
    scale = np.abs(F).max()
    assert np.abs(F[0] - F3x).max() < 1e-12 * scale and np.abs(F[1] - F3y).max() < 1e-12 * scale


def test_manufactured_settings_satisfy_continuity():
    from synth import jet  # noqa: F401
    for M in (mms.Config1(32, T=500.0), mms.CaseI(32), mms.CaseII(32), mms.CaseIII(32)):
        for t in (0.0, 77.0):
            r = mms.continuity_residual(*M.jets(t))
            assert np.abs(r).max() < 1e-15


def test_channel_field_recipe():
    phi = fields.channel_phi(256, 128)
    assert phi.shape == (128, 256)
    assert abs(phi.min() - 0.35) < 1e-12 or phi.min() >= 0.35
    assert phi.max() <= 1.0 + 1e-12
    # block interior is 0.4, its collar is 1.0
    assert np.all(phi[60:66, 120:130] == 0.4)
    assert np.all(phi[51 - 16 + 8:51 - 8, 103:153] == 1.0)
    # the same seed gives the same field
    assert np.array_equal(phi, fields.channel_phi(256, 128))
