"""Pins of the oracle's solid cells (phi = 0: the impermeable block of Sec. 3.3, Eq. 24
with phi_0 = 0): half-way bounce-back on every link into a solid cell and the
mirrored Eq. (10) ghost values next to it.

* A lattice framed by solid rows (periodic across them) steps exactly like the same
  lattice with the built-in half-way walls, and solid columns like the oracle's
  x walls: this pins the bounce-back links and the ghost rule on straight surfaces,
  diagonal links included.
* A solid block in fluid at rest stays at rest; mass is conserved in a forced flow
  past a block.
* The Eq. (24) flow past a block with phi_0 = 0.5 and a Darcy resistance approaches
  the flow past the solid block as the Darcy number falls (the comparison the paper
  draws in Sec. 3.3), while it does not when the block is a plain porous block.
"""
import numpy as np
import pytest


def _rates(O, tau=0.8):
    return O.rates_from_tau(tau, s_eps=1.2, s_q=1.4)


def _random_fields(rng, ny, nx):
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    phi = 0.55 + 0.3 * rng.uniform(size=(ny, nx))
    rho = 1 + 0.01 * np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * y / ny)
    ux = 0.02 * np.cos(2 * np.pi * y / ny) + 0.005 * rng.normal(size=(ny, nx))
    uy = 0.01 * np.sin(2 * np.pi * x / nx) + 0.005 * rng.normal(size=(ny, nx))
    fb = 1e-5 * rng.normal(size=(2, ny, nx))
    return phi, rho, ux, uy, fb


def _frame(a, pad_y, pad_x, value):
    return np.pad(a, ((pad_y, pad_y), (pad_x, pad_x)), constant_values=value)


@pytest.mark.parametrize("axis", ["y", "x", "both"])
@pytest.mark.parametrize("unsteady", [False, True])
def test_solid_frame_equals_builtin_walls(oracle_mod, axis, unsteady):
    O = oracle_mod
    ny, nx, steps = 9, 11, 8
    rng = np.random.default_rng(40 + unsteady)
    phi, rho, ux, uy, fb = _random_fields(rng, ny, nx)
    phin = np.clip(phi + 0.02 * rng.normal(size=phi.shape), 0.4, 1.0) if unsteady else None
    py, px = (1 if axis in ("y", "both") else 0), (1 if axis in ("x", "both") else 0)
    walls = O.Params(nx=nx, ny=ny, **_rates(O), kappa=0.5, bc_y=py, bc_x=px)
    solid = O.Params(nx=nx + 2 * px, ny=ny + 2 * py, **_rates(O), kappa=0.5)
    fr = lambda a, v=0.0: _frame(a, py, px, v)
    fbs = np.stack([fr(fb[0]), fr(fb[1])])
    fa = O.init(walls, rho, ux, uy, phi, fb)
    fs = O.init(solid, fr(rho, 1.0), fr(ux), fr(uy), fr(phi), fbs)
    inner = (slice(None), slice(py, py + ny), slice(px, px + nx))
    assert np.abs(fs[inner] - fa).max() <= 1e-15
    ph, pn = phi, phin
    for k in range(steps):
        fa = O.step(walls, fa, ph, pn, fb)
        fs = O.step(solid, fs, fr(ph), fr(pn) if pn is not None else None, fbs)
        if pn is not None:
            ph, pn = pn, None
    assert np.abs(fs[inner] - fa).max() <= 1e-14 * np.abs(fa).max()
    ring = np.ones((ny + 2 * py, nx + 2 * px), bool)
    ring[py:py + ny, px:px + nx] = False
    assert np.all(fs[:, ring] == 0.0)


def _block(n, lo=0.4, hi=0.6):
    m = np.zeros((n, n), bool)
    a, b = int(round(lo * n)), int(round(hi * n))
    m[a:b, a:b] = True
    return m


def test_solid_block_at_rest_stays_at_rest(oracle_mod):
    O = oracle_mod
    n = 20
    p = O.Params(nx=n, ny=n, **_rates(O), kappa=0.5)
    phi = np.where(_block(n), 0.0, 1.0)
    f = O.init(p, np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)), phi)
    f0 = f.copy()
    for _ in range(50):
        f = O.step(p, f, phi)
    assert np.abs(f - f0).max() < 1e-15
    m = O.macros(p, f, phi)
    assert np.all(m["ux"] == 0.0) and np.all(m["uy"] == 0.0)


def test_mass_conserved_around_a_solid_block(oracle_mod):
    O = oracle_mod
    n = 24
    rng = np.random.default_rng(3)
    p = O.Params(nx=n, ny=n, **_rates(O), kappa=0.5)
    phi = np.where(_block(n), 0.0, 0.6 + 0.3 * rng.uniform(size=(n, n)))
    phi[3, 5] = 0.0                      # an isolated solid cell and a diagonal pair
    phi[10, 2] = phi[11, 3] = 0.0
    fb = np.stack([phi * 1e-5, phi * 0.0])
    f = O.init(p, np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)), phi, fb)
    m0 = f.sum()
    for _ in range(200):
        f = O.step(p, f, phi, None, fb)
    assert abs(f.sum() - m0) < 1e-13 * m0
    assert np.all(f[:, phi == 0.0] == 0.0)


def _eq24_flow(O, n, phi0, da, steps, tau=0.8, G=1e-6):
    """Eq. (24): the block [0.4L, 0.6L] x [0.4H, 0.6H] of void fraction phi0 (0 =
    solid) in a periodic L x L domain of phi = 1, driven by F^B = phi G along x, with
    the Darcy resistance phi^2 nu / k0 (k0 = Da L^2) in the block only: the drag's
    beta = phi^2 d1 (1 - phi) vanishes at phi = 1, and d1 = nu / (k0 (1 - phi0))."""
    nu = (tau - 0.5) / 3
    block = _block(n)
    phi = np.where(block, phi0, 1.0)
    d1 = nu / (da * n * n * (1.0 - phi0)) if da else 0.0
    p = O.Params(nx=n, ny=n, **O.rates_from_tau(tau, s_eps=1.2, s_q=1.2), kappa=0.5, drag_d1=d1)
    fb = np.stack([phi * G, 0 * phi])
    f = O.init(p, np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)), phi, fb)
    for _ in range(steps):
        f = O.step(p, f, phi, None, fb)
    m = O.macros(p, f, phi, fb)
    return m["ux"], m["uy"], block


def test_eq24_darcy_block_approaches_the_solid_block(oracle_mod):
    """Sec. 3.3: with phi_0 = 0.5 and a high Darcy resistance in the block the flow
    around it should resemble the flow around the impermeable block (phi_0 = 0). The
    relative L2 difference of u outside the block (32 x 32, 3000 steps) falls as Da
    falls to the paper's 1e-6, and stays large for the porous block without
    resistance."""
    n, steps = 32, 3000
    us, vs, block = _eq24_flow(oracle_mod, n, 0.0, None, steps)
    out = ~block

    def diff(ux, uy):
        return np.sqrt(np.sum((ux - us)[out] ** 2 + (uy - vs)[out] ** 2) / np.sum(us[out] ** 2 + vs[out] ** 2))

    d = [diff(*_eq24_flow(oracle_mod, n, 0.5, da, steps)[:2]) for da in (1e-3, 1e-4, 1e-5, 1e-6)]
    free = diff(*_eq24_flow(oracle_mod, n, 0.5, None, steps)[:2])
    # measured: 0.60, 0.18, 0.074, 0.056 against 1.5 without the resistance
    assert d[0] > d[1] > d[2] > d[3], d
    assert d[3] < 0.07 and free > 20 * d[3], (d, free)
