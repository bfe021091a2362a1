"""Pins for the oracle's point functions: each is checked against something the
paper or the mathematics fixes independently of the oracle's own formula."""
import itertools

import numpy as np
import pytest

CS2 = 1.0 / 3.0


def _rand_state(rng):
    kappa = rng.uniform(0.2, 0.9)
    phi = rng.uniform(kappa, 1.0)
    rho = rng.uniform(0.7, 1.3)
    ux, uy = rng.uniform(-0.15, 0.15, size=2)
    return kappa, phi, rho, ux, uy


def test_lattice_matches_eq5(oracle_mod):
    e, w = oracle_mod.lattice()
    expect = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    assert [tuple(v) for v in e] == expect
    assert np.allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, atol=0, rtol=1e-15)
    # isotropy of the weights: sum w = 1, sum w e e = cs^2 I, sum w e_a e_b e_c e_d = cs^4 (dd+dd+dd)
    assert abs(w.sum() - 1) < 1e-15
    T2 = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.allclose(T2, CS2 * np.eye(2), atol=1e-15)
    T4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    d = np.eye(2)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(T4, iso, atol=1e-15)


def test_moment_matrix_rows_are_the_eq17_moments(oracle_mod):
    """Rows of M (A1) against the moment polynomials of the Lallemand-Luo basis that
    Eq. (17) names: (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy)."""
    e, _ = oracle_mod.lattice()
    ex, ey = e[:, 0].astype(float), e[:, 1].astype(float)
    e2 = ex ** 2 + ey ** 2
    rows = np.array([
        np.ones(9),
        -4 + 3 * e2,
        4 - 10.5 * e2 + 4.5 * e2 ** 2,
        ex,
        (-5 + 3 * e2) * ex,
        ey,
        (-5 + 3 * e2) * ey,
        ex ** 2 - ey ** 2,
        ex * ey,
    ])
    assert np.array_equal(oracle_mod.M(), rows)


def test_printed_inverse_is_the_inverse(oracle_mod):
    M, Mi = oracle_mod.M(), oracle_mod.Minv()
    assert np.abs(M @ Mi - np.eye(9)).max() < 1e-15
    assert np.abs(Mi @ M - np.eye(9)).max() < 1e-15
    assert np.abs(Mi - np.linalg.inv(M)).max() < 1e-15


def test_equilibrium_moments_eq14_vs_eq18(oracle_mod):
    """M f^eq (Eq. 14 in velocity space) equals m^eq (Eq. 18, printed separately)."""
    rng = np.random.default_rng(1)
    M = oracle_mod.M()
    for _ in range(50):
        s = _rand_state(rng)
        feq = oracle_mod.feq(*s)
        meq = oracle_mod.meq(*s)
        assert np.abs(M @ feq - meq).max() < 2e-15
        assert np.allclose(oracle_mod.moments(feq), M @ feq, atol=1e-15, rtol=0)


def test_force_moments_eq6_vs_eq19(oracle_mod):
    rng = np.random.default_rng(2)
    M = oracle_mod.M()
    for _ in range(50):
        ux, uy = rng.uniform(-0.15, 0.15, size=2)
        Fx, Fy = rng.normal(size=2) * 1e-3
        assert np.abs(M @ oracle_mod.guo_force(ux, uy, Fx, Fy)
                      - oracle_mod.force_moments(ux, uy, Fx, Fy)).max() < 1e-17


def test_equilibrium_velocity_moments_eq15(oracle_mod):
    """Eq. (15): moments 0-3 of the adjusted equilibrium; the isotropic pressure part
    is kappa rho cs^2 and the 'diagonal' third moment keeps phi rho cs^2."""
    e, _ = oracle_mod.lattice()
    rng = np.random.default_rng(3)
    d = np.eye(2)
    for _ in range(30):
        kappa, phi, rho, ux, uy = _rand_state(rng)
        u = np.array([ux, uy])
        f = oracle_mod.feq(kappa, phi, rho, ux, uy)
        assert abs(f.sum() - phi * rho) < 1e-15
        assert np.allclose(np.einsum("i,ia->a", f, e), phi * rho * u, atol=1e-16, rtol=0)
        P = np.einsum("i,ia,ib->ab", f, e, e)
        assert np.allclose(P, phi * rho * np.outer(u, u) + kappa * rho * CS2 * d, atol=1e-15, rtol=0)
        T = np.einsum("i,ia,ib,ic->abc", f, e, e, e)
        for a, b, c in itertools.product(range(2), repeat=3):
            sym = u[c] * d[a, b] + u[b] * d[a, c] + u[a] * d[b, c]
            coef = phi if (a == b == c) else kappa
            assert abs(T[a, b, c] - coef * rho * CS2 * sym) < 1e-15


def test_penalty_eq20_is_the_chapman_enskog_difference(oracle_mod):
    """Eq. (20) against App. A: C must be what turns the first-order non-equilibrium
    moments of (A9) into the target ones of (A10). Evaluated from the printed (A9)
    and (A10) at random primitive values and derivatives (product rule by hand,
    d_t rho replaced as App. A does)."""
    rng = np.random.default_rng(4)
    for model_b in (0, 1):
        for _ in range(50):
            kappa, phi, rho, ux, uy = _rand_state(rng)
            rx, ry, px, py, pt = rng.normal(size=5) * 0.1
            uxx, uxy, uyx, uyy = rng.normal(size=4) * 0.01   # d_x u_x, d_y u_x, d_x u_y, d_y u_y
            # (A10)'s targets carry phi rho in the viscous part; for model B
            # (Sec. 2.3, kappa - phi -> kappa - 1) the target stress carries rho
            target_coef = 1.0 if model_b else phi
            # product-rule derivatives of A = rho u and D = phi rho u
            dxA_x = rx * ux + rho * uxx
            dyA_y = ry * uy + rho * uyy
            dxA_y = rx * uy + rho * uyx
            dyA_x = ry * ux + rho * uxy
            dxD_x = px * rho * ux + phi * rx * ux + phi * rho * uxx
            dyD_y = py * rho * uy + phi * ry * uy + phi * rho * uyy
            dxD_y = px * rho * uy + phi * rx * uy + phi * rho * uyx
            dyD_x = py * rho * ux + phi * ry * ux + phi * rho * uxy
            rho_t = -(dxD_x + dyD_y + rho * pt) / phi
            # (A9) minus (A10), the C-free parts; the u.F terms are identical and cancel
            Ca = (-2 * kappa * (ux * rx + uy * ry) + kappa * (dxA_x + dyA_y)
                  + 3 * (dxD_x + dyD_y) + 2 * kappa * rho_t
                  - 2 * target_coef * rho * (uxx + uyy))
            Cb = (-(2 * kappa / 3) * (ux * rx - uy * ry) - (kappa / 3) * (dxA_x - dyA_y)
                  + (dxD_x - dyD_y) - (2 / 3) * target_coef * rho * (uxx - uyy))
            Cc = (kappa / 3) * rho * (uyx + uxy) - (1 / 3) * target_coef * rho * (uyx + uxy)
            C = oracle_mod.penalty(kappa, phi, rho,
                                   [dxA_x, dyA_y, dxA_y, dyA_x], [uxx, uyy, uyx, uxy],
                                   [dxD_x, dyD_y, dxD_y, dyD_x], pt, model_b)
            scale = 1e-15 * max(1.0, abs(Ca), abs(Cb))
            assert abs(C[1] - Ca) < 20 * scale
            assert abs(C[7] - Cb) < 20 * scale
            assert abs(C[8] - Cc) < 20 * scale
            assert np.all(C[[0, 2, 3, 4, 5, 6]] == 0)


@pytest.mark.parametrize("bc", [(0, 0), (0, 1)])
def test_gradient_eq10_exact_on_quadratics(oracle_mod, bc):
    """Eq. (10) is a second-order isotropic stencil: exact on every polynomial of
    degree <= 2 at cells whose stencil stays inside the domain."""
    nx, ny = 12, 10
    p = oracle_mod.Params(nx=nx, ny=ny, s_nu=1.0, s_e=1.0, bc_x=bc[0], bc_y=bc[1])
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    rng = np.random.default_rng(5)
    c = rng.normal(size=6)
    psi = c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y
    gx, gy = oracle_mod.gradient(p, psi)
    ex = c[1] + 2 * c[3] * x + c[4] * y
    ey = c[2] + c[4] * x + 2 * c[5] * y
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    assert np.abs(gx[inner] - ex[inner]).max() < 1e-12
    assert np.abs(gy[inner] - ey[inner]).max() < 1e-12


def test_gradient_eq10_second_order_on_periodic_waves(oracle_mod):
    errs = []
    for n in (16, 32, 64):
        p = oracle_mod.Params(nx=n, ny=n, s_nu=1.0, s_e=1.0)
        y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
        k = 2 * np.pi / n
        psi = np.sin(k * x + 0.3) * np.cos(2 * k * y)
        gx, gy = oracle_mod.gradient(p, psi)
        ex = k * np.cos(k * x + 0.3) * np.cos(2 * k * y)
        ey = -2 * k * np.sin(k * x + 0.3) * np.sin(2 * k * y)
        errs.append(max(np.abs(gx - ex).max(), np.abs(gy - ey).max()) / k)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9) and np.all(rates < 2.1), rates


def test_gradient_wall_ghost_rule(oracle_mod):
    """Reading c6: next to a half-way wall the ghost cell mirrors the first fluid
    cell; scalars keep the value, vector components change sign."""
    nx, ny = 6, 5
    p = oracle_mod.Params(nx=nx, ny=ny, s_nu=1.0, s_e=1.0, bc_y=1)
    rng = np.random.default_rng(6)
    psi = rng.normal(size=(ny, nx))
    for odd in (False, True):
        gx, gy = oracle_mod.gradient(p, psi, odd=odd)
        s = -1.0 if odd else 1.0
        ghost_lo = s * psi[0]
        ghost_hi = s * psi[-1]
        ext = np.vstack([ghost_lo, psi, ghost_hi])
        # brute force Eq. (10) on the extended array (periodic in x)
        e, w = oracle_mod.lattice()
        bx = np.zeros((ny, nx))
        by = np.zeros((ny, nx))
        for i in range(9):
            sh = np.roll(ext, shift=(-e[i, 1], -e[i, 0]), axis=(0, 1))[1:-1]
            bx += 3 * w[i] * e[i, 0] * sh
            by += 3 * w[i] * e[i, 1] * sh
        assert np.abs(gx - bx).max() < 1e-14
        assert np.abs(gy - by).max() < 1e-14


def test_rates_from_tau_bulk_viscosity(oracle_mod):
    """tau = 0.8 gives the paper's default nu = 0.1 and, with nu_e = nu/3 (Eq. A12),
    tau_e = (nu_e/cs^2 + 1/2)^-1 = 1/0.6."""
    r = oracle_mod.rates_from_tau(0.8)
    assert abs(r["s_nu"] - 1.25) < 1e-15
    assert abs(r["s_e"] - 1 / 0.6) < 1e-14
