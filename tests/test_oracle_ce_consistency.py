"""The penalty source against the Chapman-Enskog bookkeeping, evaluated numerically.

App. A obtains the penalty C (Eq. 20) as what the first-order non-equilibrium of
each stress moment has in excess of the target stress: with the first-order
equations for d_t(phi rho) and d_t(phi rho u) (Eq. A8, force included),

    C_k = d_t m^eq_k + d_a (sum_i M_ki e_ia f^eq_i) - S_k - target_k,
    target_k = sum_ab A^k_ab T_ab,  T = cs^2 phi rho (grad u + grad u^T),

where A^k is the quadratic part of moment k's basis polynomial, up to the
O(|u|^2) terms the analysis neglects. This test evaluates the right-hand side at a
point from smooth analytic fields, with the oracle's equilibrium (f^eq, m^eq) and
force moments as the only scheme ingredients and every derivative a central
difference, and compares it with the oracle's penalty. On D2Q9 the same machinery
must return the printed Eq. (20) (with App. B's equilibrium the printed (B3), and
model B's);
on D3Q19 it checks the penalty derived for that lattice. Measured residuals are 1e-14 to 2e-12 against terms of 1e-7 to 2e-2 (the
smallest, the shear term, is 3e-7), so a wrong coefficient or a dropped term in any
of them fails by orders of magnitude.
"""
import numpy as np
import pytest

import oracle as O2
from oracle import d3q19 as O3

KAPPA = 0.5
DTPHI = 2e-3
U = 1e-4
H = 1e-4  # spatial step of the central differences


def _fields(d):
    a = np.array([0.31, -0.22, 0.17][:d])
    b = np.array([0.13, 0.27, -0.19][:d])
    c = [np.array(v[:d]) for v in ([0.21, 0.11, -0.3], [-0.14, 0.25, 0.09], [0.18, -0.07, 0.23])]
    phi = lambda x: 0.7 + 0.1 * np.sin(a @ x + 0.3)            # noqa: E731
    rho = lambda x: 1.0 + 0.02 * np.sin(b @ x + 0.7)           # noqa: E731
    ph = [0.1, 0.4, -0.2]
    u = lambda x: U * np.array([np.sin(c[k] @ x + ph[k]) for k in range(d)])   # noqa: E731
    return phi, rho, u


def _grad(fn, x, d):
    return np.array([(fn(x + H * np.eye(d)[a]) - fn(x - H * np.eye(d)[a])) / (2 * H) for a in range(d)])


def _ce_penalty(d, x0, e, M, meq, feq, force_moments, F_of, stress, phi_in_target=True):
    phi, rho, u = _fields(d)
    Q = len(e)
    # fluxes sum_i M_ki e_ia f^eq_i at x, and their divergence at x0
    def flux(x):
        f = feq(phi(x), rho(x), u(x))
        return np.einsum("ki,ia,i->ka", M, e, f)
    div_flux = sum((flux(x0 + H * np.eye(d)[a])[:, a] - flux(x0 - H * np.eye(d)[a])[:, a]) / (2 * H)
                   for a in range(d))
    # first-order time derivatives (Eq. A8 with the total force F)
    p0, r0, u0 = phi(x0), rho(x0), u(x0)
    F0 = F_of(x0)
    dt_m0 = -sum(_grad(lambda x, a=a: phi(x) * rho(x) * u(x)[a], x0, d)[a] for a in range(d))
    dt_j = np.array([
        -sum(_grad(lambda x, a=a, b=b: KAPPA * rho(x) / 3 * (a == b) + phi(x) * rho(x) * u(x)[a] * u(x)[b],
                   x0, d)[b] for b in range(d)) + F0[a]
        for a in range(d)])
    dt_rho = (dt_m0 - r0 * DTPHI) / p0
    dt_u = (dt_j - u0 * dt_m0) / (p0 * r0)
    # d_t m^eq by the chain rule, derivatives of m^eq with respect to its arguments
    def dm(arg, step):
        args_p = [p0, r0, u0.copy()]
        args_m = [p0, r0, u0.copy()]
        if arg == "phi":
            args_p[0] += step; args_m[0] -= step
        elif arg == "rho":
            args_p[1] += step; args_m[1] -= step
        else:
            args_p[2][arg] += step; args_m[2][arg] -= step
        return (meq(*args_p) - meq(*args_m)) / (2 * step)
    dt_meq = dm("phi", 1e-5) * DTPHI + dm("rho", 1e-5) * dt_rho + sum(dm(a, 1e-6) * dt_u[a] for a in range(d))
    S = force_moments(u0, F0)
    gu = np.array([_grad(lambda x, b=b: u(x)[b], x0, d) for b in range(d)]).T   # gu[a, b] = d_a u_b
    T = (p0 if phi_in_target else 1.0) * r0 / 3 * (gu + gu.T)
    target = np.zeros(Q)
    for k, A in stress.items():
        target[k] = np.sum(A * T)
    return dt_meq + div_flux - S - target, gu


def _gradients(d, x0):
    phi, rho, u = _fields(d)
    dA = np.array([_grad(lambda x, a=a: rho(x) * u(x)[a], x0, d)[a] for a in range(d)])
    dD = np.array([_grad(lambda x, a=a: phi(x) * rho(x) * u(x)[a], x0, d)[a] for a in range(d)])
    return dA, dD


def _full_gradient(d, x0, fn_of_fields):
    """g[a, b] = d_a V_b for the vector field V = fn_of_fields(phi, rho, u) at x0."""
    phi, rho, u = _fields(d)
    return np.array([_grad(lambda x, b=b: fn_of_fields(phi(x), rho(x), u(x))[b], x0, d) for b in range(d)]).T


@pytest.mark.parametrize("order", [3, 2])
@pytest.mark.parametrize("x0", [(0.3, -1.2), (2.0, 0.7)])
def test_d2q9_bookkeeping_returns_eq_20_and_b3(x0, order):
    """order 3: the equilibrium of Eq. (14) and the printed Eq. (20); order 2: App. B's
    equilibrium (B1) and the printed (B3), which also reads the cross derivatives of
    rho u and phi rho u."""
    d = 2
    x0 = np.array(x0)
    e, _ = O2.lattice()
    M = O2.M()
    phi, rho, u = _fields(d)
    F_of = lambda x: (KAPPA - phi(x)) / 3 * _grad(rho, x, d)      # noqa: E731  F^p, no F^B
    stress = {1: 3 * np.eye(2), 7: np.diag([1.0, -1.0]), 8: np.array([[0, 0.5], [0.5, 0]])}
    ce, gu = _ce_penalty(d, x0, e.astype(float), M,
                         lambda p, r, v: O2.meq(KAPPA, p, r, v[0], v[1], order=order),
                         lambda p, r, v: O2.feq(KAPPA, p, r, v[0], v[1], order=order),
                         lambda v, F: O2.force_moments(v[0], v[1], F[0], F[1]), F_of, stress)
    gA = _full_gradient(d, x0, lambda p, r, v: r * v)
    gD = _full_gradient(d, x0, lambda p, r, v: p * r * v)
    # the oracle's penalty: dX = (d_x X_x, d_y X_y, d_x X_y, d_y X_x)
    cross = lambda g: [g[0, 0], g[1, 1], g[0, 1], g[1, 0]]      # noqa: E731
    C = O2.penalty(KAPPA, phi(x0), rho(x0), cross(gA), cross(gu), cross(gD), DTPHI, order=order)
    for k in stress:
        assert abs(ce[k] - C[k]) < 1e-11 + 1e-8 * abs(C[k]), (k, ce[k], C[k])
    assert abs(C[1]) > 1e-3      # the d_t phi term is exercised


@pytest.mark.parametrize("x0", [(0.3, -1.2, 0.5), (2.0, 0.7, -1.4)])
def test_d3q19_bookkeeping_returns_the_derived_penalty(x0):
    d = 3
    x0 = np.array(x0)
    e, _ = O3.lattice()
    M = O3.M()
    phi, rho, u = _fields(d)
    F_of = lambda x: (KAPPA - phi(x)) / 3 * _grad(rho, x, d)      # noqa: E731
    half = lambda a, b: np.array([[0.5 if {i, j} == {a, b} else 0 for j in range(3)] for i in range(3)])  # noqa: E731
    stress = {1: 19 * np.eye(3), 9: np.diag([2.0, -1.0, -1.0]), 11: np.diag([0.0, 1.0, -1.0]),
              13: half(0, 1), 14: half(1, 2), 15: half(0, 2)}
    ce, gu = _ce_penalty(d, x0, e.astype(float), M,
                         lambda p, r, v: O3.meq(KAPPA, p, r, v), lambda p, r, v: O3.feq(KAPPA, p, r, v),
                         lambda v, F: O3.force_moments(v, F), F_of, stress)
    dA, dD = _gradients(d, x0)
    C = O3.penalty(KAPPA, phi(x0), rho(x0), dA, gu, dD, DTPHI)
    for k in stress:
        assert abs(ce[k] - C[k]) < 1e-11 + 1e-8 * abs(C[k]), (k, ce[k], C[k])
    assert abs(C[1]) > 1e-3


@pytest.mark.parametrize("x0", [(0.3, -1.2), (2.0, 0.7)])
def test_d2q9_bookkeeping_returns_model_b(x0):
    """Model B (Sec. 2.3, VANSE set I): F^p = (kappa - 1) cs^2 grad rho and kappa - 1 in
    Eq. (20); its target stress is cs^2 rho (grad u + grad u^T), without phi."""
    d = 2
    x0 = np.array(x0)
    e, _ = O2.lattice()
    phi, rho, u = _fields(d)
    F_of = lambda x: (KAPPA - 1.0) / 3 * _grad(rho, x, d)      # noqa: E731
    stress = {1: 3 * np.eye(2), 7: np.diag([1.0, -1.0]), 8: np.array([[0, 0.5], [0.5, 0]])}
    ce, gu = _ce_penalty(d, x0, e.astype(float), O2.M(),
                         lambda p, r, v: O2.meq(KAPPA, p, r, v[0], v[1]),
                         lambda p, r, v: O2.feq(KAPPA, p, r, v[0], v[1]),
                         lambda v, F: O2.force_moments(v[0], v[1], F[0], F[1]), F_of, stress, phi_in_target=False)
    gA = _full_gradient(d, x0, lambda p, r, v: r * v)
    gD = _full_gradient(d, x0, lambda p, r, v: p * r * v)
    cross = lambda g: [g[0, 0], g[1, 1], g[0, 1], g[1, 0]]      # noqa: E731
    C = O2.penalty(KAPPA, phi(x0), rho(x0), cross(gA), cross(gu), cross(gD), DTPHI, model_b=1)
    for k in stress:
        assert abs(ce[k] - C[k]) < 1e-11 + 1e-8 * abs(C[k]), (k, ce[k], C[k])
