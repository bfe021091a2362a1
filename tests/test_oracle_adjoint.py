"""Pins of the FP64 autograd adjoint oracle (oracle/adjoint.py):

* its forward step and initial populations equal the C oracle's (itself pinned by
  test_oracle_identities / test_oracle_step) to rounding, on walled and periodic
  lattices with random populations and void fractions;
* its dJ/dphi equals central finite differences of J computed with the C oracle
  (a different implementation), at every cell of a small lattice.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as A


def _problem(nx, ny, wall_y, model_b=False, tau=0.7):
    return A.Problem(nx=nx, ny=ny, s_nu=1.0 / tau, s_e=1.2, s_eps=1.2, s_q=1.3, s_c=1.0, kappa=0.5,
                     wall_y=wall_y, model_b=model_b, gx=2e-5, gy=-1e-5)


def _c_params(O, pb):
    return O.Params(nx=pb.nx, ny=pb.ny, s_nu=pb.s_nu, s_e=pb.s_e, s_eps=pb.s_eps, s_q=pb.s_q, s_c=pb.s_c,
                    kappa=pb.kappa, bc_y=int(pb.wall_y), model_b=int(pb.model_b))


def _phi(nx, ny, seed):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return 0.6 + 0.2 * np.sin(2 * np.pi * x / nx + 1.0) * np.cos(2 * np.pi * y / ny) + 0.05 * rng.uniform(-1, 1, (ny, nx))


@pytest.mark.parametrize("wall_y", [True, False])
@pytest.mark.parametrize("model_b", [False, True])
def test_forward_step_equals_c_oracle(oracle_mod, wall_y, model_b):
    nx, ny = 11, 9
    pb = _problem(nx, ny, wall_y, model_b)
    phi = _phi(nx, ny, 3)
    rng = np.random.default_rng(4)
    f = np.array([w * (0.9 + 0.2 * rng.uniform(size=(ny, nx))) for w in A._W]) * 1.0
    f[0] += phi - 0.7
    fb = np.stack([phi * pb.gx, phi * pb.gy])
    want = oracle_mod.step(_c_params(oracle_mod, pb), f, phi, None, fb)
    g = A._Grid(pb)
    M = A._moment_matrix()
    got = A.step(torch.from_numpy(f.reshape(9, -1)), torch.from_numpy(phi.ravel()), pb, g, M, torch.linalg.inv(M))
    assert np.abs(got.numpy().reshape(9, ny, nx) - want).max() <= 1e-14 * np.abs(want).max()


def test_initial_equals_c_oracle(oracle_mod):
    nx, ny = 10, 7
    pb = _problem(nx, ny, True)
    phi = _phi(nx, ny, 5)
    want = oracle_mod.init(_c_params(oracle_mod, pb), np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), phi,
                           np.stack([phi * pb.gx, phi * pb.gy]))
    got = A.initial(torch.from_numpy(phi.ravel()), pb).numpy().reshape(9, ny, nx)
    assert np.abs(got - want).max() <= 1e-15


def _J_c(O, pb, phi, nsteps, avg):
    """J with the C oracle: init, nsteps steps, outlet samples of phi rho u_x."""
    prm = _c_params(O, pb)
    fb = np.stack([phi * pb.gx, phi * pb.gy])
    f = O.init(prm, np.ones_like(phi), np.zeros_like(phi), np.zeros_like(phi), phi, fb)
    acc = 0.0
    for n in range(nsteps):
        f = O.step(prm, f, phi, None, fb)
        if n + 1 > nsteps - avg:
            m = O.macros(prm, f, phi, fb)
            acc += np.sum((phi * m["rho"] * m["ux"])[:, -1])
    return acc / (avg * pb.ny)


@pytest.mark.parametrize("wall_y", [True, False])
def test_gradient_matches_central_differences_of_c_oracle(oracle_mod, wall_y):
    nx, ny, nsteps, avg = 8, 6, 14, 5
    pb = _problem(nx, ny, wall_y)
    phi = _phi(nx, ny, 7)
    J, grad = A.objective(phi, pb, nsteps, avg)
    # j_x is a difference of O(0.1) populations that is O(1e-4): FP64 rounding of the
    # populations alone moves J by ~1e-12 of itself
    assert abs(J - _J_c(oracle_mod, pb, phi, nsteps, avg)) <= 1e-10 * abs(J)
    # h = 1e-4: truncation ~ h^2 J''' / 6 and rounding ~ 1e-17 / h, both far below the bound
    h = 1e-4
    fd = np.zeros_like(phi)
    for y in range(ny):
        for x in range(nx):
            pp, pm = phi.copy(), phi.copy()
            pp[y, x] += h
            pm[y, x] -= h
            fd[y, x] = (_J_c(oracle_mod, pb, pp, nsteps, avg) - _J_c(oracle_mod, pb, pm, nsteps, avg)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.abs(grad - fd).max() <= 1e-6 * scale


def test_segmented_backward_equals_plain(oracle_mod):
    nx, ny, nsteps, avg = 9, 7, 12, 4
    pb = _problem(nx, ny, True)
    phi = _phi(nx, ny, 11)
    J0, g0 = A.objective(phi, pb, nsteps, avg)
    J1, g1 = A.objective(phi, pb, nsteps, avg, segment=5)
    assert J0 == J1
    assert np.abs(g0 - g1).max() <= 1e-14 * np.abs(g0).max()
