"""TEST INFRASTRUCTURE ONLY: the gradient of an outlet-momentum objective with
respect to the void fraction, by reverse-mode differentiation of a plain FP64
PyTorch (CPU) restatement of the time step.

The step is written out again here with tensor operations, in the paper's order
(Eq. 7, 10, 13 for rho, F, u; Eq. 17-20 and 16 for the collision in moment space;
(A1) for the back-transform; streaming with half-way bounce-back, Sec. 3.1), so
that torch.autograd can differentiate it exactly. It is pinned to the C oracle
(vanse_oracle.c) by equal forward results, and its gradient to central finite
differences of the C oracle's objective (tests/test_oracle_adjoint.py). It shares
no code with the CUDA library.

Problem (the differentiation workload): phi(x) is steady; F^B = phi g with a
constant g; the populations start at f(0) = f^eq(rho = 1, u = 0, phi) - F_i/2
(F^p = 0 for uniform rho); after each step n the objective samples
    O(n) = sum over y of (phi rho u_x)(x_out, y) = sum_y (j_x + F_x / 2)(x_out, y)
and J = (1 / (avg_steps * ny)) * sum of O(n) over the last avg_steps steps
n = nsteps - avg_steps + 1 .. nsteps.

Layout as the C oracle: fields [ny][nx], populations [9][ny][nx].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

# D2Q9 (Eq. 5): rest, the four axis directions counter-clockwise from +x, then the
# four diagonals counter-clockwise from (+1, +1)
_E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
_W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
_OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]


def _moment_matrix() -> torch.Tensor:
    """Rows of M (Eq. 17): 1, e = -4 + 3|e|^2, eps = 4 - 21|e|^2/2 + 9|e|^4/2,
    e_x, q_x = (-5 + 3|e|^2) e_x, e_y, q_y, e_x^2 - e_y^2, e_x e_y."""
    rows = []
    for ex, ey in _E:
        c2 = ex * ex + ey * ey
        rows.append([1.0, -4.0 + 3.0 * c2, 4.0 - 10.5 * c2 + 4.5 * c2 * c2, ex, (-5.0 + 3.0 * c2) * ex, ey,
                     (-5.0 + 3.0 * c2) * ey, ex * ex - ey * ey, ex * ey])
    return torch.tensor(rows, dtype=torch.float64).T.contiguous()


@dataclass
class Problem:
    nx: int
    ny: int
    s_nu: float
    s_e: float
    s_eps: float
    s_q: float
    s_c: float = 1.0
    kappa: float = 0.5
    wall_y: bool = True
    model_b: bool = False
    gx: float = 1e-6
    gy: float = 0.0


class _Grid:
    """Index maps of the lattice: Eq. (10) neighbours with the wall ghost rule and
    the streaming permutation."""

    def __init__(self, pb: Problem):
        nx, ny = pb.nx, pb.ny
        yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        self.nb, self.sg = [], []   # per direction: neighbour flat index, sign of a vector field there
        for ex, ey in _E:
            x2 = (xx + ex) % nx
            y2 = yy + ey
            wall = np.zeros_like(y2, dtype=bool)
            if pb.wall_y:
                lo, hi = y2 < 0, y2 >= ny
                wall = lo | hi
                y2 = np.where(lo, -1 - y2, np.where(hi, 2 * ny - 1 - y2, y2))
            else:
                y2 = y2 % ny
            self.nb.append(torch.from_numpy((y2 * nx + x2).ravel()))
            self.sg.append(torch.from_numpy(np.where(wall, -1.0, 1.0).ravel()))
        # streaming: destination (plane, cell) of every (plane, cell) of f^+
        n = nx * ny
        dest = np.empty(9 * n, dtype=np.int64)
        for i, (ex, ey) in enumerate(_E):
            xd, yd = xx + ex, yy + ey
            xd = xd % nx
            leave = np.zeros_like(yd, dtype=bool)
            if pb.wall_y:
                leave = (yd < 0) | (yd >= ny)
            else:
                yd = yd % ny
            same = (yy * nx + xx).ravel()
            moved = (np.where(leave, 0, yd) * nx + xd).ravel()
            d = np.where(leave.ravel(), _OPP[i] * n + same, i * n + moved)
            dest[i * n:(i + 1) * n] = d
        src = np.empty_like(dest)
        src[dest] = np.arange(9 * n)
        self.stream_src = torch.from_numpy(src)   # f_new.flat[k] = f_plus.flat[stream_src[k]]


def _grad(psi: torch.Tensor, g: _Grid, odd: bool):
    """Eq. (10): d_a psi = 3 sum_i w_i psi(x + e_i) e_ia, psi flat [n]."""
    gx = torch.zeros_like(psi)
    gy = torch.zeros_like(psi)
    for i, (ex, ey) in enumerate(_E):
        if ex == 0 and ey == 0:
            continue
        v = psi[g.nb[i]]
        if odd:
            v = v * g.sg[i]
        gx = gx + (3.0 * _W[i] * ex) * v
        gy = gy + (3.0 * _W[i] * ey) * v
    return gx, gy


def _macros(f: torch.Tensor, phi: torch.Tensor, pb: Problem, g: _Grid):
    """Eq. (7), (10), (13) on flat fields: s = sum f, rho, j, F, u."""
    s = f.sum(0)
    jx = sum(ex * f[i] for i, (ex, _) in enumerate(_E) if ex)
    jy = sum(ey * f[i] for i, (_, ey) in enumerate(_E) if ey)
    rho = s / phi
    drx, dry = _grad(rho, g, odd=False)
    kp = (pb.kappa - 1.0) if pb.model_b else (pb.kappa - phi)
    Fx = kp / 3.0 * drx + phi * pb.gx
    Fy = kp / 3.0 * dry + phi * pb.gy
    ux = (jx + 0.5 * Fx) / s
    uy = (jy + 0.5 * Fy) / s
    return s, jx, jy, rho, Fx, Fy, ux, uy


def step(f: torch.Tensor, phi: torch.Tensor, pb: Problem, g: _Grid, M: torch.Tensor, Minv: torch.Tensor):
    """One time step (steady phi, so d_t phi = 0); f flat [9, n]."""
    s, jx, jy, rho, Fx, Fy, ux, uy = _macros(f, phi, pb, g)
    # Eq. (20) fields and their Eq. (10) gradients
    dAxx, _ = _grad(rho * ux, g, True)
    _, dAyy = _grad(rho * uy, g, True)
    dBxx, dByx = _grad(ux, g, True)      # d_x u_x, d_y u_x
    dBxy, dByy = _grad(uy, g, True)      # d_x u_y, d_y u_y
    dDxx, _ = _grad(phi * rho * ux, g, True)
    _, dDyy = _grad(phi * rho * uy, g, True)
    X = pb.kappa / phi
    kp = (pb.kappa - 1.0) if pb.model_b else (pb.kappa - phi)
    Ca = -pb.kappa * (dAxx + dAyy) + 2.0 * kp * rho * (dBxx + dByy) + (3.0 - 2.0 * X) * (dDxx + dDyy)
    Cb = -pb.kappa * (dAxx - dAyy) + (2.0 / 3.0) * kp * rho * (dBxx - dByy) + (dDxx - dDyy)
    Cc = (1.0 / 3.0) * kp * rho * (dBxy + dByx)
    # Eq. (18) with phi rho = sum f; Eq. (19)
    pr = phi * rho
    uu = ux * ux + uy * uy
    meq = torch.stack([pr, pr * (-4.0 + 3.0 * uu + 2.0 * X), pr * (4.0 - 3.0 * uu - 3.0 * X), pr * ux,
                       pr * (X - 2.0) * ux, pr * uy, pr * (X - 2.0) * uy, pr * (ux * ux - uy * uy), pr * ux * uy])
    uF = ux * Fx + uy * Fy
    zero = torch.zeros_like(uF)
    S = torch.stack([zero, 6.0 * uF, -6.0 * uF, Fx, -Fx, Fy, -Fy, 2.0 * (ux * Fx - uy * Fy), ux * Fy + uy * Fx])
    C = torch.stack([zero, Ca, zero, zero, zero, zero, zero, Cb, Cc])
    G = torch.tensor([pb.s_c, pb.s_e, pb.s_eps, pb.s_c, pb.s_q, pb.s_c, pb.s_q, pb.s_nu, pb.s_nu],
                     dtype=torch.float64)[:, None]
    m = M @ f
    mp = m - G * (m - meq) + (1.0 - 0.5 * G) * (S + C)     # Eq. (16)
    fplus = Minv @ mp
    return fplus.reshape(-1)[g.stream_src].reshape(9, -1)


def initial(phi: torch.Tensor, pb: Problem):
    """f(0) = f^eq(1, 0, phi) - F_i(0, phi g)/2 (Eq. 14, 6; F^p = 0 at uniform rho)."""
    rows = []
    for i, (ex, ey) in enumerate(_E):
        feq = (phi - (5.0 / 9.0) * pb.kappa) if i == 0 else torch.full_like(phi, _W[i] * pb.kappa)
        Fi = _W[i] * 3.0 * (ex * pb.gx + ey * pb.gy) * phi
        rows.append(feq - 0.5 * Fi)
    return torch.stack(rows)


def objective(phi_np, pb: Problem, nsteps: int, avg_steps: int, x_out: int | None = None,
              grad: bool = True, segment: int = 0):
    """J and (if grad) dJ/dphi as numpy arrays [ny][nx]. segment > 0 recomputes the
    forward in segments of that many steps during the backward pass (memory)."""
    g = _Grid(pb)
    M = _moment_matrix()
    Minv = torch.linalg.inv(M)
    x_out = pb.nx - 1 if x_out is None else x_out
    cols = torch.arange(pb.ny) * pb.nx + x_out
    phi = torch.tensor(np.asarray(phi_np, dtype=np.float64).ravel(), requires_grad=grad)

    def sample(f):
        s, jx, jy, rho, Fx, Fy, ux, uy = _macros(f, phi, pb, g)
        return (jx + 0.5 * Fx)[cols].sum()

    def run(f, n0, n1):
        acc = torch.zeros((), dtype=torch.float64)
        for n in range(n0, n1):
            f = step(f, phi, pb, g, M, Minv)
            if n + 1 > nsteps - avg_steps:
                acc = acc + sample(f)
        return f, acc

    f = initial(phi, pb)
    total = torch.zeros((), dtype=torch.float64)
    if segment > 0:
        from torch.utils.checkpoint import checkpoint
        for n0 in range(0, nsteps, segment):
            n1 = min(nsteps, n0 + segment)
            f, acc = checkpoint(lambda ff, a=n0, b=n1: run(ff, a, b), f, use_reentrant=False)
            total = total + acc
    else:
        f, total = run(f, 0, nsteps)
    J = total / (avg_steps * pb.ny)
    if not grad:
        return float(J.detach())
    J.backward()
    return float(J.detach()), phi.grad.numpy().reshape(pb.ny, pb.nx).copy()
