"""FP64 CPU oracle for the MRTLB-VANSE step -- TEST INFRASTRUCTURE ONLY.

This package wraps ``vanse_oracle.c``, a plain, slow FP64 restatement of one time
step of the consistent MRT lattice Boltzmann method for the volume-averaged
Navier-Stokes equations (arXiv:2409.02964, Sec. 2.3, Eq. (5)-(7), (10),
(13)-(20), (A1)). Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the CUDA library never does, and the two share
no code.

Parity status of every function is recorded in the C file's header: all are
pinned by the tests in ``tests/test_oracle_*.py``.

Layouts (numpy, C order, float64): fields ``[ny, nx]``; populations
``[9, ny, nx]`` holding the post-streaming f_i(x, t); body force ``[2, ny, nx]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vanse_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libvanse_oracle.so")

Q = 9


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("s_c", ctypes.c_double), ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double),
        ("s_q", ctypes.c_double), ("s_nu", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("model_b", ctypes.c_int),
        ("nthreads", ctypes.c_int),
        ("eq_order", ctypes.c_int),
        ("drag_d0", ctypes.c_double), ("drag_d1", ctypes.c_double),
        ("us_x", ctypes.c_double), ("us_y", ctypes.c_double),
        ("nee_top", ctypes.c_int), ("uw_x", ctypes.c_double), ("uw_y", ctypes.c_double),
    ]


@dataclass
class Params:
    """Problem statement of one lattice (rates are the diagonal of Gamma, Sec. 2.3)."""
    nx: int
    ny: int
    s_nu: float
    s_e: float
    s_eps: float = 1.2
    s_q: float = 1.4
    s_c: float = 1.0
    kappa: float = 0.5
    bc_x: int = 0          # 0 periodic, 1 half-way bounce-back walls
    bc_y: int = 0
    model_b: int = 0
    nthreads: int = 1
    eq_order: int = 3      # 2: App. B equilibrium and penalty
    drag_d0: float = 0.0   # F^B += -beta (u - u_s), beta = phi^2 (d0 + d1 (1 - phi))
    drag_d1: float = 0.0
    us_x: float = 0.0
    us_y: float = 0.0
    nee_top: int = 0       # with bc_y = 1: row ny-1 is a moving wall (non-equilibrium extrapolation)
    uw_x: float = 0.0      # its velocity
    uw_y: float = 0.0

    def c(self) -> _Params:
        return _Params(self.nx, self.ny, self.s_c, self.s_e, self.s_eps, self.s_q,
                       self.s_nu, self.kappa, self.bc_x, self.bc_y, self.model_b,
                       self.nthreads, self.eq_order, self.drag_d0, self.drag_d1, self.us_x, self.us_y,
                       self.nee_top, self.uw_x, self.uw_y)


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile the oracle into ``oracle/_build/libvanse_oracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            _SRC, "-o", _LIB + ".tmp", "-lm"]
    cmds = [base[:1] + ["-fopenmp"] + base[1:]] if openmp else []
    cmds.append(base)
    err = None
    for cmd in cmds:
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(_LIB + ".tmp", _LIB)
            return _LIB
        err = r.stderr
    raise RuntimeError(f"oracle build failed:\n{err}")


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        d = ctypes.c_double
        L.vo_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), dp]
        L.vo_M.argtypes = [dp]
        L.vo_Minv.argtypes = [dp]
        L.vo_moments.argtypes = [dp, dp]
        L.vo_feq.argtypes = [d, d, d, d, d, dp]
        L.vo_guo_force.argtypes = [d, d, d, d, dp]
        L.vo_meq.argtypes = [d, d, d, d, d, dp]
        L.vo_force_moments.argtypes = [d, d, d, d, dp]
        L.vo_penalty.argtypes = [d, d, d, dp, dp, dp, d, ctypes.c_int, dp]
        L.vo_feq_order.argtypes = [ctypes.c_int, d, d, d, d, d, dp]
        L.vo_meq_order.argtypes = [ctypes.c_int, d, d, d, d, d, dp]
        L.vo_penalty_order.argtypes = [ctypes.c_int, d, d, d, dp, dp, dp, d, ctypes.c_int, dp]
        L.vo_gradient.argtypes = [pp, dp, ctypes.c_int, dp, dp]
        L.vo_macros.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.vo_step.argtypes = [pp, dp, dp, dp, dp, dp]
        L.vo_step.restype = ctypes.c_int
        L.vo_init.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        L.vo_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------- point functions
def lattice():
    """Eq. (5): (e [9,2] int, w [9])."""
    e = np.zeros((Q, 2), dtype=np.int32)
    w = np.zeros(Q)
    lib().vo_lattice(e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(w))
    return e.astype(np.int64), w


def M():
    m = np.zeros((Q, Q))
    lib().vo_M(_p(m))
    return m


def Minv():
    m = np.zeros((Q, Q))
    lib().vo_Minv(_p(m))
    return m


def moments(f):
    f = _f64(f)
    m = np.zeros(Q)
    lib().vo_moments(_p(f), _p(m))
    return m


def feq(kappa, phi, rho, ux, uy, order=3):
    """Eq. (14) (order 3) or Eq. (B1) (order 2)."""
    out = np.zeros(Q)
    lib().vo_feq_order(int(order), kappa, phi, rho, ux, uy, _p(out))
    return out


def guo_force(ux, uy, Fx, Fy):
    out = np.zeros(Q)
    lib().vo_guo_force(ux, uy, Fx, Fy, _p(out))
    return out


def meq(kappa, phi, rho, ux, uy, order=3):
    """Eq. (18) (order 3) or Eq. (B2) (order 2)."""
    out = np.zeros(Q)
    lib().vo_meq_order(int(order), kappa, phi, rho, ux, uy, _p(out))
    return out


def force_moments(ux, uy, Fx, Fy):
    out = np.zeros(Q)
    lib().vo_force_moments(ux, uy, Fx, Fy, _p(out))
    return out


def penalty(kappa, phi, rho, dA, dB, dD, dtphi, model_b=0, order=3):
    """Eq. (20) (order 3) or Eq. (B3) (order 2). dX = (d_x X_x, d_y X_y, d_x X_y, d_y X_x)
    for X = rho u, u, phi rho u."""
    out = np.zeros(Q)
    lib().vo_penalty_order(int(order), kappa, phi, rho, _p(_f64(dA)), _p(_f64(dB)), _p(_f64(dD)), dtphi,
                           int(model_b), _p(out))
    return out


# ------------------------------------------------------------- field functions
def gradient(params: Params, psi, odd=False):
    psi = _f64(psi)
    gx = np.zeros_like(psi)
    gy = np.zeros_like(psi)
    pc = params.c()
    lib().vo_gradient(ctypes.byref(pc), _p(psi), int(odd), _p(gx), _p(gy))
    return gx, gy


def macros(params: Params, f, phi, fb=None):
    """Eq. (7), (13): returns dict rho, ux, uy, Fx, Fy, p."""
    f = _f64(f)
    phi = _f64(phi)
    fb = _f64(fb)
    shp = phi.shape
    out = {k: np.zeros(shp) for k in ("rho", "ux", "uy", "Fx", "Fy")}
    pc = params.c()
    lib().vo_macros(ctypes.byref(pc), _p(f), _p(phi), _p(fb), _p(out["rho"]),
                    _p(out["ux"]), _p(out["uy"]), _p(out["Fx"]), _p(out["Fy"]))
    out["p"] = out["rho"] / 3.0
    return out


def step(params: Params, f, phi_t, phi_next=None, fb=None):
    """One time step (Eq. 16 + streaming). Returns the new post-streaming f."""
    f = _f64(f)
    out = np.empty_like(f)
    pc = params.c()
    lib().vo_step(ctypes.byref(pc), _p(f), _p(out), _p(_f64(phi_t)), _p(_f64(phi_next)),
                  _p(_f64(fb)))
    return out


def init(params: Params, rho, ux, uy, phi, fb=None):
    """Initial populations f = f^eq - F_i/2 (reading c7)."""
    rho = _f64(rho)
    f = np.zeros((Q,) + rho.shape)
    pc = params.c()
    lib().vo_init(ctypes.byref(pc), _p(rho), _p(_f64(ux)), _p(_f64(uy)), _p(_f64(phi)),
                  _p(_f64(fb)), _p(f))
    return f


def max_threads() -> int:
    return int(lib().vo_max_threads())


def rates_from_tau(tau_nu: float, s_eps: float = 1.2, s_q: float = 1.4):
    """Relaxation time tau_nu -> rates: s_nu = 1/tau_nu, nu = (tau_nu - 1/2)/3, and
    s_e from the bulk viscosity nu_e = nu/3 that App. A (Eq. A12) requires."""
    s_nu = 1.0 / tau_nu
    nu = (tau_nu - 0.5) / 3.0
    nu_e = nu / 3.0
    s_e = 1.0 / (3.0 * nu_e + 0.5)
    return dict(s_nu=s_nu, s_e=s_e, s_eps=s_eps, s_q=s_q)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
