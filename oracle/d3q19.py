"""FP64 CPU oracle for the 3-D (D3Q19) MRTLB-VANSE step -- TEST INFRASTRUCTURE ONLY.

Wraps ``vanse3d_oracle.c``: the scheme of arXiv:2409.02964 (Sec. 2.3) carried to
three dimensions on D3Q19, with the equilibrium moments and the penalty source
derived for that lattice as the C file's header states. Only ``tests/`` and
``__graft_entry__`` may import it; the CUDA library never does.

Layouts (numpy, C order, float64): fields ``[nz, ny, nx]``; populations
``[19, nz, ny, nx]`` (post-streaming f_i(x, t)); body force ``[3, nz, ny, nx]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vanse3d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libvanse3d_oracle.so")

Q = 19


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("s_c", ctypes.c_double), ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double),
        ("s_q", ctypes.c_double), ("s_nu", ctypes.c_double), ("s_pi", ctypes.c_double),
        ("s_m", ctypes.c_double), ("kappa", ctypes.c_double),
        ("bc_y", ctypes.c_int), ("nthreads", ctypes.c_int), ("no_penalty", ctypes.c_int),
    ]


@dataclass
class Params:
    """One 3-D lattice: sizes, the diagonal of Gamma, kappa and the y boundary."""
    nx: int
    ny: int
    nz: int
    s_nu: float
    s_e: float = 1.0 / 0.6  # nu_e = nu/3 at nu = 0.1 (rates_from_tau gives it for any tau)
    s_eps: float = 1.2
    s_q: float = 1.2
    s_pi: float = 1.2
    s_m: float = 1.2
    s_c: float = 1.0
    kappa: float = 0.5
    bc_y: int = 0          # 0 periodic, 1 half-way bounce-back walls
    nthreads: int = 1
    no_penalty: int = 0    # tests only: drop the penalty source (a planted mistake)

    def c(self) -> _Params:
        return _Params(self.nx, self.ny, self.nz, self.s_c, self.s_e, self.s_eps, self.s_q, self.s_nu,
                       self.s_pi, self.s_m, self.kappa, self.bc_y, self.nthreads, self.no_penalty)


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile ``vanse3d_oracle.c`` into ``oracle/_build/libvanse3d_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", _LIB + ".tmp", "-lm"]
    cmds = ([base[:1] + ["-fopenmp"] + base[1:]] if openmp else []) + [base]
    err = None
    for cmd in cmds:
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(_LIB + ".tmp", _LIB)
            return _LIB
        err = r.stderr
    raise RuntimeError(f"3-D oracle build failed:\n{err}")


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        d = ctypes.c_double
        L.v3_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), dp]
        L.v3_M.argtypes = [dp]
        L.v3_Minv.argtypes = [dp]
        L.v3_moments.argtypes = [dp, dp]
        L.v3_meq.argtypes = [d, d, d, d, d, d, dp]
        L.v3_feq.argtypes = [d, d, d, d, d, d, dp]
        L.v3_guo_force.argtypes = [d, d, d, d, d, d, dp]
        L.v3_force_moments.argtypes = [d, d, d, d, d, d, dp]
        L.v3_penalty.argtypes = [d, d, d, dp, dp, dp, d, dp]
        L.v3_gradient.argtypes = [pp, dp, ctypes.c_int, dp, dp, dp]
        L.v3_macros.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        L.v3_step.argtypes = [pp, dp, dp, dp, dp, dp]
        L.v3_step.restype = ctypes.c_int
        L.v3_init.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp]
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def lattice():
    """D3Q19: (e [19, 3] int, w [19])."""
    e = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    lib().v3_lattice(e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(w))
    return e.astype(np.int64), w


def M():
    m = np.zeros((Q, Q))
    lib().v3_M(_p(m))
    return m


def Minv():
    m = np.zeros((Q, Q))
    lib().v3_Minv(_p(m))
    return m


def feq(kappa, phi, rho, u):
    out = np.zeros(Q)
    lib().v3_feq(kappa, phi, rho, u[0], u[1], u[2], _p(out))
    return out


def meq(kappa, phi, rho, u):
    out = np.zeros(Q)
    lib().v3_meq(kappa, phi, rho, u[0], u[1], u[2], _p(out))
    return out


def guo_force(u, F):
    out = np.zeros(Q)
    lib().v3_guo_force(u[0], u[1], u[2], F[0], F[1], F[2], _p(out))
    return out


def force_moments(u, F):
    out = np.zeros(Q)
    lib().v3_force_moments(u[0], u[1], u[2], F[0], F[1], F[2], _p(out))
    return out


def penalty(kappa, phi, rho, dA, dB, dD, dtphi):
    """dA[a] = d_a (rho u)_a, dB[a, b] = d_a u_b, dD[a] = d_a (phi rho u)_a."""
    out = np.zeros(Q)
    lib().v3_penalty(kappa, phi, rho, _p(_f64(dA)), _p(_f64(np.asarray(dB).reshape(9))), _p(_f64(dD)),
                     dtphi, _p(out))
    return out


def gradient(params: Params, psi, odd=False):
    psi = _f64(psi)
    g = [np.zeros_like(psi) for _ in range(3)]
    pc = params.c()
    lib().v3_gradient(ctypes.byref(pc), _p(psi), int(odd), *(_p(x) for x in g))
    return g


def macros(params: Params, f, phi, fb=None):
    """Eq. (7), (13) in 3-D: dict rho [nz,ny,nx], F [3,...], u [3,...], p = rho/3."""
    f = _f64(f)
    phi = _f64(phi)
    rho = np.zeros_like(phi)
    F = np.zeros((3,) + phi.shape)
    u = np.zeros((3,) + phi.shape)
    pc = params.c()
    lib().v3_macros(ctypes.byref(pc), _p(f), _p(phi), _p(_f64(fb)), _p(rho), _p(F), _p(u))
    return {"rho": rho, "F": F, "u": u, "p": rho / 3.0}


def step(params: Params, f, phi_t, phi_next=None, fb=None):
    f = _f64(f)
    out = np.empty_like(f)
    pc = params.c()
    lib().v3_step(ctypes.byref(pc), _p(f), _p(out), _p(_f64(phi_t)), _p(_f64(phi_next)), _p(_f64(fb)))
    return out


def init(params: Params, rho, u, phi, fb=None):
    """f = f^eq - F_i/2; u is [3, nz, ny, nx]."""
    rho = _f64(rho)
    u = _f64(u)
    f = np.zeros((Q,) + rho.shape)
    pc = params.c()
    lib().v3_init(ctypes.byref(pc), _p(rho), _p(np.ascontiguousarray(u[0])), _p(np.ascontiguousarray(u[1])),
                  _p(np.ascontiguousarray(u[2])), _p(_f64(phi)), _p(_f64(fb)), _p(f))
    return f


def rates_from_tau(tau_nu: float, s_eps: float = 1.2, s_q: float = 1.2, s_pi: float = 1.2, s_m: float = 1.2):
    """Relaxation time -> rates for the 3-D scheme: s_nu = 1/tau_nu and s_e from
    nu_e = nu/3 as in 2-D (the 3-D stress then carries a bulk term 2/3 rho nu_e div u;
    nu_e = 0, s_e = 2, would give the Stokes form but leaves the energy mode undamped)."""
    nu = (tau_nu - 0.5) / 3.0
    return dict(s_nu=1.0 / tau_nu, s_e=1.0 / (nu + 0.5), s_eps=s_eps, s_q=s_q, s_pi=s_pi, s_m=s_m)
