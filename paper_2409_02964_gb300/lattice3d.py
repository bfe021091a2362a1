"""Python handle for one 3-D (D3Q19) lattice of the CUDA library (argument marshalling only).

Every step of the method runs in ``liblbm_vanse.so`` (``include/lbm_vanse3d.h``).
Inputs may be CUDA tensors (passed by device pointer) or host arrays (copied by the
library); outputs are float64 CUDA tensors. Fields are shaped [nz, ny, nx], vector
fields [3, nz, ny, nx], populations [19, nz, ny, nx].
"""
from __future__ import annotations

import ctypes

import torch

from . import capi
from .lattice import _BC, LbmError, _Arg

_STORAGE3 = {"fp64": capi.LBM_FP64, "fp32": capi.LBM_FP32}


class Lattice3D:
    """One D3Q19 MRTLB-VANSE lattice on the current CUDA device: ``tau`` is the
    relaxation time of the stress moments; ``s_e <= 0`` derives the energy rate from
    nu_e = nu/3; ``s_eps``, ``s_q``, ``s_pi``, ``s_m`` are rates; x and z are periodic,
    ``bc_y`` is "periodic" or "bounceback"; ``storage`` is "fp32" or "fp64"."""

    def __init__(self, nx: int, ny: int, nz: int, tau: float = 0.8, *, s_e: float = 0.0, s_eps: float = 1.2,
                 s_q: float = 1.2, s_pi: float = 1.2, s_m: float = 1.2, kappa: float = 0.5, rho0: float = 1.0,
                 bc_y: str = "periodic", storage: str = "fp32", stream=None):
        L = capi.load()
        p = capi.default_params3d()
        p.nx, p.ny, p.nz, p.tau_nu = int(nx), int(ny), int(nz), float(tau)
        p.s_e, p.s_eps, p.s_q, p.s_pi, p.s_m = float(s_e), float(s_eps), float(s_q), float(s_pi), float(s_m)
        p.kappa, p.rho0 = float(kappa), float(rho0)
        p.bc_y, p.storage = _BC[bc_y], _STORAGE3[storage]
        self.nx, self.ny, self.nz, self.storage = int(nx), int(ny), int(nz), storage
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = L.lbm_vanse3d_create(ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != capi.LBM_OK:
            raise LbmError(st, L.lbm_vanse3d_last_error(None).decode())
        self._h = h
        self._L = L

    def _check(self, st: int) -> None:
        if st != capi.LBM_OK:
            msg = self._L.lbm_vanse3d_last_error(self._h)
            raise LbmError(st, msg.decode() if msg else "")

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._L.lbm_vanse3d_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def _dense(self, k: int = 1) -> torch.Tensor:
        shape = (self.nz, self.ny, self.nx) if k == 1 else (k, self.nz, self.ny, self.nx)
        return torch.empty(shape, dtype=torch.float64, device=self.device)

    def set_void_fraction(self, phi_t, phi_next=None) -> None:
        a, b = _Arg(phi_t, self.n, self.device), _Arg(phi_next, self.n, self.device)
        if phi_next is not None and a.on_device != b.on_device:
            raise ValueError("phi_t and phi_next must both be on the device or both on the host")
        self._check(self._L.lbm_vanse3d_set_void_fraction(self._h, a.ptr, b.ptr, a.on_device))

    def set_body_force(self, gx: float = 0.0, gy: float = 0.0, gz: float = 0.0, field=None) -> None:
        a = _Arg(field, 3 * self.n, self.device)
        self._check(self._L.lbm_vanse3d_set_body_force(self._h, float(gx), float(gy), float(gz), a.ptr,
                                                       a.on_device))

    def init_fields(self, rho, u) -> None:
        """rho [nz, ny, nx] and the physical velocity u [3, nz, ny, nx]."""
        r = _Arg(rho, self.n, self.device)
        if isinstance(u, torch.Tensor):
            comps = [u[k] for k in range(3)]
        else:
            comps = [u[0], u[1], u[2]]
        us = [_Arg(c, self.n, self.device) for c in comps]
        if len({r.on_device} | {x.on_device for x in us}) != 1:
            raise ValueError("rho and u must both be on the device or both on the host")
        self._check(self._L.lbm_vanse3d_init_fields(self._h, r.ptr, us[0].ptr, us[1].ptr, us[2].ptr, r.on_device))

    def step(self, nsteps: int = 1) -> None:
        self._check(self._L.lbm_vanse3d_step(self._h, int(nsteps)))

    def sync(self) -> None:
        self._check(self._L.lbm_vanse3d_sync(self._h))

    @property
    def step_count(self) -> int:
        return int(self._L.lbm_vanse3d_step_count(self._h))

    def get_populations(self) -> torch.Tensor:
        f = self._dense(19)
        self._check(self._L.lbm_vanse3d_get_populations(self._h, f.data_ptr(), 1))
        return f

    def set_populations(self, f) -> None:
        a = _Arg(f, 19 * self.n, self.device)
        self._check(self._L.lbm_vanse3d_set_populations(self._h, a.ptr, a.on_device))

    def macros(self) -> dict:
        rho, u = self._dense(), self._dense(3)
        self._check(self._L.lbm_vanse3d_macros(self._h, rho.data_ptr(), u.data_ptr(), 1))
        return {"rho": rho, "u": u, "p": rho / 3.0}

    def reduce(self):
        m = ctypes.c_double()
        mom = (ctypes.c_double * 3)()
        self._check(self._L.lbm_vanse3d_reduce(self._h, ctypes.byref(m), mom))
        return m.value, (mom[0], mom[1], mom[2])
