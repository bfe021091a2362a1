"""Python handle for a batch of independent lattices (argument marshalling only).

Each lattice is an n x n periodic MRTLB-VANSE lattice driven by the spatiotemporal
manufactured solution phi = phi0 + A sin(kx) sin(ky) cos(2 pi t / T) with the
body force of Eq. (25), evaluated inside the kernel. All lattices advance together,
one persistent kernel per step (``lbm_vanse_batch_step``), or one launch per
lattice per step (``step_each``) for comparison.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import capi
from .lattice import LbmError

_STORAGE = {"fp32": capi.LBM_FP32, "fp16": capi.LBM_FP16, "bf16": capi.LBM_BF16}


@dataclass(frozen=True)
class BatchLattice:
    n: int              # n x n cells
    tau: float          # shear relaxation time, nu = (tau - 1/2)/3
    amplitude: float    # A of the void fraction
    period: float       # T in steps
    u0: float           # U0 of the solenoidal part of phi u


def _check(st: int, handle) -> None:
    if st != capi.LBM_OK:
        msg = capi.load().lbm_vanse_batch_last_error(handle)
        raise LbmError(st, msg.decode() if msg else "")


class Batch:
    """Lattices of one batch on the current CUDA device (see ``lbm_vanse_batch_*``).

    ``s_e <= 0`` derives the energy rate of each lattice from nu_e = nu/3."""

    def __init__(self, lattices, *, storage: str = "fp32", s_e: float = 1.2, s_eps: float = 1.2,
                 s_q: float = 1.2, kappa: float = 0.5, rho0: float = 1.0, phi0: float = 0.7,
                 strip_rows: int = 0, eager: bool = False, stream=None):
        L = capi.load()
        self.lattices = [BatchLattice(*q) if not isinstance(q, BatchLattice) else q for q in lattices]
        arr = (capi.lbm_vanse_batch_lattice * len(self.lattices))()
        for a, q in zip(arr, self.lattices):
            a.n, a.tau_nu, a.amplitude, a.period, a.u0 = int(q.n), float(q.tau), float(q.amplitude), \
                float(q.period), float(q.u0)
        p = capi.batch_default_params()
        p.storage = _STORAGE[storage]
        p.s_e, p.s_eps, p.s_q = float(s_e), float(s_eps), float(s_q)
        p.kappa, p.rho0, p.phi0 = float(kappa), float(rho0), float(phi0)
        p.strip_rows, p.eager = int(strip_rows), int(bool(eager))
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(L.lbm_vanse_batch_create(arr, len(self.lattices), ctypes.byref(p),
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), None)
        self._h = h
        self.storage = storage

    def _call(self, name: str, *args) -> None:
        _check(getattr(capi.load(), name)(self._h, *args), self._h)

    def init(self) -> None:
        self._call("lbm_vanse_batch_init")

    def step(self, nsteps: int = 1) -> None:
        self._call("lbm_vanse_batch_step", int(nsteps))

    def step_each(self, nsteps: int = 1) -> None:
        self._call("lbm_vanse_batch_step_each", int(nsteps))

    def autotune(self, trial_steps: int = 20) -> int:
        rows = ctypes.c_int()
        self._call("lbm_vanse_batch_autotune", int(trial_steps), ctypes.byref(rows))
        return rows.value

    def velocity_error(self, index: int) -> tuple[float, float]:
        """Eq. (26) sums (sum |u - u_ref|^2, sum |u_ref|^2) of one lattice at the current step."""
        num, den = ctypes.c_double(), ctypes.c_double()
        self._call("lbm_vanse_batch_velocity_error", int(index), ctypes.byref(num), ctypes.byref(den))
        return num.value, den.value

    def relative_error(self, index: int) -> float:
        num, den = self.velocity_error(index)
        return (num / den) ** 0.5

    def populations(self, index: int) -> torch.Tensor:
        """Post-streaming populations of one lattice, float64 [9, n, n] on the device."""
        n = self.lattices[index].n
        out = torch.empty((9, n, n), dtype=torch.float64, device=self.device)
        self._call("lbm_vanse_batch_get_populations", int(index), ctypes.c_void_p(out.data_ptr()), 1)
        return out

    @property
    def cells(self) -> int:
        return int(capi.load().lbm_vanse_batch_cells(self._h))

    @property
    def step_count(self) -> int:
        return int(capi.load().lbm_vanse_batch_step_count(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            capi.load().lbm_vanse_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
