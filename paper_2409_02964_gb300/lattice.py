"""Python handle for one lattice of the CUDA library (argument marshalling only).

PyTorch provides device memory and the stream; every step of the method runs in
``liblbm_vanse.so``. Inputs may be CUDA tensors (passed by device pointer) or
host arrays (numpy / CPU tensors, copied by the library). Outputs are float64
CUDA tensors unless stated otherwise.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import capi

_STORAGE = {"fp64": capi.LBM_FP64, "fp32": capi.LBM_FP32, "fp16": capi.LBM_FP16, "bf16": capi.LBM_BF16}
_BC = {"periodic": capi.LBM_BC_PERIODIC, "bounceback": capi.LBM_BC_BOUNCEBACK}


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{capi.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st: int, handle) -> None:
    if st != capi.LBM_OK:
        msg = capi.load().lbm_vanse_last_error(handle)
        raise LbmError(st, msg.decode() if msg else "")


class _Arg:
    """Holds a caller array as (pointer, on_device) for one call, converted to
    ``dtype`` (float64, or float32 for the entry points that take floats)."""

    def __init__(self, a, count: int, device: torch.device, dtype=np.float64):
        if a is None:
            self.ptr, self.on_device, self._keep = None, 1, None
            return
        if isinstance(a, torch.Tensor) and a.is_cuda:
            if a.device != device:
                raise ValueError(f"tensor on {a.device}, lattice on {device}")
            t = a.detach().to({np.float64: torch.float64, np.float32: torch.float32}[dtype]).contiguous()
            if t.numel() != count:
                raise ValueError(f"expected {count} elements, got {t.numel()}")
            self.ptr, self.on_device, self._keep = t.data_ptr(), 1, t
        else:
            arr = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
            arr = np.ascontiguousarray(arr, dtype=dtype)
            if arr.size != count:
                raise ValueError(f"expected {count} elements, got {arr.size}")
            self.ptr, self.on_device, self._keep = arr.ctypes.data, 0, arr


def _check_out(out: torch.Tensor, device: torch.device) -> None:
    """An asynchronous result buffer: 3 contiguous float64 on the lattice's device or
    in pinned host memory."""
    if out.dtype != torch.float64 or out.numel() < 3 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 tensor of at least 3 elements")
    if out.is_cuda:
        if out.device != device:
            raise ValueError(f"tensor on {out.device}, lattice on {device}")
    elif not out.is_pinned():
        raise ValueError("a host out tensor must be in pinned memory")


def _is_f32(a) -> bool:
    return (isinstance(a, torch.Tensor) and a.dtype == torch.float32) or (
        isinstance(a, np.ndarray) and a.dtype == np.float32)


class Lattice:
    """One D2Q9 MRTLB-VANSE lattice on the current CUDA device.

    Parameters follow the paper's statement of the problem (Sec. 2.3, 3): ``tau``
    is the relaxation time of the shear moments (nu = (tau - 1/2)/3); ``s_e <= 0``
    derives the energy rate from nu_e = nu/3 (Eq. A12); ``s_eps``, ``s_q``, ``s_c``
    are rates; ``kappa`` is the provisional equation-of-state constant.
    ``dev_base="momentum"`` stores FP16 / BF16 deviations from f^rest plus the
    momentum term of the equilibrium (lbm_dev_base; kernel 5).
    """

    def __init__(self, nx: int, ny: int, tau: float = 0.8, *, s_e: float = 0.0, s_eps: float = 1.2,
                 s_q: float = 1.4, s_c: float = 1.0, kappa: float = 0.5, rho0: float = 1.0,
                 bc_y: str = "periodic", bc_x: str = "periodic", storage: str = "fp32", model_b: bool = False,
                 scale_log2: int | None = None, strip_rows: int = 0, eager: bool = False, kernel: int = 0,
                 eq_order: int = 3, dev_base: str = "rest", stream=None):
        L = capi.load()
        p = capi.default_params()
        p.nx, p.ny, p.tau_nu = int(nx), int(ny), float(tau)
        p.s_e, p.s_eps, p.s_q, p.s_c = float(s_e), float(s_eps), float(s_q), float(s_c)
        p.kappa, p.rho0 = float(kappa), float(rho0)
        p.bc_x, p.bc_y = _BC[bc_x], _BC[bc_y]
        p.storage, p.model_b = _STORAGE[storage], int(bool(model_b))
        if scale_log2 is not None:
            p.storage_scale_log2 = int(scale_log2)
        p.strip_rows = int(strip_rows)
        p.eager = int(bool(eager))
        p.kernel = int(kernel)
        p.eq_order = int(eq_order)
        p.dev_base = {"rest": capi.LBM_BASE_REST, "momentum": capi.LBM_BASE_MOMENTUM}[dev_base]
        self.nx, self.ny, self.storage = int(nx), int(ny), storage
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = L.lbm_vanse_create(ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != capi.LBM_OK:
            raise LbmError(st, L.lbm_vanse_last_error(None).decode())
        self._h = h
        self._L = L

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "_h", None):
            self._L.lbm_vanse_destroy(self._h)
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
        return self.nx * self.ny

    def _dense(self, k: int = 1) -> torch.Tensor:
        shape = (self.ny, self.nx) if k == 1 else (k, self.ny, self.nx)
        return torch.empty(shape, dtype=torch.float64, device=self.device)

    # -- inputs
    def set_void_fraction(self, phi_t, phi_next=None) -> None:
        """float32 arrays (numpy or torch) go through lbm_vanse_set_void_fraction_f32,
        everything else as float64 through lbm_vanse_set_void_fraction."""
        f32 = _is_f32(phi_t) and (phi_next is None or _is_f32(phi_next))
        dt = np.float32 if f32 else np.float64
        a, b = _Arg(phi_t, self.n, self.device, dt), _Arg(phi_next, self.n, self.device, dt)
        if phi_next is not None and a.on_device != b.on_device:
            raise ValueError("phi_t and phi_next must both be on the device or both on the host")
        fn = self._L.lbm_vanse_set_void_fraction_f32 if f32 else self._L.lbm_vanse_set_void_fraction
        _check(fn(self._h, a.ptr, b.ptr, a.on_device), self._h)

    def set_body_force(self, gx: float = 0.0, gy: float = 0.0, field=None) -> None:
        a = _Arg(field, 2 * self.n, self.device)
        _check(self._L.lbm_vanse_set_body_force(self._h, float(gx), float(gy), a.ptr, a.on_device), self._h)

    def set_drag(self, d0: float = 0.0, d1: float = 0.0, us_x: float = 0.0, us_y: float = 0.0) -> None:
        """F^B += -beta (u - u_s), beta = phi^2 (d0 + d1 (1 - phi)) (lbm_vanse_set_drag)."""
        _check(self._L.lbm_vanse_set_drag(self._h, float(d0), float(d1), float(us_x), float(us_y)), self._h)

    def set_solid_cells(self, enable: bool = True) -> None:
        """Cells with phi = 0 are solid (lbm_vanse_set_solid_cells; kernels 1 and 5,
        before init_fields)."""
        _check(self._L.lbm_vanse_set_solid_cells(self._h, int(enable)), self._h)

    def set_moving_wall(self, uw_x: float = 0.0, uw_y: float = 0.0, enable: bool = True) -> None:
        """Row ny-1 as a wall moving at (uw_x, uw_y) by non-equilibrium extrapolation
        (lbm_vanse_set_moving_wall; bounce-back walls, kernels 1 and 5)."""
        _check(self._L.lbm_vanse_set_moving_wall(self._h, int(enable), float(uw_x), float(uw_y)), self._h)

    def init_fields(self, rho, ux, uy) -> None:
        args = [_Arg(v, self.n, self.device) for v in (rho, ux, uy)]
        on = {a.on_device for a in args}
        if len(on) != 1:
            raise ValueError("rho, ux, uy must all be on the device or all on the host")
        _check(self._L.lbm_vanse_init_fields(self._h, args[0].ptr, args[1].ptr, args[2].ptr, on.pop()), self._h)

    # -- time stepping
    def step(self, nsteps: int = 1) -> None:
        _check(self._L.lbm_vanse_step(self._h, int(nsteps)), self._h)

    def sync(self) -> None:
        _check(self._L.lbm_vanse_sync(self._h), self._h)

    @property
    def step_count(self) -> int:
        return int(self._L.lbm_vanse_step_count(self._h))

    @property
    def bytes_per_cell(self) -> float:
        return float(self._L.lbm_vanse_bytes_per_cell(self._h))

    def launch_shape(self) -> dict:
        v = [ctypes.c_int() for _ in range(6)]
        _check(self._L.lbm_vanse_launch_shape(self._h, *[ctypes.byref(x) for x in v]), self._h)
        return dict(zip(("threads", "cols", "rows", "grid_x", "grid_y", "smem_bytes"), [x.value for x in v]))

    # -- outputs
    def macros(self) -> dict:
        rho, ux, uy, p = (self._dense() for _ in range(4))
        _check(self._L.lbm_vanse_macros(self._h, rho.data_ptr(), ux.data_ptr(), uy.data_ptr(), p.data_ptr(), 1),
               self._h)
        return {"rho": rho, "ux": ux, "uy": uy, "p": p}

    def get_populations(self) -> torch.Tensor:
        f = self._dense(9)
        _check(self._L.lbm_vanse_get_populations(self._h, f.data_ptr(), 1), self._h)
        return f

    def set_populations(self, f) -> None:
        a = _Arg(f, 9 * self.n, self.device)
        _check(self._L.lbm_vanse_set_populations(self._h, a.ptr, a.on_device), self._h)

    def save_state(self) -> np.ndarray:
        """A checkpoint of the whole lattice state (lbm_vanse_save_state) as a uint8
        array in host memory; load_state resumes from it bit for bit."""
        n = int(self._L.lbm_vanse_state_bytes(self._h))
        if n < 0:
            raise LbmError(capi.LBM_ERR_STATE, "lattice not initialised")
        buf = np.empty(n, dtype=np.uint8)
        _check(self._L.lbm_vanse_save_state(self._h, buf.ctypes.data, 0), self._h)
        return buf

    def load_state(self, state) -> None:
        """Resume from a state saved by save_state (a uint8 host array or CUDA tensor)."""
        if isinstance(state, torch.Tensor) and state.is_cuda:
            _check(self._L.lbm_vanse_load_state(self._h, state.data_ptr(), 1), self._h)
        else:
            arr = np.ascontiguousarray(state, dtype=np.uint8)
            _check(self._L.lbm_vanse_load_state(self._h, arr.ctypes.data, 0), self._h)

    def reduce(self):
        m, jx, jy = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self._L.lbm_vanse_reduce(self._h, ctypes.byref(m), ctypes.byref(jx), ctypes.byref(jy)), self._h)
        return m.value, jx.value, jy.value

    def step_sums(self, out: torch.Tensor) -> None:
        """One step that also queues the sums of the post-collision m_0 and j over the
        lattice into ``out`` (3 float64, on this device or pinned host memory), without
        waiting (lbm_vanse_step_sums)."""
        _check_out(out, self.device)
        _check(self._L.lbm_vanse_step_sums(self._h, out.data_ptr(), int(out.is_cuda)), self._h)

    def reduce_async(self, out: torch.Tensor) -> None:
        """Queue the mass and momentum sums into ``out`` (3 float64, on this device or
        in pinned host memory) without waiting; they are there once the stream has
        passed this point (e.g. a ``torch.cuda.Event`` recorded after the call)."""
        _check_out(out, self.device)
        _check(self._L.lbm_vanse_reduce_async(self._h, out.data_ptr(), int(out.is_cuda)), self._h)

    def velocity_error(self, ux_ref, uy_ref):
        a, b = _Arg(ux_ref, self.n, self.device), _Arg(uy_ref, self.n, self.device)
        num, den = ctypes.c_double(), ctypes.c_double()
        _check(self._L.lbm_vanse_velocity_error(self._h, a.ptr, b.ptr, a.on_device, ctypes.byref(num),
                                                ctypes.byref(den)), self._h)
        return num.value, den.value
