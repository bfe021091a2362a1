"""Gradient of the outlet-momentum objective with respect to the void fraction
(``lbm_vanse_outlet_momentum_grad``; argument marshalling only).

J(phi) is the mean of phi rho u_x over the outlet column and the last ``avg_steps``
of ``nsteps`` steps, from f(0) = f^eq(1, 0, phi) - F_i/2 with F^B = phi g; the
library computes J and dJ/dphi (FP64, discrete adjoint with checkpointing).
``OutletMomentum`` wraps the call as a torch.autograd.Function of phi.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import capi
from .lattice import LbmError


@dataclass(frozen=True)
class Channel:
    """Lattice and run of the objective (rates as in ``Lattice``)."""
    nx: int
    ny: int
    tau: float = 0.6
    s_e: float = 1.2
    s_eps: float = 1.2
    s_q: float = 1.2
    kappa: float = 0.5
    bc_y: str = "bounceback"
    model_b: bool = False
    gx: float = 1e-6
    gy: float = 0.0
    nsteps: int = 4000
    avg_steps: int = 100
    checkpoint_every: int = 200
    x_out: int = -1          # -1: the last column
    dense_segments: bool = False   # True: checkpoints and whole segments on the device


def _params(ch: Channel):
    p = capi.default_params()
    p.nx, p.ny, p.tau_nu = ch.nx, ch.ny, ch.tau
    p.s_e, p.s_eps, p.s_q = ch.s_e, ch.s_eps, ch.s_q
    p.kappa = ch.kappa
    p.bc_x = capi.LBM_BC_PERIODIC
    p.bc_y = capi.LBM_BC_BOUNCEBACK if ch.bc_y == "bounceback" else capi.LBM_BC_PERIODIC
    p.model_b = int(ch.model_b)
    p.storage = capi.LBM_FP64
    a = capi.lbm_vanse_adjoint_params()
    a.nsteps, a.avg_steps, a.checkpoint_every = ch.nsteps, ch.avg_steps, ch.checkpoint_every
    a.x_out = ch.x_out if ch.x_out >= 0 else ch.nx - 1
    a.gx, a.gy = ch.gx, ch.gy
    a.dense_segments = int(ch.dense_segments)
    return p, a


def outlet_momentum(phi, ch: Channel, grad: bool = True, stream=None):
    """Returns (J, dJ/dphi as a float64 CUDA tensor [ny, nx] or None, stats dict)."""
    L = capi.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    phi_t = torch.as_tensor(np.asarray(phi) if not isinstance(phi, torch.Tensor) else phi)
    phi_t = phi_t.detach().to(device=dev, dtype=torch.float64).contiguous()
    if phi_t.shape != (ch.ny, ch.nx):
        raise ValueError(f"phi has shape {tuple(phi_t.shape)}, expected {(ch.ny, ch.nx)}")
    stream = stream if stream is not None else torch.cuda.current_stream(dev)
    p, a = _params(ch)
    out = torch.empty_like(phi_t) if grad else None
    J = ctypes.c_double()
    st = capi.lbm_vanse_adjoint_stats()
    rc = L.lbm_vanse_outlet_momentum_grad(ctypes.byref(p), ctypes.byref(a), ctypes.c_void_p(phi_t.data_ptr()), 1,
                                          ctypes.c_void_p(stream.cuda_stream), ctypes.byref(J),
                                          ctypes.c_void_p(out.data_ptr()) if grad else None, ctypes.byref(st))
    if rc != capi.LBM_OK:
        msg = L.lbm_vanse_last_error(None)
        raise LbmError(rc, msg.decode() if msg else "")
    stats = {"forward_ms": st.forward_ms, "backward_ms": st.backward_ms, "device_bytes": st.device_bytes,
             "host_bytes": st.host_bytes}
    return J.value, out, stats


class OutletMomentum(torch.autograd.Function):
    """J = OutletMomentum.apply(phi, channel): differentiable in phi (a float64
    CUDA tensor [ny, nx]); the gradient comes from the library's adjoint."""

    @staticmethod
    def forward(ctx, phi, ch: Channel):
        J, g, _ = outlet_momentum(phi, ch, grad=True)
        ctx.save_for_backward(g)
        return torch.tensor(J, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return gJ * g, None
