#!/usr/bin/env python3
"""Throughput benchmark of the fused D2Q9 MRTLB-VANSE stream + collide step.

Workload (one GPU): the porous channel, 4096 x 4096 cells, FP32 populations,
half-way bounce-back walls at the bottom and top, periodic in x, body force
F^B = phi (1e-6, 0), tau = 0.6, kappa = 0.5, void fraction a seeded Gaussian
random field (correlation length 32) mapped to [0.35, 1.0] with an embedded
sharp block (1.0 -> 0.4 over two cells). One step = one time step of the whole
lattice. Metric: MLUPS (million lattice-cell updates per second), with the
achieved fraction of the measured HBM bandwidth for the step kernel.

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle on
the host cores instead, on bounded row bands of the same channel.
Multi-GPU runs (torchrun) are independent replicas, one lattice per rank.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MRT-VANSE MLUPS & % HBM roofline; FP16-store vs FP32 at equal MMS L2 error"
WORKLOAD = ("porous channel 4096x4096, D2Q9 MRT-VANSE, bounce-back walls top/bottom, periodic x, "
            "g_x=1e-6, tau=0.6, s_e=s_eps=s_q=1.2, kappa=0.5, GRF void fraction [0.35,1] (l=32, seed 2409) "
            "with a sharp block")
TAU, G = 0.6, 1e-6
# non-shear rates of the channel: all 1.2 (s_e from nu_e = nu/3 would be 1.875 at tau = 0.6,
# which does not stay stable next to the sharp block)
RATES = dict(s_e=1.2, s_eps=1.2, s_q=1.2)
DTYPE = {"fp32": "f32", "fp16": "f32", "bf16": "f32", "fp64": "f64"}
SBYTES = {"fp32": 4, "fp16": 2, "bf16": 2, "fp64": 8}


def _config(n: int, storage: str, gpus: int, dev_base: str = "rest") -> dict:
    """The workload as both arms name it (identical keys and values): the lattice, and
    how the timed steps relate to L2 (inputs larger than L2, no flush needed); the
    FP16 / BF16 deviation base when it is not the rest state."""
    pop_gb = 2 * (11 if dev_base == "momentum" else 9) * n * n * SBYTES[storage] / 1e9
    cfg = {"workload": WORKLOAD, "nx": n, "ny": n, "storage": storage,
           "l2": f"inputs larger than L2: two population buffers of {pop_gb:.2f} GB against the 129 MB L2",
           "parallelism": "replicas" if gpus > 1 else "single"}
    if dev_base != "rest":
        cfg["dev_base"] = dev_base
    return cfg


def _kernel_traffic(cells: int):
    """DRAM bytes per launch of the step kernel from the committed ncu capture (a
    smaller channel, scaled by cells), or None when a source the kernel is built
    from has changed since that capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "vanse_warp_fp32_channel_traffic.json")) as fh:
            rec = json.load(fh)
        h = hashlib.sha256()
        for f in sorted(rec["sources"]):
            with open(os.path.join(ROOT, "paper_2409_02964_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() != rec["source_sha256"]:
            return None
        return round(rec["dram_bytes_per_cell"] * cells)
    except Exception:
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        pass

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            try:
                sm.append(float(r[0]))
                smax = float(r[1])
            except ValueError:
                continue
            for nm, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        loaded = sorted(sm)[len(sm) // 2:] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def build_channel(n: int, storage: str, strip_rows: int = 0, kernel: int = 0, eq_order: int = 3, drag=None,
                  moving_wall=None, solid_block: bool = False, dev_base: str = "rest"):
    """The channel lattice; variants: a drag, App. B (eq_order 2), the top wall moving
    at moving_wall = (u_x, u_y), or the block's interior (inside its two-cell ramp)
    made solid (phi = 0)."""
    import paper_2409_02964_gb300 as P
    from synth import fields
    phi = fields.channel_phi(n, n)
    lat = P.Lattice(n, n, TAU, bc_y="bounceback", storage=storage, strip_rows=strip_rows, kernel=kernel,
                    eq_order=eq_order, dev_base=dev_base, **RATES)
    if drag:
        lat.set_drag(*drag)
    if moving_wall:
        lat.set_moving_wall(*moving_wall)
    if solid_block:
        x0, x1, y0, y1 = (int(round(f * n)) for f in (0.4, 0.6, 0.4, 0.6))
        phi = phi.copy()
        phi[y0 + 2:y1 - 2, x0 + 2:x1 - 2] = 0.0
        lat.set_solid_cells()
    lat.set_void_fraction(phi)
    lat.set_body_force(G, 0.0)
    rho, ux, uy = fields.rest_fields(n, n)
    lat.init_fields(rho, ux, uy)
    return lat, phi


def time_steps(lat, steps: int, warmup: int):
    """Device time of `steps` step kernels on the library's stream (CUDA events)."""
    import torch
    lat.step(warmup)
    lat.sync()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(lat.stream)
    lat.step(steps)
    ev1.record(lat.stream)
    ev1.synchronize()
    lat.sync()
    return ev0.elapsed_time(ev1) / 1e3


def e2e_run(lat, phi: np.ndarray, steps: int, dtype=np.float32):
    """The per-step user sequence through the public API with host buffers: upload
    phi(x, t) from pinned host memory (float32, the precision the FP32/FP16/BF16
    storages compute with phi in), advance one step whose kernel also sums the FP64
    mass and momentum it writes, and copy those sums into pinned host memory
    (lbm_vanse_step_sums). The host reads each step's sums one step later, so the
    upload of step t+1 (copied on the library's own stream) overlaps step t."""
    import torch
    host_phi = torch.from_numpy(np.ascontiguousarray(phi, dtype=dtype)).pin_memory()
    out = torch.zeros((2, 3), dtype=torch.float64).pin_memory()
    ev = [torch.cuda.Event(), torch.cuda.Event()]
    lat.set_void_fraction(host_phi)
    lat.step_sums(out[0])
    torch.cuda.synchronize()
    mass = []
    t0 = time.perf_counter()
    for t in range(steps):
        k = t & 1
        lat.set_void_fraction(host_phi)
        lat.step_sums(out[k])
        ev[k].record(lat.stream)
        if t:
            ev[k ^ 1].synchronize()
            mass.append(float(out[k ^ 1, 0]))
    ev[(steps - 1) & 1].synchronize()
    mass.append(float(out[(steps - 1) & 1, 0]))
    dt = time.perf_counter() - t0
    if not all(np.isfinite(mass)) or max(mass) - min(mass) > 1e-4 * abs(mass[0]):
        raise RuntimeError(f"end-to-end run: implausible mass read-back {mass[:3]} ... {mass[-3:]}")
    return dt, host_phi.numel() * host_phi.element_size(), 3 * 8


BATCH_WORKLOAD = ("512 independent periodic lattices, n uniform over {32,48,...,1024} (seed 2409), "
                  "tau ~ U[0.55,1.5], phi amplitude A ~ U[0.05,0.3], spatiotemporal manufactured solution "
                  "phi = 0.7 + A sin sin cos(2 pi t/T) with T = 1000 (n/64)^2, U0 = 0.01 (64/n), "
                  "s_e = s_eps = s_q = 1.2, FP32, 2000 steps each")


def mms_errors(steps: int = 1000):
    """E_u (Eq. 26) of the 64 x 64 spatiotemporal manufactured solution (A = 0.2,
    T = 1000, U0 = 0.01, tau = 0.8, s_e from nu_e = nu/3, s_eps = s_q = 1.2) after
    `steps` steps, per population storage, with phi and the Eq. (25) force evaluated
    in the kernel (a one-lattice batch): the accuracy side of the FP16-vs-FP32
    comparison."""
    import paper_2409_02964_gb300 as P
    out = {}
    for st in ("fp32", "fp16", "bf16"):
        b = P.Batch([(64, 0.8, 0.2, 1000.0, 0.01)], storage=st, s_e=0.0)
        b.init()
        b.step(steps)
        out[st] = b.relative_error(0)
        b.close()
    return out


def mms_errors_lattice(forms, steps: int = 1000):
    """E_u (Eq. 26) of the same 64 x 64 manufactured solution through the single-lattice
    step (phi(t), phi(t+1) and the Eq. (25) force uploaded every step), for storage
    forms the batch kernel does not take: "fp64" (the discretisation error on this
    path) and the momentum-base forms "fp16_momentum", "bf16_momentum"."""
    import paper_2409_02964_gb300 as P
    from synth import mms
    n, nu = 64, 0.1
    M = mms.Config1(n=n, T=1000.0)
    phis = [M.phi(t) for t in range(steps + 1)]
    forces = [M.force(t, nu) for t in range(steps + 1)]
    out = {}
    for form in forms:
        base = "momentum" if form.endswith("_momentum") else "rest"
        lat = P.Lattice(n, n, 0.8, s_eps=1.2, s_q=1.2, storage=form.split("_")[0], dev_base=base)
        ux0, uy0 = M.velocity(0)
        lat.set_void_fraction(phis[0], phis[1])
        lat.set_body_force(0.0, 0.0, forces[0])
        lat.init_fields(np.ones((n, n)), ux0, uy0)
        for t in range(steps):
            lat.set_void_fraction(phis[t], phis[t + 1])
            lat.set_body_force(0.0, 0.0, forces[t])
            lat.step(1)
        lat.set_void_fraction(phis[steps])
        lat.set_body_force(0.0, 0.0, forces[steps])
        uxr, uyr = M.velocity(steps)
        num, den = lat.velocity_error(uxr, uyr)
        out[form] = float(np.sqrt(num / den))
        lat.close()
    return out


def _channel512_golden():
    """The FP64 oracle's u and p after 10 000 steps of the channel recipe at 512 x 512
    (tests/golden/channel512_oracle.txt, written by tests/golden/make_channel512.py
    from the oracle alone): full-field sums and the values at 2048 seeded cells."""
    path = os.path.join(ROOT, "tests", "golden", "channel512_oracle.txt")
    head, rows = {}, []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) == 2:
                head[parts[0]] = float(parts[1])
            else:
                rows.append([float(v) for v in parts])
    a = np.array(rows)
    return head, a[:, 0].astype(int), a[:, 1].astype(int), a[:, 2], a[:, 3], a[:, 4]


def channel_precision(n: int = 512, steps: int = 10000):
    """The channel recipe regenerated at n x n, `steps` steps from rest per storage,
    against the FP64 oracle's run of the same recipe (a committed golden: its
    velocity and pressure at 2048 seeded cells and its full-field sum of |u|^2).
    E_u: relative L2 velocity error (Eq. 26) over the sampled cells; p_rms_err: RMS
    error of p = rho / 3 there; max_rel_u: largest |u - u_oracle| relative to the
    largest |u_oracle| of the sample."""
    import paper_2409_02964_gb300 as P
    from synth import fields
    head, xs, ys, ux_o, uy_o, p_o = _channel512_golden()
    phi = fields.channel_phi(n, n)
    rho, ux, uy = fields.rest_fields(n, n)
    out = {"workload": f"channel recipe at {n}x{n}, {steps} steps from rest, each storage against the FP64 "
                       f"oracle (golden tests/golden/channel512_oracle.txt: {len(xs)} seeded cells)",
           "u_max_oracle": head["u_max"]}
    den = np.sum(ux_o ** 2 + uy_o ** 2)
    umax = float(np.max(np.sqrt(ux_o ** 2 + uy_o ** 2)))
    for st in ("fp64", "fp32", "fp16", "bf16"):
        lat = P.Lattice(n, n, TAU, bc_y="bounceback", storage=st, **RATES)
        lat.set_void_fraction(phi)
        lat.set_body_force(G, 0.0)
        lat.init_fields(rho, ux, uy)
        lat.step(steps)
        m = {k: v.cpu().numpy()[ys, xs] for k, v in lat.macros().items()}
        lat.close()
        du2 = (m["ux"] - ux_o) ** 2 + (m["uy"] - uy_o) ** 2
        out[st] = {"E_u": float(np.sqrt(np.sum(du2) / den)),
                   "p_rms_err": float(np.sqrt(np.mean((m["p"] - p_o) ** 2))),
                   "max_rel_u": float(np.sqrt(du2.max()) / umax)}
    return out


def batch_lattices(count: int = 512):
    from synth import fields
    return fields.batch_lattices(count)


def batch_run(steps: int = 2000, count: int = 512, each_steps: int = 200):
    """The batched workload from t = 0: all `steps` steps as one persistent kernel
    per step in captured CUDA graphs (autotuned unit height); then, for comparison,
    `each_steps` steps with one launch per lattice per step (each lattice cut as a
    lone lattice would be), whose rate is steady from step to step. Device time with
    CUDA events on the library's stream."""
    import torch
    import paper_2409_02964_gb300 as P
    lats = batch_lattices(count)
    b = P.Batch(lats, storage="fp32")
    rows = b.autotune(trial_steps=8)
    stream = b.stream
    res = {}
    errs = None
    for mode in ("persistent", "per_lattice"):
        b.init()
        run = b.step if mode == "persistent" else b.step_each
        ns = steps if mode == "persistent" else min(each_steps, steps)
        run(16 if mode == "persistent" else 3)
        b.init()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        run(ns)
        ev1.record(stream)
        ev1.synchronize()
        secs = ev0.elapsed_time(ev1) / 1e3
        res[mode] = {"steps": ns, "seconds": round(secs, 4),
                     "solves_per_s": round(count * ns / steps / secs, 2),
                     "MLUPS": round(b.cells * ns / secs / 1e6, 1),
                     "GB_s": round(72 * b.cells * ns / secs / 1e9, 1),
                     "gpu_launches": ns * (3 if mode == "persistent" else count + 2)}
        if mode == "persistent":
            errs = np.array([b.relative_error(i) for i in range(count)])
    out = {"workload": BATCH_WORKLOAD, "lattices": count, "cells": b.cells, "steps": steps,
           "unit_rows": rows, "bytes_per_cell": 72, **res,
           "speedup": round(res["persistent"]["MLUPS"] / res["per_lattice"]["MLUPS"], 3),
           "E_u": {"median": float(np.median(errs)), "max": float(np.max(errs)),
                   "finite": int(np.isfinite(errs).sum())}}
    b.close()
    return out


ADJOINT_WORKLOAD = ("1024x1024 porous channel (the 4096^2 channel recipe regenerated at 1024^2), walls, "
                    "tau=0.6, s_e=s_eps=s_q=1.2, kappa=0.5, g_x=1e-6; J = mean outlet phi rho u_x over the last "
                    "100 of 4000 steps from rest; dJ/dphi for every cell; FP64; checkpoint every 200 steps")


def d3q19_run(n: int = 256, steps: int = 200, warmup: int = 5):
    """The 3-D (D3Q19) form of the scheme on an n^3 porous channel (walls in y,
    periodic x and z, g_x = 1e-6, tau = 0.6, the other rates 1.2 as in the 2-D channel,
    from rest), FP32 storage: MLUPS over
    ``steps`` steps timed with CUDA events on the lattice's stream (populations 2 x
    19 x n^3 x 4 B, larger than L2), algorithmic HBM bytes 19 x 4 x 2 + 4 = 156 per
    cell (populations read and written once, phi read once), and the FP64 rate on a
    smaller lattice."""
    import torch
    import paper_2409_02964_gb300 as P
    from synth.fields3d import channel3d_fields
    phi, g = channel3d_fields(n)
    out = {"workload": f"3-D porous channel {n}^3, D3Q19 MRT-VANSE, bounce-back walls in y, periodic x and z, "
                       "g_x=1e-6, tau=0.6, s_e=s_eps=s_q=s_pi=s_m=1.2, kappa=0.5, GRF void "
                       "fraction [0.35,1] (l=16, seed 2409) with a cube block",
           "kernels_per_step": 3}
    peak, _ = _peaks()
    for storage, size, k in (("fp32", n, steps), ("fp64", n // 2, max(10, steps // 10))):
        ph = phi if size == n else channel3d_fields(size)[0]
        lat = P.Lattice3D(size, size, size, 0.6, s_e=1.2, bc_y="bounceback", storage=storage)
        lat.set_void_fraction(ph)
        lat.set_body_force(g, 0.0, 0.0)
        lat.init_fields(np.ones((size,) * 3), np.zeros((3,) + (size,) * 3))
        lat.step(warmup)
        lat.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        m0, _ = lat.reduce()
        e0.record(lat.stream)
        lat.step(k)
        e1.record(lat.stream)
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        m1, _ = lat.reduce()
        lat.close()
        mlups = size ** 3 * k / sec / 1e6
        bpc = 19 * 2 * (4 if storage == "fp32" else 8) + (4 if storage == "fp32" else 8)
        out[storage] = {"n": size, "steps": k, "MLUPS": round(mlups, 1), "bytes_per_cell": bpc,
                        "GB_s": round(mlups * bpc / 1e3, 1), "hbm_frac": round(mlups * bpc / 1e3 / peak, 4),
                        "mass_drift": (m1 - m0) / m0}
    return out


def adjoint_run(n: int = 1024, nsteps: int = 4000, avg: int = 100, ckpt: int = 200):
    """The differentiation workload: J and dJ/dphi through the C ABI, with the two-level
    host checkpoints (the default: sub-segments of ceil(sqrt(K)) states on the device)
    and with whole segments on the device; forward and backward device time from CUDA
    events inside the call, device and pinned host memory held."""
    import paper_2409_02964_gb300 as P
    from synth import fields
    phi = fields.channel_phi(n, n)
    P.outlet_momentum(phi[:64, :64], P.Channel(nx=64, ny=64, nsteps=4, avg_steps=2, checkpoint_every=2))  # warm-up
    lups = n * n * nsteps
    out = {"workload": ADJOINT_WORKLOAD}
    for name, dense in (("two_level", False), ("dense_segments", True)):
        ch = P.Channel(nx=n, ny=n, nsteps=nsteps, avg_steps=avg, checkpoint_every=ckpt, dense_segments=dense)
        J, g, st = P.outlet_momentum(phi, ch)
        fwd_s, bwd_s = st["forward_ms"] / 1e3, st["backward_ms"] / 1e3
        # FP64 flops per cell: a forward step 598; a backward step with its segment
        # recompute 1614 (ncu instruction counts of the adjoint kernels); the two-level
        # scheme recomputes every step once more (598)
        flops = 598.0 + 1614.0 + (0.0 if dense else 598.0)
        achieved = flops * lups / (fwd_s + bwd_s) / 1e12
        out[name] = {"J": J, "max_abs_grad": float(g.abs().max()),
                     "forward_s": round(fwd_s, 3), "backward_s": round(bwd_s, 3),
                     "forward_MLUPS": round(lups / fwd_s / 1e6, 1),
                     "forward_backward_MLUPS": round(lups / (fwd_s + bwd_s) / 1e6, 1),
                     "device_bytes": st["device_bytes"], "host_bytes": st["host_bytes"],
                     "roofline": {"bound": "alu", "unit": "FP64 TFLOP/s", "achieved": round(achieved, 3),
                                  "peak": 1.25, "frac": round(achieved / 1.25, 3), "flops_per_cell_step": flops,
                                  "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak)"}}
        del g
    out["bit_identical"] = out["two_level"]["J"] == out["dense_segments"]["J"]
    out["dtype"] = "f64"
    return out


def adjoint_fd_check(n: int = 1024, nsteps: int = 4000, avg: int = 100, ckpt: int = 200, cells: int = 64,
                     h: float = 1e-4):
    """Central differences (h = 1e-4) of the device's own J at `cells` seeded cells of
    the full differentiation workload against its dJ/dphi (2 * cells forward runs)."""
    import paper_2409_02964_gb300 as P
    from synth import fields
    phi = fields.channel_phi(n, n)
    ch = P.Channel(nx=n, ny=n, nsteps=nsteps, avg_steps=avg, checkpoint_every=ckpt)
    J, g, _ = P.outlet_momentum(phi, ch)
    g = g.cpu().numpy()
    rng = np.random.default_rng(2409)
    pts = [(int(rng.integers(n)), int(rng.integers(n))) for _ in range(cells)]
    gmax = float(np.abs(g).max())
    worst, rows = 0.0, []
    for y, x in pts:
        pp, pm = phi.copy(), phi.copy()
        pp[y, x] += h
        pm[y, x] -= h
        fd = (P.outlet_momentum(pp, ch, grad=False)[0] - P.outlet_momentum(pm, ch, grad=False)[0]) / (2 * h)
        worst = max(worst, abs(fd - g[y, x]) / gmax)
        rows.append([y, x, fd, float(g[y, x])])
    return {"workload": ADJOINT_WORKLOAD, "cells": cells, "h": h, "J": J, "max_abs_grad": gmax,
            "largest_difference_over_max_grad": worst, "samples": rows}


def oracle_rate(n_rows: int, nx: int, steps: int, threads: int):
    """FP64 oracle on a band of the channel: returns (MLUPS, seconds, cells)."""
    import oracle as O
    from synth import fields
    phi = fields.channel_phi(nx, n_rows)
    prm = O.Params(nx=nx, ny=n_rows, s_nu=1.0 / TAU, **RATES, kappa=0.5, bc_y=1, nthreads=threads)
    fb = np.stack([phi * G, np.zeros_like(phi)])
    f = O.init(prm, np.ones((n_rows, nx)), np.zeros((n_rows, nx)), np.zeros((n_rows, nx)), phi, fb)
    t0 = time.perf_counter()
    for _ in range(steps):
        f = O.step(prm, f, phi, None, fb)
    dt = time.perf_counter() - t0
    return nx * n_rows * steps / dt / 1e6, dt, nx * n_rows


def cpu_baseline(nx: int, budget_s: float = 15.0):
    import oracle as O
    threads = O.max_threads()
    rate, dt, _ = oracle_rate(64, nx, 1, threads)          # calibration
    rows = min(1024, nx)
    steps = int(max(2, min(500, budget_s * rate * 1e6 / (rows * nx))))
    rate, dt, cells = oracle_rate(rows, nx, steps, threads)
    return {"value": round(rate, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"FP64 oracle, {steps} steps of a {nx}x{rows} band of the channel (same recipe), {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    nx = args.n
    threads = O.max_threads()
    rate, _, _ = oracle_rate(16, nx, 1, threads)
    # each step: one oracle step of a row band sized so warmup + steps stay within ~90 s
    per_step_s = 90.0 / max(1, args.steps + args.warmup)
    rows = int(max(3, min(args.n, per_step_s * rate * 1e6 / nx)))
    from synth import fields
    phi = fields.channel_phi(nx, rows)
    prm = O.Params(nx=nx, ny=rows, s_nu=1.0 / TAU, **RATES, kappa=0.5, bc_y=1, nthreads=threads)
    fb = np.stack([phi * G, np.zeros_like(phi)])
    f = O.init(prm, np.ones((rows, nx)), np.zeros((rows, nx)), np.zeros((rows, nx)), phi, fb)
    for _ in range(args.warmup):
        f = O.step(prm, f, phi, None, fb)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = O.step(prm, f, phi, None, fb)
    dt = time.perf_counter() - t0
    value = nx * rows * args.steps / dt / 1e6
    sample = f"FP64 oracle, each step a {nx}x{rows} row band of the channel"
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args.n, args.storage, args.gpus, args.dev_base),
        "arithmetic": "FP64 oracle on the host cores",
        "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["fp32", "fp16", "bf16", "fp64"], default="fp32")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--strip-rows", type=int, default=0)
    ap.add_argument("--kernel", type=int, default=0, help="step-kernel variant (0 = the library's choice)")
    ap.add_argument("--dev-base", choices=["rest", "momentum"], default="rest",
                    help="FP16 / BF16 deviation base (momentum: lbm_dev_base LBM_BASE_MOMENTUM)")
    ap.add_argument("--quick", action="store_true", help="timed steps only (no e2e / variants / CPU baseline)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-lattice workload")
    ap.add_argument("--batch-only", action="store_true", help="run only the batched-lattice workload")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the differentiation workload")
    ap.add_argument("--adjoint-only", action="store_true", help="run only the differentiation workload")
    ap.add_argument("--adjoint-n", type=int, default=1024)
    ap.add_argument("--adjoint-steps", type=int, default=4000)
    ap.add_argument("--adjoint-fd", action="store_true",
                    help="central differences at 64 seeded cells of the differentiation workload (slow)")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=2000)
    ap.add_argument("--no-3d", action="store_true", help="skip the 3-D (D3Q19) workload")
    ap.add_argument("--d3q19-only", action="store_true", help="run only the 3-D (D3Q19) workload")
    ap.add_argument("--d3q19-n", type=int, default=256, help="edge of the 3-D channel")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.adjoint_fd:
        print(json.dumps({"adjoint_fd": adjoint_fd_check(args.adjoint_n, args.adjoint_steps)}), flush=True)
        return 0
    if args.adjoint_only:
        print(json.dumps({"adjoint": adjoint_run(args.adjoint_n, args.adjoint_steps, min(100, args.adjoint_steps),
                                                  min(200, args.adjoint_steps))}), flush=True)
        return 0
    if args.batch_only:
        print(json.dumps({"batch": batch_run(args.batch_steps, args.batch_count)}), flush=True)
        return 0
    if args.d3q19_only:
        print(json.dumps({"d3q19": d3q19_run(args.d3q19_n)}), flush=True)
        return 0

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    lat, phi = build_channel(args.n, args.storage, args.strip_rows, args.kernel, dev_base=args.dev_base)
    cells = args.n * args.n
    m0 = lat.reduce()[0]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local).__enter__() if rank == 0 else None
    secs = time_steps(lat, args.steps, args.warmup)
    clocks = sampler.stop() if sampler else None
    m1 = lat.reduce()[0]
    from paper_2409_02964_gb300.replicas import job_throughput
    value, secs, _ = job_throughput(secs, cells * args.steps / 1e6, device=torch.device("cuda", local))
    if dist:
        dist.barrier()
    bpc = lat.bytes_per_cell
    step_s = secs / args.steps
    achieved = bpc * cells / step_s / 1e9
    peak, peak_kind = _peaks()
    shape = lat.launch_shape()

    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.storage], "data": "synthetic",
            "config": _config(args.n, args.storage, world, args.dev_base),
            "bytes_per_cell": bpc, "launch": shape,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         "traffic": _kernel_traffic(cells) if (args.storage == "fp32" and shape["threads"] == 32) else None,
                         "traffic_unit": "bytes per launch",
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "kernel": {32: "vanse_warp_kernel"}.get(shape["threads"], "vanse_step_kernel / vanse_pair_kernel")},
            # the one-warp step kernel is followed by the ghost-column refresh
            "gpu_launches": args.steps * (2 if shape["threads"] == 32 else 1),
            "clocks": clocks,
            "mass_drift": (m1 - m0) / m0,
        }
    if not args.quick and rank == 0:
        e2e_steps = 30
        e2e_dtype = np.float64 if args.storage == "fp64" else np.float32
        dt, h2d, d2h = e2e_run(lat, phi, e2e_steps, e2e_dtype)
        out["e2e"] = {"value": round(world * cells * e2e_steps / dt / 1e6, 1), "unit": "MLUPS",
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "sequence": f"set_void_fraction(pinned host phi, {np.dtype(e2e_dtype).name}) + "
                                  "step_sums(pinned host out) per step (one step that also sums its FP64 mass "
                                  "and momentum); each step's sums read on the host one step later"}
    lat.close()
    if not args.quick and rank == 0:
        variants = {}
        for st in ("fp16", "bf16", "fp64", "fp16_momentum", "bf16_momentum"):
            if st == args.storage:
                continue
            lv, _ = build_channel(args.n, st.split("_")[0], dev_base="momentum" if st.endswith("_momentum") else "rest")
            ns = 2000 if st != "fp64" else 200
            s = time_steps(lv, ns, 5)
            variants[st] = {"MLUPS": round(cells * ns / s / 1e6, 1),
                            "GB_s": round(lv.bytes_per_cell * cells * ns / s / 1e9, 1),
                            "bytes_per_cell": lv.bytes_per_cell, "steps": ns}
            lv.close()
        # physics variants on the same channel, all on the one-warp kernel: a Darcy drag
        # (Sec. 3.1, Da = k0 / H^2 = 1e-2) and the moving top wall (Sec. 3.1) take its
        # general row path on every row / the rows next to the wall, App. B its
        # branch-free path, solid cells (the block's interior, Sec. 3.3) the general
        # path with the neighbour-by-neighbour stencil next to the solid
        nu = (TAU - 0.5) / 3
        for name, kw in (("fp32_darcy_drag", dict(drag=(nu / (1e-2 * args.n * args.n), 0.0, 0.0, 0.0))),
                         ("fp32_appB_eq2", dict(eq_order=2)),
                         ("fp32_moving_wall", dict(moving_wall=(0.01, 0.0))),
                         ("fp32_solid_block", dict(solid_block=True))):
            lv, _ = build_channel(args.n, "fp32", **kw)
            s = time_steps(lv, 1000, 5)
            mlups = cells * 1000 / s / 1e6
            variants[name] = {"MLUPS": round(mlups, 1), "steps": 1000, "kernel": lv.launch_shape()["threads"],
                              "of_plain_fp32": round(mlups * world / value, 3) if args.storage == "fp32" else None}
            lv.close()
        out["precision_channel_512"] = channel_precision()
        errs = mms_errors()
        errs.update(mms_errors_lattice(("fp16_momentum", "bf16_momentum")))
        for st, e in errs.items():
            variants.setdefault(st, {})["mms64_E_u"] = e
        # the discretisation error on the per-step-upload path (equals the batch's FP32 value)
        variants["fp64"]["mms64_E_u"] = mms_errors_lattice(("fp64",))["fp64"]
        out["variants"] = variants
        if not args.no_batch:
            out["batch"] = batch_run(args.batch_steps, args.batch_count)
        if not args.no_adjoint:
            out["adjoint"] = adjoint_run()
        if not args.no_3d:
            out["d3q19"] = d3q19_run(args.d3q19_n)
        out["cpu_baseline"] = cpu_baseline(args.n)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
