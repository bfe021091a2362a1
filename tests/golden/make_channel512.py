"""Writes channel512_oracle.txt: the FP64 oracle's velocity and pressure after 10 000
steps of the porous-channel recipe regenerated at 512 x 512 (the reduced-precision
accuracy workload), at 2048 seeded sample cells, with the full-field sums the error
norms need. Calls only oracle/ (and the seeded input generator synth.fields).

Recipe: walls at the bottom and top (half-way bounce-back), periodic in x; body force
F^B = phi (1e-6, 0) (the phi G form of Sec. 3.1); tau = 0.6 (s_nu = 1 / 0.6), s_e =
s_eps = s_q = 1.2, kappa = 0.5, rho0 = 1; void fraction synth.fields.channel_phi(512,
512) (seed 2409); from rest (rho = 1, u = 0; the initial populations of Eq. 6, 14).
Velocity u from Eq. (7), pressure p = rho c_s^2 = rho / 3.

Usage: python tests/golden/make_channel512.py   (about 5 minutes on 8 cores)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N, STEPS, TAU, G = 512, 10000, 0.6, 1e-6
RATES = dict(s_e=1.2, s_eps=1.2, s_q=1.2)
SAMPLES, SAMPLE_SEED = 2048, 2409 + 512
OUT = os.path.join(HERE, "channel512_oracle.txt")


def sample_cells():
    """The seeded sample: (x, y) of SAMPLES distinct cells, uniform over the lattice."""
    rng = np.random.default_rng(SAMPLE_SEED)
    k = np.sort(rng.choice(N * N, size=SAMPLES, replace=False))
    return k % N, k // N


def main():
    import oracle as O
    from synth import fields
    phi = fields.channel_phi(N, N)
    prm = O.Params(nx=N, ny=N, s_nu=1.0 / TAU, **RATES, kappa=0.5, bc_y=1, nthreads=O.max_threads())
    fb = np.stack([phi * G, np.zeros_like(phi)])
    rho, ux, uy = fields.rest_fields(N, N)
    f = O.init(prm, rho, ux, uy, phi, fb)
    mass0 = float(f.sum())
    t0 = time.perf_counter()
    for _ in range(STEPS):
        f = O.step(prm, f, phi, None, fb)
    dt = time.perf_counter() - t0
    m = O.macros(prm, f, phi, fb)
    xs, ys = sample_cells()
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle: porous channel recipe at 512x512, 10000 steps from rest "
                 "(tests/golden/make_channel512.py)\n")
        fh.write(f"# oracle threads {prm.nthreads}, {dt:.1f} s\n")
        fh.write(f"sum_uu {float(np.sum(m['ux'] ** 2 + m['uy'] ** 2)):.17e}\n")
        fh.write(f"mean_p {float(m['p'].mean()):.17e}\n")
        fh.write(f"u_max {float(np.abs(m['ux']).max()):.17e}\n")
        fh.write(f"mass0 {mass0:.17e}\n")
        fh.write(f"mass {float(f.sum()):.17e}\n")
        fh.write("# x y ux uy p\n")
        for x, y in zip(xs, ys):
            fh.write(f"{x} {y} {m['ux'][y, x]:.17e} {m['uy'][y, x]:.17e} {m['p'][y, x]:.17e}\n")
    print(f"wrote {OUT} ({dt:.1f} s)")


if __name__ == "__main__":
    main()
