"""The committed oracle golden of the 512 x 512 channel (tests/golden/channel512_oracle.txt,
written by tests/golden/make_channel512.py from the oracle alone): its format, the
seeded sample it holds, and what the scheme fixes about it. The oracle conserves
mass to round-off over the 10 000 steps (S_0 = C_0 = 0, half-way bounce-back), the
flow runs along the forcing (+x), and its pressure stays at kappa rho0 / 3 on average
(the provisional equation of state of Eq. 14 gives p = rho c_s^2 with rho near rho0
= 1; the mean of p over the lattice follows the mean of rho)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))


def _load():
    head, rows = {}, []
    with open(os.path.join(HERE, "golden", "channel512_oracle.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) == 2:
                head[parts[0]] = float(parts[1])
            else:
                rows.append([float(v) for v in parts])
    return head, np.array(rows)


def test_golden_format_and_sample():
    import make_channel512 as g
    head, a = _load()
    assert set(head) == {"sum_uu", "mean_p", "u_max", "mass0", "mass"}
    assert a.shape == (g.SAMPLES, 5)
    xs, ys = g.sample_cells()
    assert np.array_equal(a[:, 0].astype(int), xs) and np.array_equal(a[:, 1].astype(int), ys)
    assert len(set(zip(xs, ys))) == g.SAMPLES


def test_golden_physics():
    head, a = _load()
    # mass conserved to round-off over 10 000 steps of 262 144 cells
    assert abs(head["mass"] - head["mass0"]) <= 1e-12 * head["mass0"]
    ux, uy, p = a[:, 2], a[:, 3], a[:, 4]
    assert np.all(np.isfinite(a))
    assert ux.mean() > 0 and np.abs(ux).max() <= head["u_max"] * (1 + 1e-12)
    assert np.abs(uy).max() < np.abs(ux).max()
    # rho stays close to rho0 = 1 (weakly compressible, Ma ~ 1e-2): p = rho / 3
    assert np.all(np.abs(3 * p - 1) < 1e-3)
    assert abs(3 * head["mean_p"] - 1) < 1e-3
