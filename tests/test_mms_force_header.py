"""The closed-form Eq. (25) force compiled into the batch kernel (csrc/mms_force.cuh,
generated symbolically) against the same force evaluated independently with
Taylor jets (synth.mms), in FP64: the header text is translated to Python and
evaluated on whole lattices. A wrong sign, term or factor in the generated code
fails at ~1e-2 relative; the pass bound is 1e-11 (FP64 rounding)."""
import math
import os
import re

import numpy as np
import pytest

from synth import mms

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_2409_02964_gb300", "csrc", "mms_force.cuh")


def _compile_header():
    text = open(HEADER).read()
    body = text[text.index("{", text.index("mms_force(")) + 1:text.rindex("}", 0, text.rindex("}"))]
    lines = []
    for raw in body.strip().splitlines():
        line = raw.strip().rstrip(";")
        line = re.sub(r"^const (float|T) ", "", line)
        line = re.sub(r"(\d+\.\d*(?:e[-+]?\d+)?)f\b", r"\1", line)
        line = line.replace("mms_rcp(", "1.0/(")
        lines.append(line)
    src = "def f(sx, cx, sy, cy, ct, st, k, w, A, U0, phi0, nu):\n" + "\n".join(
        "    " + ln for ln in lines) + "\n    return fx, fy\n"
    ns = {}
    exec(compile(src, HEADER, "exec"), ns)
    return ns["f"]


@pytest.mark.parametrize("n,T,A,U0,tau,t", [
    (64, 1000.0, 0.2, 0.01, 0.8, 0.0),
    (64, 1000.0, 0.2, 0.01, 0.8, 137.0),
    (48, 700.0, 0.05, 0.02, 0.55, 411.0),
    (96, 2250.0, 0.3, 0.0, 1.5, 1900.0),
])
def test_generated_force_matches_jets(n, T, A, U0, tau, t):
    f = _compile_header()
    cfg = mms.Config1(n=n, T=T, A=A, U0=U0)
    nu = (tau - 0.5) / 3.0
    k, w = 2 * math.pi / n, 2 * math.pi / T
    yy, xx = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    fx, fy = f(np.sin(k * xx), np.cos(k * xx), np.sin(k * yy), np.cos(k * yy), math.cos(w * t), math.sin(w * t),
               k, w, A, U0, cfg.phi0, nu)
    ref = cfg.force(t, nu, rho0=1.0)
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(fx - ref[0]).max() <= 1e-11 * scale
    assert np.abs(fy - ref[1]).max() <= 1e-11 * scale


def test_generated_force_detects_a_changed_viscosity():
    """The comparison is sensitive: a 1% change of nu is seen."""
    f = _compile_header()
    n, T, A, U0, t = 64, 1000.0, 0.2, 0.01, 250.0
    cfg = mms.Config1(n=n, T=T, A=A, U0=U0)
    k, w = 2 * math.pi / n, 2 * math.pi / T
    yy, xx = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    fx, _ = f(np.sin(k * xx), np.cos(k * xx), np.sin(k * yy), np.cos(k * yy), math.cos(w * t), math.sin(w * t),
              k, w, A, U0, cfg.phi0, 0.1 * 1.01)
    ref = cfg.force(t, 0.1, rho0=1.0)
    assert np.abs(fx - ref[0]).max() > 1e-5 * np.abs(ref).max()
