"""Compile the CUDA library ``liblbm_vanse.so`` for sm_103a, in-tree.

One translation unit (``csrc/lbm_vanse.cu``) holds the C ABI of
``include/lbm_vanse.h`` and every kernel; it is built with nvcc for
``arch=compute_103a,code=sm_103a`` into ``paper_2409_02964_gb300/_build/``.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm_vanse.so")
SOURCES = ["lbm_vanse.cu"]
HEADERS = ["vanse_common.cuh", "vanse_step.cuh", "vanse_aux.cuh", "vanse_pair.cuh", "vanse_warp.cuh",
           "vanse_batch.cuh", "mms_force.cuh", "vanse_adjoint.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm_vanse.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "lbm_vanse.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None, out: str | None = None) -> str:
    """Build (if stale) and return the path of liblbm_vanse.so.

    extra_flags: additional nvcc flags (e.g. -D tuning knobs; also read from the
    LBM_VANSE_NVCC_FLAGS environment variable); out: alternative output path."""
    lib = out or LIB
    flags = list(extra_flags or []) + os.environ.get("LBM_VANSE_NVCC_FLAGS", "").split()
    if not force and not flags and out is None and not _stale():
        return LIB
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    tmp = lib + ".tmp"
    cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           f"-I{INCLUDE}", "-o", tmp] + flags + [os.path.join(CSRC, s) for s in SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed ({' '.join(cmd)}):\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(r.stderr)
    return lib


if __name__ == "__main__":  # pragma: no cover
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
