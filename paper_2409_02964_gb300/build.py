"""Compile the CUDA library ``liblbm_vanse.so`` for sm_103a, in-tree.

Two translation units, compiled in parallel and linked into one shared library in
``paper_2409_02964_gb300/_build/`` with nvcc for ``arch=compute_103a,code=sm_103a``:
``csrc/lbm_vanse.cu`` (the C ABI of ``include/lbm_vanse.h`` and the D2Q9 kernels) and
``csrc/lbm_vanse3d.cu`` (``include/lbm_vanse3d.h``, the D3Q19 step).
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
SOURCES = ["lbm_vanse.cu", "vanse_warp_solid.cu", "vanse_warp_jb.cu", "vanse_warp_nee.cu", "lbm_vanse3d.cu"]
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
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, h)
                                                                for h in ("lbm_vanse.h", "lbm_vanse3d.h")]
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
    common = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}"] + flags
    if verbose:
        common.insert(1, "-Xptxas=-v")
    objs, procs = [], []
    for s in SOURCES:
        obj = os.path.join(os.path.dirname(lib), os.path.splitext(s)[0] + ".o")
        cmd = common + ["-c", "-o", obj, os.path.join(CSRC, s)]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
        objs.append(obj)
    logs = []
    for cmd, pr in procs:
        _, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(f"nvcc failed ({' '.join(cmd)}):\n{err}")
        logs.append(err)
    link = [nvcc(), ARCH, "-shared", "-o", tmp] + objs
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed ({' '.join(link)}):\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print("".join(logs))
    return lib


if __name__ == "__main__":  # pragma: no cover
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
