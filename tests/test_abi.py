"""CPU checks of the boundary: the library builds, loads without a GPU and exports
every entry point that include/lbm_vanse.h and include/lbm_vanse3d.h declare."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_vanse(?:3d)?_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lbm_vanse_create", "lbm_vanse_init_fields", "lbm_vanse_set_void_fraction",
                     "lbm_vanse_step", "lbm_vanse_macros", "lbm_vanse_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2409_02964_gb300 import build, capi
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(capi.EXPORTS) == _declared()


def test_default_params_and_create_errors_without_gpu():
    from paper_2409_02964_gb300 import capi
    L = capi.load()
    p = capi.default_params()
    assert (p.tau_nu, p.s_eps, p.s_q, p.s_c, p.kappa, p.rho0) == (0.8, 1.2, 1.4, 1.0, 0.5, 1.0)
    # argument checks happen before any CUDA call
    h = ctypes.c_void_p()
    p.nx, p.ny = 0, 4
    assert L.lbm_vanse_create(ctypes.byref(p), None, ctypes.byref(h)) == capi.LBM_ERR_ARG
    assert b"nx" in L.lbm_vanse_last_error(None)
    p.nx, p.ny, p.tau_nu = 4, 4, 0.5
    assert L.lbm_vanse_create(ctypes.byref(p), None, ctypes.byref(h)) == capi.LBM_ERR_ARG
    p.tau_nu, p.bc_x, p.kernel = 0.8, capi.LBM_BC_BOUNCEBACK, 5      # x walls run on kernel 1 only
    assert L.lbm_vanse_create(ctypes.byref(p), None, ctypes.byref(h)) == capi.LBM_ERR_ARG
    p.bc_x, p.kernel = 7, 0
    assert L.lbm_vanse_create(ctypes.byref(p), None, ctypes.byref(h)) == capi.LBM_ERR_ARG
    p.bc_x = capi.LBM_BC_PERIODIC
    assert L.lbm_vanse_step(None, 1) == capi.LBM_ERR_ARG
    L.lbm_vanse_destroy(None)


def test_3d_create_checks_arguments_without_gpu():
    from paper_2409_02964_gb300 import capi
    L = capi.load()
    p = capi.default_params3d()
    assert (p.tau_nu, p.s_e, p.s_eps, p.s_q, p.s_pi, p.s_m, p.kappa, p.rho0, p.storage) == \
        (0.8, 0.0, 1.2, 1.2, 1.2, 1.2, 0.5, 1.0, capi.LBM_FP32)
    h = ctypes.c_void_p()
    assert L.lbm_vanse3d_create(ctypes.byref(p), None, ctypes.byref(h)) == capi.LBM_ERR_ARG   # nx = 0
    assert b"size" in L.lbm_vanse3d_last_error(None)
    p.nx = p.ny = p.nz = 4
    p.storage = capi.LBM_FP16
    assert L.lbm_vanse3d_create(ctypes.byref(p), None, ctypes.byref(h)) == capi.LBM_ERR_ARG
    p.storage, p.s_q = capi.LBM_FP32, 2.5
    assert L.lbm_vanse3d_create(ctypes.byref(p), None, ctypes.byref(h)) == capi.LBM_ERR_ARG
    assert L.lbm_vanse3d_step(None, 1) == capi.LBM_ERR_ARG
    L.lbm_vanse3d_destroy(None)


def test_graft_entry_build_compiles_everything():
    import __graft_entry__ as g
    g.build()
    from paper_2409_02964_gb300 import build
    assert os.path.exists(build.LIB)
