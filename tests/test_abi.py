"""CPU checks of the boundary: the library builds, loads without a GPU and exports
every entry point that include/lbm_vanse.h declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm_vanse.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_vanse_\w+)\s*\(", src)))


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
    p.tau_nu, p.bc_x = 0.8, capi.LBM_BC_BOUNCEBACK
    assert L.lbm_vanse_create(ctypes.byref(p), None, ctypes.byref(h)) == capi.LBM_ERR_ARG
    assert L.lbm_vanse_step(None, 1) == capi.LBM_ERR_ARG
    L.lbm_vanse_destroy(None)


def test_graft_entry_build_compiles_everything():
    import __graft_entry__ as g
    g.build()
    from paper_2409_02964_gb300 import build
    assert os.path.exists(build.LIB)
