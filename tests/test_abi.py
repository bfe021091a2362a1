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


def _header_struct(name):
    """(field, c type) of `typedef struct { ... } name;` in include/*.h, in order."""
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", h)).read(), flags=re.S)
        m = re.search(r"typedef\s+struct\s*\{([^}]*)\}\s*" + name + r"\s*;", src)
        if m:
            out = []
            for decl in m.group(1).split(";"):
                decl = decl.strip()
                if not decl:
                    continue
                m2 = re.match(r"((?:(?:unsigned|long|short)\s+)*\w+)\s+(.*)$", decl, flags=re.S)
                ctype, names = " ".join(m2.group(1).split()), m2.group(2)
                out += [(n.strip(), ctype) for n in names.split(",")]
            return out
    raise AssertionError(f"{name} not found")


def test_ctypes_structs_match_the_header():
    from paper_2409_02964_gb300 import capi
    ct = {ctypes.c_int: "int", ctypes.c_double: "double", ctypes.c_longlong: "long long"}
    for name in ("lbm_vanse_params", "lbm_vanse3d_params", "lbm_vanse_batch_lattice", "lbm_vanse_batch_params",
                 "lbm_vanse_adjoint_params", "lbm_vanse_adjoint_stats"):
        py = [(f, ct[t]) for f, t in getattr(capi, name)._fields_]
        assert py == _header_struct(name), name


def test_momentum_base_checks_without_gpu():
    """lbm_dev_base: checked before any CUDA call, like the other arguments."""
    from paper_2409_02964_gb300 import capi
    L = capi.load()
    h = ctypes.c_void_p()
    p = capi.default_params()
    assert p.dev_base == capi.LBM_BASE_REST
    p.nx, p.ny = 16, 8
    for storage, kernel, bc_x, dev_base, word in (
            (capi.LBM_BF16, 0, capi.LBM_BC_PERIODIC, 7, b"dev_base"),
            (capi.LBM_FP32, 0, capi.LBM_BC_PERIODIC, capi.LBM_BASE_MOMENTUM, b"FP16 / BF16"),
            (capi.LBM_FP64, 0, capi.LBM_BC_PERIODIC, capi.LBM_BASE_MOMENTUM, b"FP16 / BF16"),
            (capi.LBM_BF16, 1, capi.LBM_BC_PERIODIC, capi.LBM_BASE_MOMENTUM, b"kernel 5"),
            (capi.LBM_FP16, 2, capi.LBM_BC_PERIODIC, capi.LBM_BASE_MOMENTUM, b"kernel 5"),
            (capi.LBM_FP16, 0, capi.LBM_BC_BOUNCEBACK, capi.LBM_BASE_MOMENTUM, b"kernel 5")):
        p.storage, p.kernel, p.bc_x, p.dev_base = storage, kernel, bc_x, dev_base
        assert L.lbm_vanse_create(ctypes.byref(p), None, ctypes.byref(h)) == capi.LBM_ERR_ARG
        assert word in L.lbm_vanse_last_error(None), L.lbm_vanse_last_error(None)
