"""The allocation-free reduction entry point, lbm_vanse_reduce_noalloc.

Some callers cannot let a library allocate device memory while they run (a loop
whose memory is planned once, an application whose own allocator owns the GPU, code
that must not synchronise the device as cudaMalloc/cudaFree may). For them the
library offers a reduction whose scratch is one fixed device array inside the
library. These tests call it through the C ABI and compare it with the ordinary
lbm_vanse_reduce, which allocates its scratch at creation.

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_02964_gb300 as pkg
    pkg.capi.load()
    return pkg


def _channel(P, nx, ny, storage, solid_block=False):
    from synth import fields
    phi = fields.channel_phi(nx, ny)
    kw = {}
    if solid_block:
        # an impermeable block (phi = 0 cells, Sec. 3.3) and a few isolated solid cells;
        # solid cells run on step kernel 1
        phi[ny // 3:ny // 2, nx // 4:nx // 3] = 0.0
        phi[5, 7] = phi[ny - 3, nx - 2] = 0.0
        kw = dict(kernel=1)
    lat = P.Lattice(nx, ny, 0.6, s_e=1.2, s_eps=1.2, s_q=1.2, bc_y="bounceback", storage=storage, **kw)
    if solid_block:
        lat.set_solid_cells()
    lat.set_void_fraction(phi)
    lat.set_body_force(1e-5, 0.0)
    rho, ux, uy = fields.rest_fields(nx, ny)
    lat.init_fields(rho, ux, uy)
    return lat


@pytest.mark.parametrize("storage,solid_block", [("fp64", False), ("fp32", False), ("fp16", False),
                                                 ("bf16", False), ("fp64", True), ("fp32", True)])
def test_noalloc_reduce_matches_reduce_on_consecutive_calls(P, storage, solid_block):
    """Every storage decodes its populations in the reduction (FP16/BF16 hold scaled
    deviations from the rest state); solid cells hold no populations and are skipped."""
    import torch
    L = P.capi.load()
    lat = _channel(P, 300, 173, storage, solid_block)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        lat.step(7)
        st = L.lbm_vanse_reduce_noalloc(lat._h, ctypes.c_void_p(out.data_ptr()))
        assert st == P.capi.LBM_OK, L.lbm_vanse_last_error(lat._h)
        lat.sync()
        got = out.cpu().numpy()
        ref = np.array(lat.reduce())
        # same FP64 sums in a different order: agree to FP64 rounding
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref).max()), (call, got, ref)
    # a second call right after the first gives the same sums again
    st = L.lbm_vanse_reduce_noalloc(lat._h, ctypes.c_void_p(out.data_ptr()))
    assert st == P.capi.LBM_OK
    lat.sync()
    again = out.cpu().numpy()
    assert np.array_equal(again, got)
    lat.close()


def test_noalloc_reduce_rejects_lattices_taller_than_its_scratch(P):
    import torch
    L = P.capi.load()
    lat = _channel(P, 2, P.capi.NOALLOC_MAX_ROWS + 1, "fp32")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    st = L.lbm_vanse_reduce_noalloc(lat._h, ctypes.c_void_p(out.data_ptr()))
    assert st == P.capi.LBM_ERR_ARG
    assert b"exceeds" in L.lbm_vanse_last_error(lat._h)
    assert L.lbm_vanse_reduce_noalloc(lat._h, None) == P.capi.LBM_ERR_ARG
    lat.close()
