"""Checkpoint and resume (lbm_vanse_save_state / lbm_vanse_load_state): a state saved
after some steps, loaded into a fresh lattice of the same shape, continues the run bit
for bit, for every storage (FP16/BF16 with the stochastic rounding seeded by the
restored step counter), with a pending phi(t+1), a force field and a drag; through
host and device buffers; and a state is refused by a lattice of another shape or
storage, and when it is not a state at all."""
import numpy as np
import pytest

from gpu_cases import random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_02964_gb300 as pkg
    pkg.capi.load()
    return pkg


def _lattice(P, nx, ny, storage, case, drag=False):
    lat = P.Lattice(nx, ny, 0.7, s_eps=1.2, s_q=1.4, bc_y="bounceback", storage=storage)
    if drag:
        lat.set_drag(0.02, 0.3, 1e-3, 0.0)
    lat.set_void_fraction(case["phi"])
    lat.set_body_force(case["g"][0], case["g"][1], case["fb"])
    lat.init_fields(case["rho"], case["ux"], case["uy"])
    return lat


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("device_buffer", [False, True])
def test_resume_continues_bit_for_bit(P, storage, device_buffer):
    import torch
    nx, ny = 150, 70
    case = random_case(nx, ny, seed=12, wall_y=True, unsteady=True, field=True, g=(1e-5, 0.0))
    ref = _lattice(P, nx, ny, storage, case, drag=True)
    ref.step(37)
    # a pending phi(t+1): the state must carry it
    ref.set_void_fraction(case["phi"], case["phin"])
    if device_buffer:
        n = int(P.capi.load().lbm_vanse_state_bytes(ref._h))
        state = torch.empty(n, dtype=torch.uint8, device="cuda")
        assert P.capi.load().lbm_vanse_save_state(ref._h, state.data_ptr(), 1) == P.capi.LBM_OK
    else:
        state = ref.save_state()
    ref.step(45)
    want = ref.get_populations().cpu().numpy()
    steps_ref = ref.step_count
    ref.close()
    # a fresh lattice of the same shape with other fields: the state replaces them all
    other = random_case(nx, ny, seed=99, wall_y=True)
    lat = P.Lattice(nx, ny, 0.7, s_eps=1.2, s_q=1.4, bc_y="bounceback", storage=storage)
    lat.set_drag(0.02, 0.3, 1e-3, 0.0)
    lat.set_void_fraction(other["phi"])
    lat.init_fields(other["rho"], other["ux"], other["uy"])
    lat.step(3)
    lat.load_state(state)
    assert lat.step_count == 37
    lat.step(45)
    got = lat.get_populations().cpu().numpy()
    assert lat.step_count == steps_ref
    lat.close()
    assert np.array_equal(got, want)


def test_state_of_another_lattice_is_refused(P):
    case = random_case(40, 20, seed=3, wall_y=True)
    lat = _lattice(P, 40, 20, "fp32", case)
    lat.step(2)
    state = lat.save_state()
    lat.close()
    for nx, ny, storage in ((41, 20, "fp32"), (40, 20, "fp16")):
        c = random_case(nx, ny, seed=4, wall_y=True)
        other = _lattice(P, nx, ny, storage, c)
        with pytest.raises(P.LbmError) as e:
            other.load_state(state)
        assert e.value.status == P.capi.LBM_ERR_ARG
        other.close()
    lat = _lattice(P, 40, 20, "fp32", case)
    with pytest.raises(P.LbmError):
        lat.load_state(np.zeros_like(state))
    lat.close()
    fresh = P.Lattice(40, 20, 0.7)
    assert P.capi.load().lbm_vanse_state_bytes(fresh._h) == -1
    with pytest.raises(P.LbmError):
        fresh.save_state()
    fresh.close()
