"""Failure paths of the single-lattice C ABI, made on the host or by a bounded wait
that runs out (no GPU fault is provoked):

* void-fraction validation: phi divides in Eq. (7) and sets X = kappa / phi in
  Eq. (20) (Sec. 2.3), so NaN, negative or > 1 values are rejected with
  LBM_ERR_ARG before they replace the lattice's field, through every upload path
  (pageable host doubles, pinned host floats, device arrays), for phi(t) and for
  phi(t+1); the lattice is left as it was;
* divergence: a NaN population written through set_populations is reported by
  lbm_vanse_reduce as LBM_ERR_DIVERGED after a step;
* the timeout path: with every staged-row wait limited to zero polls
  (lbm_vanse_set_row_wait_limit) each step kernel gives up at once, drains its
  copies and flags the lattice; lbm_vanse_sync returns LBM_ERR_TIMEOUT, and a lattice
  with the default bound then steps cleanly (its result equal to the oracle's).
"""
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


def _lattice(P, nx=70, ny=24, storage="fp32", kernel=0):
    phi = 0.6 + 0.2 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, :] * np.cos(np.pi * np.arange(ny) / ny)[:, None]
    lat = P.Lattice(nx, ny, 0.6, s_e=1.2, s_eps=1.2, s_q=1.2, bc_y="bounceback", storage=storage, kernel=kernel)
    lat.set_void_fraction(phi)
    lat.set_body_force(1e-5, 0.0)
    z = np.zeros((ny, nx))
    lat.init_fields(np.ones((ny, nx)), z, z)
    return lat, phi


def _oracle(nx, ny, phi, steps):
    import oracle as O
    prm = O.Params(nx=nx, ny=ny, s_nu=1 / 0.6, s_e=1.2, s_eps=1.2, s_q=1.2, kappa=0.5, bc_y=1)
    z = np.zeros((ny, nx))
    fb = np.stack([phi * 1e-5, z])
    f = O.init(prm, np.ones((ny, nx)), z, z, phi, fb)
    for _ in range(steps):
        f = O.step(prm, f, phi, None, fb)
    return f


BAD = {"nan": np.nan, "negative": -0.25, "above_one": 1.0 + 1e-6}


@pytest.mark.parametrize("path", ["host_double", "pinned_float", "device"])
@pytest.mark.parametrize("which", ["phi_t", "phi_next"])
@pytest.mark.parametrize("kind", list(BAD))
def test_invalid_void_fraction_is_rejected_and_the_lattice_kept(P, path, which, kind):
    import torch
    nx, ny = 70, 24
    lat, phi = _lattice(P, nx, ny)
    lat.step(3)
    before = lat.get_populations().cpu().numpy()
    bad = phi.copy()
    bad[ny // 2, nx // 3] = BAD[kind]
    good = phi.copy()
    args = (bad, good) if which == "phi_t" else (good, bad)
    if path == "pinned_float":
        args = tuple(torch.from_numpy(a.astype(np.float32)).pin_memory() for a in args)
    elif path == "device":
        args = tuple(torch.from_numpy(a).cuda() for a in args)
    with pytest.raises(P.LbmError) as e:
        lat.set_void_fraction(*args)
    assert e.value.status == P.capi.LBM_ERR_ARG
    assert which in str(e.value) and "unchanged" in str(e.value)
    # nothing changed: the populations, and the steps that follow (steady phi as before)
    assert np.array_equal(lat.get_populations().cpu().numpy(), before)
    lat.step(5)
    lat.sync()
    f = _oracle(nx, ny, phi, 8)
    assert np.abs(lat.get_populations().cpu().numpy() - f).max() <= 8 * 32 * 2.0 ** -24 * np.abs(f).max()
    lat.close()


def test_valid_boundary_values_pass(P):
    nx, ny = 70, 24
    lat, phi = _lattice(P, nx, ny)
    edge = phi.copy()
    edge[3, 5] = 1.0                      # the upper end of (0, 1] is a valid void fraction
    lat.set_void_fraction(edge)
    lat.step(2)
    lat.sync()
    lat.close()


def test_nan_population_reports_divergence(P):
    for storage in ("fp64", "fp32"):
        lat, _ = _lattice(P, storage=storage)
        lat.step(2)
        f = lat.get_populations().cpu().numpy()
        f[4, 10, 20] = np.nan
        lat.set_populations(f)
        lat.step(1)
        lat.sync()
        with pytest.raises(P.LbmError) as e:
            lat.reduce()
        assert e.value.status == P.capi.LBM_ERR_DIVERGED
        lat.close()


@pytest.mark.parametrize("storage,kernel,steps", [("fp32", 5, 3), ("fp32", 5, 70), ("fp16", 5, 3),
                                                  ("fp64", 1, 3), ("fp32", 2, 3)])
def test_row_wait_timeout_is_reported_and_a_fresh_lattice_steps_cleanly(P, storage, kernel, steps):
    """steps = 70 runs through the replayed CUDA graph of 32 steps as well."""
    L = P.capi.load()
    nx, ny = 300, 200
    lat, _ = _lattice(P, nx, ny, storage, kernel)
    assert L.lbm_vanse_set_row_wait_limit(lat._h, 0) == P.capi.LBM_OK
    lat.step(steps)
    st = L.lbm_vanse_sync(lat._h)
    assert st == P.capi.LBM_ERR_TIMEOUT, P.capi.STATUS_NAMES.get(st, st)
    assert b"gave up" in L.lbm_vanse_last_error(lat._h)
    # the flag stays set: the populations of a lattice that timed out are not valid
    assert L.lbm_vanse_set_row_wait_limit(lat._h, -1) == P.capi.LBM_OK
    assert L.lbm_vanse_sync(lat._h) == P.capi.LBM_ERR_TIMEOUT
    lat.close()
    # a new lattice with the default bound steps as before
    nx, ny = 70, 24
    lat, phi = _lattice(P, nx, ny, storage, kernel)
    lat.step(6)
    lat.sync()
    f = _oracle(nx, ny, phi, 6)
    dev = np.abs(f - f.mean(axis=(1, 2), keepdims=True)).max()
    if storage == "fp64":
        tol = 1e-12 * dev
    else:   # the per-step rounding bounds of the parity tests (FP32 compute; FP16's 11-bit stores)
        tol = 6 * 32 * 2.0 ** -24 * np.abs(f).max() + (2 * 6 * 2.0 ** -11 * dev if storage == "fp16" else 0.0)
    assert np.abs(lat.get_populations().cpu().numpy() - f).max() <= tol
    lat.close()


def test_row_wait_limit_argument_checks(P):
    L = P.capi.load()
    assert L.lbm_vanse_set_row_wait_limit(None, 5) == P.capi.LBM_ERR_ARG
