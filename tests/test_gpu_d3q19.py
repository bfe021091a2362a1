"""GPU parity of the 3-D (D3Q19) step against the FP64 oracle, through the C ABI of
include/lbm_vanse3d.h: element by element on small ragged lattices (periodic and
walled, a moving phi and per-cell forces), the macroscopic fields, mass and
momentum balance, the 3-D manufactured solution (same E_u as the oracle), and at
the benchmark's size (256^3) one step on sampled windows recomputed by the oracle."""
import numpy as np
import pytest

from oracle import d3q19 as D
from synth.mms3 import Config3

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_02964_gb300 as pkg
    pkg.capi.load()
    return pkg


def _case(nx, ny, nz, seed, field=True):
    rng = np.random.default_rng(seed)
    shp = (nz, ny, nx)
    phi = rng.uniform(0.45, 1.0, size=shp)
    phin = np.clip(phi + 0.01 * rng.normal(size=shp), 0.4, 1.0)
    rho = 1 + 0.01 * rng.normal(size=shp)
    u = 0.02 * rng.normal(size=(3,) + shp)
    g = (1e-5, -2e-6, 3e-6)
    fb = 1e-5 * rng.normal(size=(3,) + shp) if field else None
    return dict(phi=phi, phin=phin, rho=rho, u=u, g=g, fb=fb)


def _total_force(c):
    F = np.stack([c["phi"] * c["g"][a] for a in range(3)])
    return F + c["fb"] if c["fb"] is not None else F


def _gpu(P, nx, ny, nz, c, storage, walls, tau=0.8):
    lat = P.Lattice3D(nx, ny, nz, tau, bc_y="bounceback" if walls else "periodic", storage=storage)
    lat.set_void_fraction(c["phi"], c["phin"])
    lat.set_body_force(*c["g"], field=c["fb"])
    lat.init_fields(c["rho"], c["u"])
    return lat


def _params(nx, ny, nz, walls, tau=0.8):
    return D.Params(nx, ny, nz, bc_y=int(walls), **D.rates_from_tau(tau))


SHAPES = [(9, 7, 5, False), (13, 6, 4, True), (1, 5, 3, True), (7, 1, 4, False), (17, 11, 3, True)]


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,ny,nz,walls", SHAPES)
def test_populations_match_oracle(P, nx, ny, nz, walls, storage):
    c = _case(nx, ny, nz, seed=nx * 100 + ny * 10 + nz)
    lat = _gpu(P, nx, ny, nz, c, storage, walls)
    p = _params(nx, ny, nz, walls)
    f0 = D.init(p, c["rho"], c["u"], c["phi"], _total_force(c))
    g0 = lat.get_populations().cpu().numpy()
    tol0 = 1e-15 if storage == "fp64" else 3e-7
    assert np.abs(g0 - f0).max() < tol0
    f = D.step(p, f0, c["phi"], c["phin"], _total_force(c))     # first step: phi moves
    c2 = dict(c, phi=c["phin"], phin=None)
    for _ in range(3):
        f = D.step(p, f, c2["phi"], None, _total_force(c2))
    lat.step(4)
    lat.sync()
    g = lat.get_populations().cpu().numpy()
    dev = np.abs(f - f0).max()
    err = np.abs(g - f).max()
    tol = 1e-13 if storage == "fp64" else 4 * 2e-6
    print(f"{storage} {nx}x{ny}x{nz} walls={walls}: max |f_gpu - f_oracle| = {err:.2e} (change {dev:.2e})")
    assert err < tol, (err, tol)
    # the macroscopic fields of Eq. (7)
    mo = D.macros(p, f, c2["phi"], _total_force(c2))
    m = lat.macros()
    tolm = 1e-12 if storage == "fp64" else 2e-5
    assert np.abs(m["rho"].cpu().numpy() - mo["rho"]).max() < tolm
    assert np.abs(m["u"].cpu().numpy() - mo["u"]).max() < tolm
    lat.close()


@pytest.mark.parametrize("walls", [False, True])
def test_mass_and_momentum_balance(P, walls):
    nx, ny, nz = 24, 16, 12
    c = _case(nx, ny, nz, seed=3, field=False)
    c["phin"] = None
    lat = _gpu(P, nx, ny, nz, c, "fp64", walls)
    m0, j0 = lat.reduce()
    lat.step(50)
    m1, j1 = lat.reduce()
    assert abs(m1 - m0) < 1e-13 * m0
    if not walls:
        # with phi steady: sum F^p is not zero for a varying phi, so compare one step's
        # change with the oracle's sum of F
        p = _params(nx, ny, nz, walls)
        f = lat.get_populations().cpu().numpy()
        F = D.macros(p, f, c["phi"], _total_force(c))["F"]
        _, ja = lat.reduce()
        lat.step(1)
        _, jb = lat.reduce()
        assert np.abs(np.array(jb) - np.array(ja) - F.reshape(3, -1).sum(1)).max() < 1e-13
    lat.close()


def _mms_gpu(P, n, T, U0, storage, tau=0.8):
    M = Config3(n=n, T=float(T), U0=U0)
    r = D.rates_from_tau(tau)
    nu, nu_e = (tau - 0.5) / 3, (1 / r["s_e"] - 0.5) / 3
    lat = P.Lattice3D(n, n, n, tau, storage=storage)
    lat.set_void_fraction(M.phi(0), M.phi(1))
    lat.set_body_force(field=M.force(0, nu, nu_e))
    lat.init_fields(np.ones((n, n, n)), M.velocity(0))
    for t in range(T):
        lat.set_void_fraction(M.phi(t), M.phi(t + 1))
        lat.set_body_force(field=M.force(t, nu, nu_e))
        lat.step(1)
    lat.set_void_fraction(M.phi(T))
    lat.set_body_force(field=M.force(T, nu, nu_e))
    u = lat.macros()["u"].cpu().numpy()
    lat.close()
    ur = M.velocity(T)
    return float(np.sqrt(((u - ur) ** 2).sum() / (ur ** 2).sum()))


def test_manufactured_solution_matches_oracle_and_converges(P):
    """E_u of the 3-D manufactured solution: the FP64 device path equals the oracle's
    (1.185e-2 at 12^3, 3.010e-3 at 24^3, measured on the oracle) and the FP32 path
    stays within 1 % of it; the error falls by 4 from 12^3 to 24^3."""
    e12 = _mms_gpu(P, 12, 64, 0.02, "fp64")
    e24 = _mms_gpu(P, 24, 256, 0.01, "fp64")
    e24f = _mms_gpu(P, 24, 256, 0.01, "fp32")
    print(f"E_u fp64 12^3 {e12:.6e}, 24^3 {e24:.6e}; fp32 24^3 {e24f:.6e}")
    assert abs(e12 - 1.185e-2) < 0.01e-2 and abs(e24 - 3.010e-3) < 0.01e-3
    assert abs(e24f - e24) < 0.01 * e24
    assert 3.5 < e12 / e24 < 4.5


def test_full_size_channel_step_on_sampled_windows(P):
    """The benchmark's 256^3 FP32 channel (walls in y, periodic x and z, the non-shear
    rates at 1.2 as in the 2-D channel; s_e derived from nu_e = nu/3 is 1.875 at
    tau = 0.6 and diverges on this channel, in the oracle too): after a few
    steps from rest (200), one more device step against the oracle on three sampled
    windows (full height, 12 x 12 cells in x and z), each recomputed from the device
    state with a 3-cell periodic-wrapped halo (the step's dependency radius)."""
    import torch
    from synth.fields3d import channel3d_fields
    n = 256
    phi, g = channel3d_fields(n)
    lat = P.Lattice3D(n, n, n, 0.6, s_e=1.2, bc_y="bounceback", storage="fp32")
    lat.set_void_fraction(phi)
    lat.set_body_force(g, 0.0, 0.0)
    lat.init_fields(np.ones((n, n, n)), np.zeros((3, n, n, n)))
    lat.step(200)
    f = lat.get_populations()
    lat.step(1)
    f1 = lat.get_populations()
    p = D.Params(18, n, 18, bc_y=1, **dict(D.rates_from_tau(0.6), s_e=1.2))
    rng = np.random.default_rng(1)
    for (x0, z0) in [(0, 0), (n - 12, 120), tuple(rng.integers(0, n - 12, size=2))]:
        xs = [(x0 - 3 + k) % n for k in range(18)]
        zs = [(z0 - 3 + k) % n for k in range(18)]
        ix = torch.tensor(xs, device=f.device)
        iz = torch.tensor(zs, device=f.device)
        win = f.index_select(3, ix).index_select(1, iz).cpu().numpy()
        ph = phi[np.ix_(zs, range(n), xs)]
        fb = np.stack([ph * g, 0 * ph, 0 * ph])
        want = D.step(p, win, ph, None, fb)[:, 3:15, :, 3:15]
        got = f1.index_select(3, ix[3:15]).index_select(1, iz[3:15]).cpu().numpy()
        err = np.abs(got - want).max()
        assert err < 2e-6, (x0, z0, err)
    m0, _ = lat.reduce()
    assert np.isfinite(m0)
    lat.close()


def test_error_paths(P):
    """Invalid calls return an error status and leave the handle usable."""
    from paper_2409_02964_gb300.lattice import LbmError
    n = 4
    lat = P.Lattice3D(n, n, n, storage="fp64")
    with pytest.raises(LbmError, match="STATE"):
        lat.step(1)                                   # before init
    with pytest.raises(LbmError, match="STATE"):
        lat.init_fields(np.ones((n, n, n)), np.zeros((3, n, n, n)))   # before phi
    bad = np.full((n, n, n), 0.8)
    bad[1, 2, 3] = 0.0
    with pytest.raises(LbmError, match="ARG"):
        lat.set_void_fraction(bad)
    bad[1, 2, 3] = 1.5
    with pytest.raises(LbmError, match="ARG"):
        lat.set_void_fraction(bad)
    lat.set_void_fraction(np.full((n, n, n), 0.8))
    lat.init_fields(np.ones((n, n, n)), np.zeros((3, n, n, n)))
    with pytest.raises(LbmError, match="ARG"):
        lat.set_void_fraction(bad)                     # rejected: the lattice keeps phi = 0.8
    with pytest.raises(LbmError, match="ARG"):
        lat.step(-1)
    lat.step(0)
    lat.step(3)
    m, j = lat.reduce()
    assert abs(m - 0.8 * n ** 3) < 1e-12 and max(abs(x) for x in j) < 1e-14
    assert lat.step_count == 3
    lat.close()


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_new_phi_keeps_populations_and_steps_match_oracle(P, storage):
    """The populations are stored as deviations from the rest state of the lattice's
    current phi; a new phi(t) moves f_0's stored deviation so that the populations
    (and the mass) stay those the steps left, as in the oracle, and the following
    steps agree with it."""
    nx, ny, nz = 10, 7, 6
    c = _case(nx, ny, nz, seed=77)
    c["phin"] = None
    lat = _gpu(P, nx, ny, nz, c, storage, True)
    p = _params(nx, ny, nz, True)
    f = D.init(p, c["rho"], c["u"], c["phi"], _total_force(c))
    for _ in range(2):
        f = D.step(p, f, c["phi"], None, _total_force(c))
    lat.step(2)
    before = lat.get_populations().cpu().numpy()
    m0, _ = lat.reduce()
    phi2 = np.clip(c["phi"] + np.random.default_rng(1).uniform(0.0, 0.1, size=c["phi"].shape), 0.3, 1.0)
    lat.set_void_fraction(phi2)
    after = lat.get_populations().cpu().numpy()
    m1, _ = lat.reduce()
    tol = 1e-15 if storage == "fp64" else 1e-7
    assert np.abs(after - before).max() < tol
    assert abs(m1 - m0) < (1e-13 if storage == "fp64" else 1e-5)
    c2 = dict(c, phi=phi2)
    for _ in range(2):
        f = D.step(p, f, phi2, None, _total_force(c2))
    lat.step(2)
    g = lat.get_populations().cpu().numpy()
    lat.close()
    assert np.abs(g - f).max() < (1e-13 if storage == "fp64" else 4e-6)
