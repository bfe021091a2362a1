"""The CUDA discrete adjoint (lbm_vanse_outlet_momentum_grad, FP64) against the
autograd adjoint oracle (oracle/adjoint.py), against central finite differences of
its own objective, and against the library's FP64 forward step.

Tolerances: J is a sum of j_x + F_x/2, a difference of O(0.1) populations of size
O(1e-4): FP64 rounding alone moves it by ~1e-12 of itself, so J is compared at
1e-10 relative. The gradient carries the same cancellation through the backward
pass; it is compared at 1e-8 of its largest entry. Finite differences use h = 1e-4
(truncation ~h^2, rounding ~1e-16 |J| / h) at 1e-5 of the largest entry.
"""
import numpy as np
import pytest

from synth import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_02964_gb300 as pkg
    pkg.capi.load()
    return pkg


def _phi(nx, ny, seed):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return 0.6 + 0.2 * np.sin(2 * np.pi * x / nx + 0.3) * np.cos(2 * np.pi * y / ny) + 0.05 * rng.uniform(-1, 1, (ny, nx))


def _oracle(ch, phi, segment=0):
    from oracle import adjoint as A
    nu = (ch.tau - 0.5) / 3.0
    pb = A.Problem(nx=ch.nx, ny=ch.ny, s_nu=1.0 / ch.tau, s_e=ch.s_e if ch.s_e > 0 else 1.0 / (nu + 0.5),
                   s_eps=ch.s_eps, s_q=ch.s_q, kappa=ch.kappa, wall_y=ch.bc_y == "bounceback", model_b=ch.model_b,
                   gx=ch.gx, gy=ch.gy)
    x_out = ch.x_out if ch.x_out >= 0 else ch.nx - 1
    return A.objective(phi, pb, ch.nsteps, ch.avg_steps, x_out=x_out, segment=segment)


@pytest.mark.parametrize("bc_y,model_b,s_e", [("bounceback", False, 1.2), ("periodic", False, 0.0),
                                              ("bounceback", True, 1.1), ("periodic", True, 1.3)])
def test_gradient_matches_autograd_oracle(P, bc_y, model_b, s_e):
    ch = P.Channel(nx=23, ny=14, tau=0.7, s_e=s_e, s_q=1.3, bc_y=bc_y, model_b=model_b, gx=2e-5, gy=-5e-6,
                   nsteps=30, avg_steps=8, checkpoint_every=7, x_out=17)
    phi = _phi(ch.nx, ch.ny, 1)
    J, g, _ = P.outlet_momentum(phi, ch)
    Jo, go = _oracle(ch, phi)
    assert abs(J - Jo) <= 1e-10 * abs(Jo)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-8 * np.abs(go).max()


def test_channel_crop_128_matches_autograd_oracle(P):
    """The differentiation workload's channel recipe regenerated at 128 x 128 (a GRF
    void fraction in [0.35, 1] with the sharp block), walls, tau = 0.6."""
    ch = P.Channel(nx=128, ny=128, nsteps=120, avg_steps=40, checkpoint_every=50)
    phi = fields.channel_phi(128, 128)
    J, g, st = P.outlet_momentum(phi, ch)
    Jo, go = _oracle(ch, phi, segment=40)
    assert abs(J - Jo) <= 1e-10 * abs(Jo)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-8 * np.abs(go).max()
    assert st["device_bytes"] > 0 and st["backward_ms"] > 0


def test_checkpoint_spacing_does_not_change_the_result(P):
    """Any checkpoint spacing, with the two-level host checkpoints (sub-segments of
    ceil(sqrt(K)) states on the device) or with whole segments on the device: the
    recomputed states are the same kernels' results, so J and dJ/dphi are
    bit-identical."""
    base = dict(nx=31, ny=17, nsteps=25, avg_steps=6)
    phi = _phi(31, 17, 2)
    outs = []
    for K in (1, 4, 7, 25, 100):
        for dense in (False, True):
            J, g, st = P.outlet_momentum(phi, P.Channel(**base, checkpoint_every=K, dense_segments=dense))
            outs.append((J, g.cpu().numpy()))
            assert (st["host_bytes"] == 0) == dense
    for J, g in outs[1:]:
        assert J == outs[0][0]
        assert np.array_equal(g, outs[0][1])


def test_gradient_matches_central_differences(P):
    ch = P.Channel(nx=64, ny=48, tau=0.6, nsteps=200, avg_steps=50, checkpoint_every=40, gx=1e-5)
    phi = fields.channel_phi(64, 48)
    J, g, _ = P.outlet_momentum(phi, ch)
    g = g.cpu().numpy()
    rng = np.random.default_rng(2409)
    cells = [(int(rng.integers(48)), int(rng.integers(64))) for _ in range(12)] + [(0, 63), (47, 63), (24, 62), (1, 0)]
    h = 1e-4
    for y, x in cells:
        pp, pm = phi.copy(), phi.copy()
        pp[y, x] += h
        pm[y, x] -= h
        Jp, _, _ = P.outlet_momentum(pp, ch, grad=False)
        Jm, _, _ = P.outlet_momentum(pm, ch, grad=False)
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - g[y, x]) <= 1e-5 * np.abs(g).max(), (y, x, fd, g[y, x])


def test_objective_matches_library_fp64_forward(P):
    """J from the adjoint's own dense forward against the library's FP64 step."""
    nx, ny, T, M = 40, 22, 30, 10
    phi = _phi(nx, ny, 3)
    ch = P.Channel(nx=nx, ny=ny, tau=0.8, s_e=0.0, s_q=1.4, nsteps=T, avg_steps=M, checkpoint_every=8, gx=3e-5,
                   gy=1e-5)
    J, _, _ = P.outlet_momentum(phi, ch, grad=False)
    lat = P.Lattice(nx, ny, 0.8, s_e=0.0, s_eps=1.2, s_q=1.4, bc_y="bounceback", storage="fp64")
    lat.set_void_fraction(phi)
    lat.set_body_force(3e-5, 1e-5)
    lat.init_fields(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    acc = 0.0
    for n in range(T):
        lat.step(1)
        if n + 1 > T - M:
            m = {k: v.cpu().numpy() for k, v in lat.macros().items()}
            acc += np.sum((phi * m["rho"] * m["ux"])[:, -1])
    lat.close()
    assert abs(J - acc / (M * ny)) <= 1e-10 * abs(J)


def test_autograd_function(P):
    import torch
    ch = P.Channel(nx=20, ny=12, nsteps=15, avg_steps=5, checkpoint_every=4, gx=1e-5)
    phi = torch.tensor(_phi(20, 12, 4), dtype=torch.float64, device="cuda", requires_grad=True)
    J = P.OutletMomentum.apply(phi, ch)
    (gphi,) = torch.autograd.grad(3.0 * J, phi)
    _, g, _ = P.outlet_momentum(phi.detach(), ch)
    assert torch.allclose(gphi, 3.0 * g, rtol=0, atol=0)


def test_adjoint_argument_errors(P):
    phi = _phi(10, 8, 5)
    for kw in (dict(nsteps=0), dict(avg_steps=0), dict(avg_steps=20, nsteps=10), dict(checkpoint_every=0),
               dict(x_out=10), dict(tau=0.5)):
        base = dict(nx=10, ny=8, nsteps=10, avg_steps=3, checkpoint_every=4)
        base.update(kw)
        with pytest.raises(P.LbmError):
            P.outlet_momentum(phi, P.Channel(**base))
    with pytest.raises(ValueError):
        P.outlet_momentum(phi[:, :9], P.Channel(nx=10, ny=8, nsteps=10, avg_steps=3))


def test_full_size_workload_central_differences(P):
    """The differentiation workload at full size (1024 x 1024 channel recipe, 4000
    steps, J over the last 100, a checkpoint every 200): dJ/dphi against central
    differences of the device's own J (h = 1e-4) at three cells: the largest
    |dJ/dphi|, a cell of the outlet column and a seeded interior cell."""
    n = 1024
    ch = P.Channel(nx=n, ny=n, nsteps=4000, avg_steps=100, checkpoint_every=200)
    phi = fields.channel_phi(n, n)
    J, g, st = P.outlet_momentum(phi, ch)
    g = g.cpu().numpy()
    # two-level checkpoints: 15-state sub-segments on the device (under 2 GB), the 20
    # checkpoints and 14 sub-checkpoints on the host; whole segments on the device
    # (17 GB) give the same bits
    print(f"device {st['device_bytes'] / 1e9:.2f} GB, host {st['host_bytes'] / 1e9:.2f} GB, "
          f"forward {st['forward_ms']:.0f} ms, backward {st['backward_ms']:.0f} ms")
    assert st["device_bytes"] <= 2e9
    Jd, gd, std = P.outlet_momentum(phi, P.Channel(nx=n, ny=n, nsteps=4000, avg_steps=100, checkpoint_every=200,
                                                   dense_segments=True))
    assert Jd == J and np.array_equal(gd.cpu().numpy(), g)
    assert std["device_bytes"] > 10e9 and std["host_bytes"] == 0
    rng = np.random.default_rng(2409)
    cells = [tuple(int(v) for v in np.unravel_index(np.argmax(np.abs(g)), g.shape)), (n // 2, n - 1),
             (int(rng.integers(n)), int(rng.integers(n)))]
    h = 1e-4
    for y, x in cells:
        pp, pm = phi.copy(), phi.copy()
        pp[y, x] += h
        pm[y, x] -= h
        fd = (P.outlet_momentum(pp, ch, grad=False)[0] - P.outlet_momentum(pm, ch, grad=False)[0]) / (2 * h)
        assert abs(fd - g[y, x]) <= 1e-4 * np.abs(g).max(), (y, x, fd, g[y, x])
