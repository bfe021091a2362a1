"""Stochastic rounding of FP16 / BF16 stores in the one-warp kernel.

A uniform periodic flow (rho = 1, u = (0.02, 0), phi = 0.7 everywhere, so F^p = 0)
driven by a body force F^B = phi g with g = 5e-7: each step the collision adds F^B
to every cell's momentum (Eq. 16 with the Guo source), so the lattice's momentum
grows by exactly T N phi g over T steps, whatever the rounding, provided the
rounding is unbiased. Per step a population changes by about w_i 3 phi g ~ 1e-7,
far below half a unit in the last place of its stored deviation from rest (2e-6 in
FP16 at 2^16 scale, 1.5e-5 in BF16): round-to-nearest would store the old value
every step and the momentum would not move. Rounding up with probability equal to
the discarded fraction keeps the expectation; what is left is the random walk of
the roundings, about sqrt(N T) x (the rounding's spread per cell and step).
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


# random-walk spread of the momentum sum relative to the expected growth, estimated
# from half an ulp per rounding and ~6 populations per cell: 0.2 % (FP16), 0.9 % (BF16)
TOL = {"fp16": 0.01, "bf16": 0.05}


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_forced_uniform_flow_gains_momentum_below_the_rounding_unit(P, storage):
    nx, ny, steps, g, phi = 512, 128, 2000, 5e-7, 0.7
    lat = P.Lattice(nx, ny, 0.8, s_eps=1.2, s_q=1.2, storage=storage, kernel=5)
    lat.set_void_fraction(np.full((ny, nx), phi))
    lat.set_body_force(g, 0.0)
    lat.init_fields(np.ones((ny, nx)), np.full((ny, nx), 0.02), np.zeros((ny, nx)))
    m0, jx0, jy0 = lat.reduce()
    lat.step(steps)
    m1, jx1, jy1 = lat.reduce()
    lat.close()
    want = steps * nx * ny * phi * g
    print(f"{storage}: momentum gain {jx1 - jx0:.6e}, expected {want:.6e}, "
          f"ratio {(jx1 - jx0) / want:.5f}; y drift {jy1 - jy0:.2e}; mass drift {(m1 - m0) / m0:.2e}")
    assert abs((jx1 - jx0) - want) < TOL[storage] * want, (jx1 - jx0, want)
    # no force along y: its momentum stays at zero up to the same random walk
    assert abs(jy1 - jy0) < TOL[storage] * want, (jy0, jy1)
    assert abs(m1 - m0) < TOL[storage] * want, (m0, m1)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_stochastic_rounding_is_reproducible_and_changes_with_the_step(P, storage):
    """The random bits come from the cell, the row and the device's step count (which
    set_populations does not reset). The same state stepped at two successive step
    counts rounds differently in a good share of its values, by one unit of the stored
    deviation at most, so the rounding errors of successive steps do not repeat; a
    second lattice taking the same calls stores the same values bit for bit."""
    nx, ny = 96, 40
    rng = np.random.default_rng(5)
    ux = 0.02 + 0.005 * rng.standard_normal((ny, nx))
    runs = []
    for _ in range(2):
        lat = P.Lattice(nx, ny, 0.8, storage=storage, kernel=5)
        lat.set_void_fraction(np.full((ny, nx), 0.7))
        lat.set_body_force(5e-7, 0.0)
        lat.init_fields(np.ones((ny, nx)), ux, np.zeros((ny, nx)))
        f_init = lat.get_populations().cpu().numpy()
        out = []
        for _ in range(2):
            lat.set_populations(f_init)
            lat.step(1)
            out.append(lat.get_populations().cpu().numpy())
        lat.close()
        runs.append(out)
    a, b = runs[0]
    assert np.array_equal(a, runs[1][0]) and np.array_equal(b, runs[1][1])
    differ = a != b
    # one unit in the last place of a stored deviation |f - f_rest| < 0.05: 2^-10 x 0.05
    # with FP16's 11 significant bits (its 2^16 scale cancels), 2^-7 x 0.05 with BF16's 8
    ulp = {"fp16": 2.0 ** -10, "bf16": 2.0 ** -7}[storage] * 0.05
    print(f"{storage}: {differ.mean():.3f} of the values round differently, max |a - b| {np.abs(a - b).max():.2e}")
    assert differ.mean() > 0.05
    assert np.abs(a - b).max() <= ulp
