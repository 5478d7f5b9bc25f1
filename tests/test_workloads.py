"""The synthetic input recipes (seeded, no arithmetic of the scheme) hold
the properties their descriptions state: the random box is positive,
divergence-free with the requested peak speed and correlation length, the
sphere and the shock tubes have the stated geometry and states, and the
generators are deterministic.  CPU."""
import numpy as np
import pytest

import workloads as W


def test_random_box_recipe():
    w = W.random_box(L=48, sigma=4.0)
    assert w.eps.min() > 0 and np.isclose(np.abs(w.eps - 1.0).max(), 0.2)
    assert np.allclose(w.n, w.eps ** 0.75)
    bmag = np.sqrt((w.beta ** 2).sum(0))
    assert np.isclose(bmag.max(), 0.3)
    # divergence-free: spectral divergence of beta vanishes
    k = [2 * np.pi * np.fft.fftfreq(48)] * 3
    kz, ky, kx = np.meshgrid(*k, indexing="ij")
    div = 1j * kx * np.fft.fftn(w.beta[0]) + 1j * ky * np.fft.fftn(w.beta[1]) + 1j * kz * np.fft.fftn(w.beta[2])
    assert np.abs(div).max() <= 1e-9 * np.abs(np.fft.fftn(w.beta[0])).max()
    # smooth on the filter scale (sigma = 4 cells): a step between neighbours stays
    # well below the range
    assert np.abs(np.diff(w.eps, axis=2)).max() < 1.0 / 4.0 * (w.eps.max() - w.eps.min())  # white noise: ~1
    # seeded: the same call gives the same fields, other seeds do not
    w2 = W.random_box(L=48, sigma=4.0)
    assert np.array_equal(w.eps, w2.eps) and np.array_equal(w.beta, w2.beta)
    w3 = W.random_box(L=48, sigma=4.0, seeds=(5, 6, 7, 8))
    assert not np.array_equal(w.eps, w3.eps)


def test_sphere_recipe():
    w = W.sphere_3d()
    assert (w.nx, w.ny, w.nz, w.tau, w.c_l) == (200, 100, 100, 0.8, 1.0)
    z, y, x = np.nonzero(w.solid)
    assert ((x - 60) ** 2 + (y - 50) ** 2 + (z - 50) ** 2 <= 15 ** 2).all()
    assert w.solid.sum() == sum(1 for a in range(-15, 16) for b in range(-15, 16) for c in range(-15, 16)
                                if a * a + b * b + c * c <= 225)
    assert w.beta_in[0] == 0.5 and w.n_in == 1.0 and w.eps_in == 1.0
    fluid = w.solid == 0
    assert np.all(w.beta[:, fluid] == 0) and np.all(w.n[fluid] == 0.3) and np.all(w.eps[fluid] == 1.0)


@pytest.mark.parametrize("make", [W.shock_tube_1d, W.perturbed_shock_tube])
def test_shock_tubes(make):
    w = make()
    assert (w.nx, w.ny, w.nz) == (1600, 1, 1) and w.xbc == 2
    left = np.arange(1600) < 800
    if make is W.shock_tube_1d:
        assert np.all(w.eps[0, 0, left] == 1.0) and np.all(w.eps[0, 0, ~left] == 1 / 16)
        assert np.all(w.n[0, 0, left] == 1.0) and np.all(w.n[0, 0, ~left] == 1 / 8)
    else:
        base = W.shock_tube_1d()
        r = w.eps / base.eps
        assert np.abs(r - 1).max() <= 0.05 and np.abs(r - 1).max() > 0.04
        assert np.array_equal(w.eps, W.perturbed_shock_tube().eps)  # seeded


def test_riemann_tube_states():
    w = W.riemann_tube(2.0, 1.0, 0.5, 0.25, cells=10)
    assert w.nx == 12 and w.xbc == 2
    assert np.allclose(w.eps[0, 0, :6], 6.0) and np.allclose(w.eps[0, 0, 6:], 3.0)
    assert np.allclose(w.n[0, 0, :6], 4.0) and np.allclose(w.n[0, 0, 6:], 4.0)
