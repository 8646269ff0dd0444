"""Pins of the oracle's face-on surface density (cloud-in-cell deposition,
the map of Fig. 4): hand-computed single particles, exact conservation of
mass and of the first moments (bilinear weights reproduce linear
functions), range selection and dropping outside the window, and an
independent brute-force formulation with tent functions."""
import numpy as np

import oracle


def test_particle_at_a_pixel_centre_fills_that_pixel():
    pos = np.array([[0.75], [0.25], [3.0]])
    m = oracle.surface_density(pos, np.array([2.0]), 0, 1, (0.0, 1.0, 0.0, 1.0), 2, 2)
    want = np.zeros((2, 2))
    want[0, 1] = 2.0 / 0.25
    assert np.array_equal(m, want)


def test_particle_on_a_shared_corner_splits_in_quarters():
    pos = np.array([[0.5], [0.5], [0.0]])
    m = oracle.surface_density(pos, np.array([1.0]), 0, 1, (0.0, 1.0, 0.0, 1.0), 2, 2)
    assert np.array_equal(m, np.full((2, 2), 0.25 / 0.25))


def test_mass_and_first_moments_are_conserved():
    rng = np.random.default_rng(3)
    n, nx, ny = 5000, 40, 30
    window = (-2.0, 3.0, -1.0, 2.0)
    hx, hy = 5.0 / nx, 3.0 / ny
    # interior particles: all four deposit pixels inside the grid
    pos = np.stack([rng.uniform(-2.0 + hx, 3.0 - hx, n), rng.uniform(-1.0 + hy, 2.0 - hy, n),
                    rng.normal(size=n)])
    mass = rng.uniform(0.5, 2.0, n)
    m = oracle.surface_density(pos, mass, 0, n, window, nx, ny)
    xc = -2.0 + (np.arange(nx) + 0.5) * hx
    yc = -1.0 + (np.arange(ny) + 0.5) * hy
    area = hx * hy
    assert np.isclose(m.sum() * area, mass.sum(), rtol=1e-13)
    assert np.isclose((m * xc[None, :]).sum() * area, (mass * pos[0]).sum(), rtol=1e-12)
    assert np.isclose((m * yc[:, None]).sum() * area, (mass * pos[1]).sum(), rtol=1e-12)


def test_range_selection_and_window_edges():
    pos = np.array([[0.2, 0.7, 50.0, -0.9], [0.3, 0.6, 0.0, 0.5], [0.0, 0.0, 0.0, 0.0]])
    mass = np.array([1.0, 2.0, 3.0, 4.0])
    w = (0.0, 1.0, 0.0, 1.0)
    only_second = oracle.surface_density(pos, mass, 1, 1, w, 4, 4)
    assert np.isclose(only_second.sum() * (0.25 * 0.25), 2.0)
    far = oracle.surface_density(pos, mass, 2, 2, w, 4, 4)  # one far away, one beyond the left edge
    assert np.all(far == 0.0)


def test_tent_function_brute_force():
    rng = np.random.default_rng(7)
    n, nx, ny = 300, 13, 9
    window = (-1.0, 1.0, -0.5, 0.7)
    pos = np.stack([rng.uniform(-1.3, 1.3, n), rng.uniform(-0.8, 1.0, n), rng.normal(size=n)])
    mass = rng.uniform(0.1, 1.0, n)
    hx, hy = 2.0 / nx, 1.2 / ny
    xc = -1.0 + (np.arange(nx) + 0.5) * hx
    yc = -0.5 + (np.arange(ny) + 0.5) * hy
    tx = np.maximum(0.0, 1.0 - np.abs(pos[0][:, None] - xc[None, :]) / hx)  # (n, nx)
    ty = np.maximum(0.0, 1.0 - np.abs(pos[1][:, None] - yc[None, :]) / hy)  # (n, ny)
    want = np.einsum("i,iy,ix->yx", mass / (hx * hy), ty, tx)
    got = oracle.surface_density(pos, mass, 0, n, window, nx, ny)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * want.max())
