"""Host-side measurements of the Sec. 4.3/4.4 experiments (no GPU): the
phi = 1/2 contour area and volume against the exact disc and ball, and the
periodic connected components against hand-made masks; the workload
generators of Eqs. 45 and 46 against their printed forms."""
import numpy as np
import pytest

import workloads as W
from paper_2505_10899_gb300 import experiments as E


@pytest.mark.parametrize("R", [5.3, 8.0, 12.7])
def test_contour_area_of_tanh_disc(R):
    phi = W.tanh_disc(64, 48, 31.4, 22.8, R, 4.0)
    assert abs(E.contour_measure(phi) / (np.pi * R * R) - 1) < 0.02


def test_contour_volume_of_tanh_ball():
    R = 9.5
    phi = W.tanh_ball(40, 36, 32, 20.2, 17.7, 15.9, R, 4.0)
    assert abs(E.contour_measure(phi, up=2) / (4 / 3 * np.pi * R ** 3) - 1) < 0.02


def test_contour_area_wraps_only_when_periodic():
    # a disc cut by the x = 0 face: whole when periodic; clamping the
    # interpolant at the edges can only lose area
    phi = W.tanh_disc(40, 40, 0.0, 20.0, 8.0, 4.0, periodic=True)
    a = E.contour_measure(phi, periodic=True)
    assert abs(a / (np.pi * 64) - 1) < 0.02
    assert E.contour_measure(phi, periodic=False) <= a


def test_components_join_across_periodic_faces():
    m = np.zeros((6, 7, 8), bool)
    m[0, 2, 2] = m[5, 2, 2] = True               # joined through axis 0
    m[3, 3, 0] = m[3, 3, 7] = m[3, 4, 7] = True  # joined through axis 2
    m[2, 5, 4] = True                            # alone
    assert E.components(m) == [3, 2, 1]
    assert E.components(m, periodic_axes=()) == [2, 1, 1, 1, 1]
    assert E.components(m, periodic_axes=(0,)) == [2, 2, 1, 1]
    assert E.components(np.zeros((4, 4), bool)) == []
    assert E.components(np.ones((3, 5), bool)) == [15]


def test_components_diagonal_neighbours_are_apart():
    m = np.zeros((5, 5), bool)
    m[1, 1] = m[2, 2] = True
    assert E.components(m, periodic_axes=()) == [1, 1]


def test_eq45_film_and_column_shapes():
    case, phi = W.film_eq45()
    ny, nx = phi.shape
    assert (nx, ny) == (256, 128) and case["walls"] == 1 and case["u_top"] == case["u_bot"] == 0
    h = np.pi / ny
    # liquid height along y (the sum of phi) = a + amp cos x in lattice units
    height = phi.sum(axis=0)
    x = np.arange(nx) * 2 * np.pi / nx
    assert np.abs(height - (0.15 + 0.05 * np.cos(x)) / h).max() < 0.05
    n = 64
    case3, phi3 = W.column_eq45(n=n)
    assert (case3["nx"], case3["ny"], case3["nz"]) == (n, n, n)
    h3 = 2 * np.pi / n
    # the phi = 1/2 radius, from the profile 3 nodes off the axis in each
    # z plane, is (a + amp cos z) / h3 lattice units
    r_half = 3.0 + 0.5 * case3["W"] * np.arctanh(2 * phi3[:, n // 2, n // 2 + 3] - 1)
    assert np.abs(r_half - (0.15 + 0.05 * np.cos(np.arange(n) * h3)) / h3).max() < 1e-9
    sec = phi3.sum(axis=(1, 2))
    assert sec.argmax() == 0 and sec.argmin() == n // 2
    case4, phi4 = W.column_eq45(n=n, n_side=24)
    assert phi4.shape == (n, 24, 24) and (case4["nx"], case4["nz"]) == (24, n)


def test_coarse_sheared_droplet_is_eq46():
    case, phi, u = W.coarse_sheared_droplet()
    assert phi.shape == (64, 128) and case["walls"] == 1
    assert case["u_top"] == -case["u_bot"] == 0.01
    assert abs(E.contour_measure(phi) / (np.pi * 64) - 1) < 0.02
    iy, ix = np.unravel_index(phi.argmax(), phi.shape)
    assert abs(ix - 64) <= 1 and abs(iy - 31.5) <= 1
    assert np.allclose(u[0, :, 0], -0.01 + 0.02 * (np.arange(64) + 0.5) / 64)
