"""Pins of the oracle's lattice tables and MRT matrices (Eqs. 19, 24).

The oracle's tables must equal what the paper prints (golden files typed from
Eq. 19 and Eq. 24) AND satisfy the mathematical requirements of a D2Q9 lattice
(isotropy of the weighted velocity moments up to fourth order) and of an MRT
moment basis (rows are the known polynomials in c_i, mutually orthogonal).
"""
import numpy as np

import oracle


def test_lattice_matches_eq19(lattice_golden):
    c, w = lattice_golden
    cx, cy, wo = oracle.lattice()
    assert np.array_equal(cx, c[:, 0]) and np.array_equal(cy, c[:, 1])
    assert np.array_equal(wo, w)


def test_lattice_isotropy(lattice_golden):
    # Textbook D2Q9 conditions: sum w = 1, odd moments vanish,
    # sum w c_a c_b = cs2 delta, sum w c_a c_b c_c c_d = cs2^2 (dd + dd + dd).
    c, w = lattice_golden
    cs2 = 1.0 / 3.0
    d = np.eye(2)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), cs2 * d, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    t4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(t4, iso, atol=1e-15)


def test_M_matches_eq24(M_golden):
    M, _ = oracle.matrices()
    assert np.array_equal(M, M_golden)


def test_M_rows_are_the_moment_polynomials(lattice_golden):
    # Rows of the D2Q9 MRT basis as polynomials of c (Lallemand & Luo 2000):
    # 1, 3c^2-4, (9c^4-21c^2+8)/2, cx, (3c^2-5)cx, cy, (3c^2-5)cy, cx^2-cy^2, cx cy.
    c, _ = lattice_golden
    cx, cy = c[:, 0], c[:, 1]
    c2 = cx * cx + cy * cy
    rows = np.array([np.ones(9), 3 * c2 - 4, (9 * c2 * c2 - 21 * c2 + 8) / 2, cx,
                     (3 * c2 - 5) * cx, cy, (3 * c2 - 5) * cy, cx * cx - cy * cy, cx * cy])
    M, _ = oracle.matrices()
    assert np.array_equal(M, rows)


def test_M_orthogonal_and_inverse():
    M, Mi = oracle.matrices()
    G = M @ M.T
    assert np.array_equal(G, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]).astype(float))
    assert np.abs(Mi @ M - np.eye(9)).max() < 1e-15
    assert np.abs(M @ Mi - np.eye(9)).max() < 1e-15
    # the inverse of an orthogonal-row matrix is M^T diag(1/|row|^2)
    assert np.abs(Mi - M.T @ np.diag(1.0 / np.diag(G))).max() < 1e-16


def test_model_constants(constants_golden):
    # beta and kappa of Sec. 2 reproduce the surface tension: for the tanh
    # profile of Eq. 4, sigma = kappa * integral(phi'^2) = kappa * 2/(3W).
    W, sigma = 4.0, 1e-3
    beta = constants_golden["beta_over_sigma_times_W"] * sigma / W
    kappa = constants_golden["kappa_over_sigma_over_W"] * sigma * W
    s = np.linspace(-40, 40, 400001)
    dphi = (1.0 / W) / np.cosh(2 * s / W) ** 2
    assert abs(kappa * np.trapezoid(dphi ** 2, s) - sigma) < 1e-9
    # and the oracle's chemical potential uses exactly these beta, kappa:
    # hbar(phi, lap) = 4 beta phi (phi-1)(phi-1/2) - kappa lap
    for phi, lap in [(0.3, 0.0), (0.0, 1.0), (0.7, -0.2)]:
        ref = 4 * beta * phi * (phi - 1) * (phi - 0.5) - kappa * lap
        assert abs(oracle.chem(phi, lap, W, sigma) - ref) < 1e-18
