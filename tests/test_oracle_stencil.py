"""Pins of the isotropic finite-difference stencils of Sec. 3.2 (Thampi et al.).

The second-order isotropic gradient and Laplacian are exact on quadratic
polynomials and converge at second order on smooth periodic fields.
"""
import numpy as np

import oracle


def test_exact_on_quadratics():
    nx, ny = 23, 17
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    a, b, c, d, e, f = 0.3, -1.2, 0.7, 0.05, -0.11, 0.02
    chi = a + b * x + c * y + d * x * x + e * x * y + f * y * y
    gx, gy, lap = oracle.stencil(chi)
    inner = (slice(1, ny - 1), slice(1, nx - 1))   # away from the periodic seam
    assert np.abs(gx[inner] - (b + 2 * d * x + e * y)[inner]).max() < 1e-12
    assert np.abs(gy[inner] - (c + e * x + 2 * f * y)[inner]).max() < 1e-12
    assert np.abs(lap[inner] - (2 * d + 2 * f)).max() < 1e-12


def test_constant_field_has_zero_gradient_exactly():
    chi = np.full((9, 11), 0.123456789)
    gx, gy, lap = oracle.stencil(chi)
    assert not gx.any() and not gy.any() and not lap.any()


def _errors(n):
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    k = 2 * np.pi / n
    chi = np.sin(k * x + 0.3) * np.cos(2 * k * y)
    gx, gy, lap = oracle.stencil(chi)
    ex_gx = k * np.cos(k * x + 0.3) * np.cos(2 * k * y)
    ex_gy = -2 * k * np.sin(k * x + 0.3) * np.sin(2 * k * y)
    ex_lap = -5 * k * k * chi
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    return rel(gx, ex_gx), rel(gy, ex_gy), rel(lap, ex_lap)


def test_second_order_convergence():
    e1 = np.array(_errors(32))
    e2 = np.array(_errors(64))
    order = np.log2(e1 / e2)
    assert np.all(order > 1.9) and np.all(order < 2.1), order
    assert np.all(e2 < 1e-2)


def test_interface_gradient_of_psi_is_far_above_the_ridge_cut():
    # psi of Eq. 14 is a signed distance: across the interface band of a
    # resolved droplet its isotropic gradient is close to 1, so the cut of the
    # normal at |grad psi| < 0.1 touches only the saturated bulk and the
    # ridge at the centre (node-centred and off-node droplets, R = 6 and 12).
    import numpy as np
    import oracle
    import workloads as W
    for R, cx in ((12.0, 32.0), (6.0, 32.0), (12.0, 32.4)):
        phi = W.tanh_disc(64, 64, cx, 32.0, R, 4.0, periodic=True)
        psi = np.vectorize(lambda p: oracle.psi(p, 4.0, 1e-10))(phi)
        gx, gy, _ = oracle.stencil(psi)
        g = np.hypot(gx, gy)
        band = (phi > 0.01) & (phi < 0.99)
        assert g[band].min() > 0.9
        assert (phi[g < 0.1] * (1 - phi[g < 0.1])).max() < 1e-2
