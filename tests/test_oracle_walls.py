"""Pins of the oracle's moving walls (halfway bounce-back below y = 0 and above
y = ny - 1, moving-wall momentum term on f, plain bounce-back of g, mirrored
ghost row for the stencils of Sec. 3.2):
  * Couette flow: the steady profile between walls moving at -U and +U is the
    exact linear profile through the half-way wall positions;
  * the walls let no phi through: sum(phi) is conserved in a sheared channel;
  * a mirror y -> ny - 1 - y that swaps the walls maps solutions onto solutions;
  * walls at rest around a fluid at rest with a flat interface parallel to
    them are a steady state;
  * a droplet in simple shear deforms as Taylor's small-deformation theory
    predicts (D = (35/32) Ca for equal viscosities), within the confinement
    and finite-width error.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def channel(nx, ny, **kw):
    c = W.base_case(nx, ny, walls=1, **kw)
    return c


def test_couette_profile_is_exact():
    nx, ny, U = 4, 16, 0.01
    for tau in (0.8, 1.3):
        case = channel(nx, ny, sigma=0.0, tau_f_l=tau, tau_f_g=tau, u_top=U, u_bot=-U,
                       **{"lambda": 0.0})
        o = oracle.Oracle(case, np.zeros((ny, nx)))
        o.step(int(12 / ((tau - 0.5) / 3.0 * (np.pi / ny) ** 2)))
        phi, ux, uy, p = o.fields()
        y = np.arange(ny)
        exact = -U + 2 * U * (y + 0.5) / ny  # walls half-way outside the end rows
        assert np.abs(ux[:, 0] - exact).max() < 1e-9 * U
        assert np.abs(uy).max() < 1e-12
        assert np.abs(p).max() < U * U  # an O(U^2) pressure level, no gradient along x
        assert np.abs(p - p[:, :1]).max() < 1e-15


def test_walls_conserve_phi():
    nx, ny = 48, 32
    case = channel(nx, ny, sigma=1e-2, rho_l=3.0, tau_f_l=0.7, u_top=0.02, u_bot=-0.01)
    phi0 = W.tanh_disc(nx, ny, 20.0, 5.0, 8.0, 4.0)  # touches the bottom wall
    u0 = np.zeros((2, ny, nx))
    u0[0] = -0.01 + 0.03 * (np.arange(ny)[:, None] + 0.5) / ny
    o = oracle.Oracle(case, phi0, u0)
    v0 = o.volume()[0]
    o.step(400)
    assert np.isfinite(o.f).all()
    assert abs(o.volume()[0] / v0 - 1) < 1e-13


def test_mirror_symmetry_swaps_the_walls():
    nx, ny = 24, 20
    kw = dict(sigma=1e-2, rho_l=2.0, tau_f_l=0.8)
    # centre off the nodes: at a node where grad(psi) vanishes by symmetry, the
    # normal of Eq. 32 takes its direction from rounding noise (ill-conditioned)
    phi0 = W.tanh_disc(nx, ny, 11.3, 7.6, 5.0, 4.0)
    u0 = W.uniform(7, (2, ny, nx), -0.005, 0.005)
    a = oracle.Oracle(channel(nx, ny, u_top=0.015, u_bot=-0.005, **kw), phi0, u0).step(60)
    m = lambda q: q[::-1].copy()
    um = np.stack([m(u0[0]), -m(u0[1])])
    b = oracle.Oracle(channel(nx, ny, u_top=-0.005, u_bot=0.015, **kw), m(phi0), um).step(60)
    pa, uxa, uya, pra = a.fields()
    pb, uxb, uyb, prb = b.fields()
    assert np.abs(pb - m(pa)).max() < 1e-13
    assert np.abs(uxb - m(uxa)).max() < 1e-15
    assert np.abs(uyb + m(uya)).max() < 1e-15
    assert np.abs(prb - m(pra)).max() < 1e-15
    # and the walls matter: the unswapped mirror is not a solution
    c = oracle.Oracle(channel(nx, ny, u_top=0.015, u_bot=-0.005, **kw), m(phi0), um).step(60)
    assert np.abs(c.fields()[1] - m(uxa)).max() > 1e-4


def test_resting_walls_and_flat_interface_are_steady():
    nx, ny = 4, 48
    case = channel(nx, ny, sigma=1e-2, rho_l=4.0, tau_f_l=0.7)
    # interface parallel to the walls, at y = 16 and y = 32
    phi0 = np.ascontiguousarray(W.flat_slab(ny, nx, 16, 32, 4.0).T)
    o = oracle.Oracle(case, phi0)
    # Resting walls admit only u = 0 as a steady state: the set-up is uniform
    # in x and symmetric under x -> -x, so u_x = 0 at every step, and between
    # walls that pass no mass a steady u_y(y) must vanish.  The profile
    # settling to its discrete equilibrium at density ratio 4 starts a flow
    # along y (pressure waves and the slower Cahn-Hilliard relaxation); its
    # largest value over successive windows of four times the length must
    # fall steadily towards zero.
    env = []
    for a, b in ((250, 1000), (1000, 4000), (4000, 16000)):
        m = 0.0
        o.step(a - o.t)
        while o.t < b:
            o.step(25)
            phi, ux, uy, p = o.fields()
            assert np.abs(ux).max() == 0.0
            m = max(m, np.abs(uy).max())
        env.append(m)
    assert env[0] > 2.5 * env[1] > 2.5 * 2.5 * env[2]
    assert env[2] < 3e-7
    assert np.abs(phi - phi0).max() < 2e-2


def _taylor_D(phi):
    # deformation D = (L - B)/(L + B) from the second moments of phi about its
    # centroid: L, B proportional to the square roots of their eigenvalues
    ny, nx = phi.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    m = phi.sum()
    cx, cy = (phi * x).sum() / m, (phi * y).sum() / m
    dx, dy = x - cx, y - cy
    I = np.array([[(phi * dx * dx).sum(), (phi * dx * dy).sum()],
                  [(phi * dx * dy).sum(), (phi * dy * dy).sum()]]) / m
    ev = np.linalg.eigvalsh(I)
    L, B = np.sqrt(ev[1]), np.sqrt(ev[0])
    return (L - B) / (L + B)


@pytest.mark.slow
def test_droplet_deformation_in_shear_follows_taylor():
    nx, ny, R, U, Ca, Re = 128, 64, 10.0, 0.01, 0.1, 0.1
    gam = 2 * U / ny
    nu = gam * R * R / Re
    tau = 3 * nu + 0.5
    sigma = nu * gam * R / Ca
    case = channel(nx, ny, sigma=sigma, tau_f_l=tau, tau_f_g=tau, tau_g=0.8, u_top=U,
                   u_bot=-U, W=4.0)
    phi0 = W.tanh_disc(nx, ny, nx / 2, ny / 2, R, 4.0)
    u0 = np.zeros((2, ny, nx))
    u0[0] = -U + 2 * U * (np.arange(ny)[:, None] + 0.5) / ny
    o = oracle.Oracle(case, phi0, u0).step(3000)
    D = _taylor_D(o.fields()[0])
    assert abs(D / ((35.0 / 32.0) * Ca) - 1) < 0.25


def test_half_disc_on_a_wall_keeps_its_90_degree_contact_angle():
    # The mirrored ghost row is a zero normal gradient of phi at the wall:
    # neutral wetting, contact angle 90 degrees.  A half-disc centred on the
    # wall (y = -1/2) is then an equilibrium shape; it must stay put.
    nx, ny, R = 64, 32, 10.0
    case = channel(nx, ny, sigma=1e-2, tau_f_l=0.8, tau_f_g=0.8)
    phi0 = W.tanh_disc(nx, ny, nx / 2 - 0.3, -0.5, R, 4.0)
    o = oracle.Oracle(case, phi0).step(2000)
    phi, ux, uy, p = o.fields()
    assert np.abs(phi - phi0).max() < 2e-2
    assert np.abs(ux).max() < 2e-4 and np.abs(uy).max() < 2e-4
    # contact line still where the tanh profile puts it: phi = 1/2 at |x - xc| = R
    row = phi[0]
    xc = nx / 2 - 0.3
    right = np.interp(0.5, row[int(xc) + 14:int(xc) + 4:-1], np.arange(int(xc) + 14, int(xc) + 4, -1))
    assert abs(right - (xc + np.sqrt(R * R - 0.25))) < 0.3
