"""Physics pins of the oracle's full time step (Secs. 2-4).

Each test checks a fact fixed by the paper or by textbook physics, not by the
oracle's own code:
  * the flat tanh profile (Eq. 4) is a steady state of Eq. 17 with hbar = 0;
  * Laplace's law dp = sigma / R for a static 2-D droplet (Eq. 18 with F_s);
  * sum(phi) is conserved on periodic grids (Eq. 35 with sum G_i = 0);
  * a uniform state is a fixed point;
  * with sigma = lambda = 0 the phase field is advected at the fluid speed;
  * a shear wave decays at the viscosity of Eq. 27, nu = c_s^2 (tau_f - 1/2);
  * the modified model (lambda = 0.5) keeps a small droplet's volume far
    better than the classical model (lambda = 0), as Sec. 4.1 reports.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _tanh_eq_hbar(Wd, sigma=1e-2):
    n = int(24 * Wd)
    phi = W.flat_slab(n, 1, n / 4, 3 * n / 4, Wd)
    _, _, lap = oracle.stencil(phi)
    hb = np.array([oracle.chem(p, l, Wd, sigma) for p, l in zip(phi[0], lap[0])])
    return np.abs(hb).max()


def test_tanh_profile_zero_chemical_potential():
    # hbar = 4 beta phi(phi-1)(phi-1/2) - kappa phi'' vanishes for Eq. 4 when
    # beta = 12 sigma/W, kappa = 3 sigma W/2; the discrete Laplacian leaves an
    # O(W^-3) residual (sigma/W scale times the O(W^-2) stencil error, whose
    # coefficient kappa phi''''/12 is about 4/W^2 of sigma/W).
    sigma = 1e-2
    h4, h8, h16 = (_tanh_eq_hbar(w, sigma) for w in (4.0, 8.0, 16.0))
    assert h4 < 0.3 * sigma / 4 and h16 < 0.02 * sigma / 16
    assert 6.0 < h4 / h8 < 10.0 and 6.0 < h8 / h16 < 10.0


@pytest.mark.parametrize("lam", [0.5, 0.0])
def test_flat_interface_is_steady(lam):
    devs = []
    for Wd in (4.0, 8.0):
        nx = int(16 * Wd)
        case = W.base_case(nx, 2, W=Wd, sigma=1e-2, **{"lambda": lam})
        phi0 = W.flat_slab(nx, 2, nx / 4, 3 * nx / 4, Wd)
        o = oracle.Oracle(case, phi0).step(3000)
        phi, ux, uy, _ = o.fields()
        row = phi[0]
        i = int(nx / 4) - 3
        while row[i + 1] < 0.5:
            i += 1
        pos = i + (0.5 - row[i]) / (row[i + 1] - row[i])
        assert abs(pos - nx / 4) < 0.01          # interface stays put
        assert np.abs(ux).max() < 1e-6
        devs.append(np.abs(phi - phi0).max())
    # the discrete profile departs from tanh only at O(W^-2)
    assert devs[0] < 1e-2 and devs[1] < devs[0] / 3.0


def test_laplace_law():
    n, R, sigma = 64, 12.0, 1e-2
    case = W.base_case(n, n, sigma=sigma)
    phi0 = W.tanh_disc(n, n, n / 2, n / 2, R, case["W"])
    o = oracle.Oracle(case, phi0).step(3000)
    phi, ux, uy, p = o.fields()
    R_eff = np.sqrt(phi.sum() / np.pi)
    dp = p[n // 2, n // 2] - p[0, 0]
    assert abs(dp / (sigma / R_eff) - 1.0) < 0.05
    assert np.abs(ux).max() < 1e-4 * 0.5  # spurious currents stay small


def test_global_phi_conserved():
    case, phi0, _, _, _ = W.two_droplets(noise=1e-3)
    o = oracle.Oracle(case, phi0)
    v0 = o.volume()[0]
    o.step(1000)
    assert abs(o.volume()[0] / v0 - 1.0) < 1e-13


def test_uniform_state_is_fixed_point():
    case = W.base_case(7, 5, sigma=1e-2, rho_l=3.0, tau_f_l=0.7, s_f=[1.3] * 9,
                       s_g=[0.9] * 9)
    phi0 = np.full((5, 7), 0.37)
    o = oracle.Oracle(case, phi0)
    f0, g0, j0 = o.f.copy(), o.g.copy(), o.j.copy()
    o.step(50)
    assert np.abs(o.g - g0).max() < 1e-14 and np.abs(o.f - f0).max() < 1e-14
    assert np.array_equal(o.j, j0)
    for a in (o.f, o.g):   # spatially uniform, bit for bit
        assert np.array_equal(a, np.broadcast_to(a[:, :1, :1], a.shape))


@pytest.mark.parametrize("u", [0.01, 0.02])
def test_pure_advection(u):
    # sigma = 0 and lambda = 0: Eq. 17 reduces to d_t phi + div(phi u) = 0.
    n, N = 64, 1000
    case = W.base_case(n, 4, sigma=0.0, **{"lambda": 0.0})
    x = np.arange(n)[None, :] * np.ones((4, 1))
    phi0 = 0.5 + 0.3 * np.sin(2 * np.pi * x / n)
    u0 = np.zeros((2, 4, n))
    u0[0] = u
    o = oracle.Oracle(case, phi0, u0).step(N)
    phi = o.fields()[0][0]
    c, c0 = np.fft.fft(phi)[1], np.fft.fft(phi0[0])[1]
    shift = -np.angle(c / c0) / (2 * np.pi / n)
    assert abs(shift / (u * N) - 1.0) < 3e-3
    assert abs(abs(c) / abs(c0) - 1.0) < 1e-4


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.4])
def test_shear_wave_viscosity(tau):
    n, U = 64, 1e-3
    case = W.base_case(4, n, sigma=0.0, tau_f_l=tau, tau_f_g=tau, **{"lambda": 0.0})
    y = np.arange(n)[:, None] * np.ones((1, 4))
    u0 = np.zeros((2, n, 4))
    u0[0] = U * np.sin(2 * np.pi * y / n)
    o = oracle.Oracle(case, np.zeros((n, 4)), u0)
    amps = []
    for t in (200, 1200):
        o.step(t - o.t)
        ux = o.fields()[1][:, 0]
        amps.append((ux * np.sin(2 * np.pi * np.arange(n) / n)).sum() * 2 / n)
    k = 2 * np.pi / n
    nu = -np.log(amps[1] / amps[0]) / (1000 * k * k)
    assert abs(nu / ((tau - 0.5) / 3.0) - 1.0) < 5e-3


def test_variable_density_rest_state():
    # Density ratio 10 with a flat interface at rest: no force drives flow
    # beyond the discretisation residual and phi stays conserved.
    nx = 64
    case = W.base_case(nx, 2, sigma=1e-2, rho_l=10.0, tau_f_l=0.6, tau_f_g=1.0)
    phi0 = W.flat_slab(nx, 2, 16, 48, case["W"])
    o = oracle.Oracle(case, phi0)
    v0 = o.volume()[0]
    o.step(2000)
    phi, ux, uy, p = o.fields()
    assert np.isfinite(phi).all() and np.abs(ux).max() < 1e-5
    assert abs(o.volume()[0] / v0 - 1) < 1e-13


def test_small_droplet_volume_modified_vs_classical():
    # Sec. 4.1: the classical C-H model (lambda = 0) shrinks the small
    # droplet; the modified model keeps it "nearly constant".  Paper values
    # of Sec. 4.1: W = 3, M = 0.1 (tau_g = 0.8), sigma = 0.01, ratios 1.
    n = 64
    drops = [(20.0, 32.0, 12.0), (46.0, 32.0, 5.0)]
    lab = W.nearest_surface_labels(n, n, drops)
    loss = {}
    for lam in (0.5, 0.0):
        case = W.base_case(n, n, W=3.0, sigma=0.01, **{"lambda": lam})
        o = oracle.Oracle(case, W.droplets_field(n, n, drops, 3.0))
        v0 = o.volume(lab, 2)
        o.step(3000)
        loss[lam] = (o.volume(lab, 2) - v0) / v0
    assert loss[0.0][1] < 0 and loss[0.5][1] < 0
    assert abs(loss[0.5][1]) < 0.5 * abs(loss[0.0][1])


def test_uniform_translation_is_fixed_point():
    # phi const, u const, no force: f = f_eq(p = 0, u) and g = g_eq stay put
    # exactly (Galilean uniform flow; p from Eq. 29 is 0 for f_eq(p = 0, u)).
    case = W.base_case(6, 5, sigma=1e-2, rho_l=2.0)
    phi0 = np.full((5, 6), 0.4)
    u0 = np.zeros((2, 5, 6))
    u0[0], u0[1] = 0.03, -0.02
    o = oracle.Oracle(case, phi0, u0)
    f0, g0 = o.f.copy(), o.g.copy()
    o.step(20)
    phi, ux, uy, p = o.fields()
    assert np.abs(p).max() < 1e-15
    assert np.abs(ux - 0.03).max() < 1e-15 and np.abs(uy + 0.02).max() < 1e-15
    assert np.abs(o.f - f0).max() < 1e-15 and np.abs(o.g - g0).max() < 1e-15


def test_coarse_sheared_droplet_classical_shrinks_modified_keeps():
    # Sec. 4.4 on its own grid (128 x 64 cavity, droplet radius 8, walls at
    # -U and +U): the classical model (lambda = 0) moves phi from the droplet
    # into the bulk from the start, the modified model holds the area
    # enclosed by phi = 1/2 (after the initial profile settles).  The area is
    # counted on a 4x bilinear refinement of phi.
    from scipy import ndimage

    def area(phi):
        z = ndimage.zoom(phi, 4, order=1, mode="grid-wrap", grid_mode=True)
        return np.count_nonzero(z > 0.5) / 16.0

    change = {}
    for lam in (0.5, 0.0):
        case, phi0, u0 = W.coarse_sheared_droplet(lam=lam)
        o = oracle.Oracle(case, phi0, u0).step(3000)
        change[lam] = area(o.fields()[0]) / area(phi0) - 1
    assert change[0.0] < -0.02
    assert abs(change[0.5]) < 0.25 * abs(change[0.0])
