"""Pins of the oracle's prescribed single-vortex flow (Sec. 4.2, Eqs. 43-44).

The paper prints the velocity only in a garbled form.  The reading the oracle
takes (node-centred coordinates X = (x + 1/2)/nx, Y = (y + 1/2)/ny, time in
steps, u = -U sin^2(pi X) sin(2 pi Y) cos(pi t/T), v = +U sin^2(pi Y)
sin(2 pi X) cos(pi t/T)) is checked here through what the set-up fixes, not
by evaluating the formula again:

  * the flow is incompressible: both components are single Fourier modes in
    each direction, so on a square grid the isotropic divergence of Sec. 3.2
    cancels exactly (to rounding); swapping X and Y, a flipped sign of one
    component, or sin for sin^2 each leave an O(U/L) divergence;
  * the field is symmetric about the centre of the unit square, which falls
    between nodes with node-centred coordinates: u is even and v odd under
    x -> nx-1-x, and the reverse under y -> ny-1-y;
  * its peak speed is U, reached between nodes, so the node maximum falls
    short of U by O(L^-2);
  * the time factor reverses the flow: u(T - t) = -u(t), u(T/2) = 0;
  * so the advected droplet returns to its start after one period (the test
    of Sec. 4.2): its shape error at t = T is far below that at T/2, and the
    error at 3T/4 equals the one at T/4 (the motion retraces itself);
  * sum(phi) is conserved under the prescribed flow, as in the coupled step.
"""
import numpy as np

import oracle
import workloads as W


def _vortex(n, U=0.02, T=512, nx=None):
    case, phi0, _ = W.single_vortex(n=n, W=3.0, U=U, T=T)
    if nx is not None:  # a non-square grid: X and Y scale with their own edges
        case = dict(case, nx=nx)
        phi0 = W.tanh_disc(nx, n, 0.5 * nx, 0.75 * n, 0.15 * n, 3.0)
    return case, phi0


def _velocity(case, phi0, t):
    o = oracle.Oracle(case, phi0)
    o.t = int(t)  # the prescribed field depends on the step index only
    _, ux, uy, _ = o.fields()
    return ux, uy


def test_vortex_is_divergence_free():
    # on the square grid of Sec. 4.2 the two terms of the discrete divergence
    # are the same product of one x-mode and one y-mode with opposite signs
    for n in (32, 64, 96):
        case, phi0 = _vortex(n)
        ux, uy = _velocity(case, phi0, 0)
        gxu, _, _ = oracle.stencil(ux)
        _, gyv, _ = oracle.stencil(uy)
        scale = np.abs(gxu).max()
        assert scale > 0.5 * 0.02 * np.pi / n  # each term is O(U/L), not 0
        assert np.abs(gxu + gyv).max() < 1e-13 * scale


def test_vortex_mirror_symmetry_node_centred():
    case, phi0 = _vortex(64, nx=96)
    ux, uy = _velocity(case, phi0, 0)
    tol = 1e-15
    # x -> nx-1-x: u even, v odd; y -> ny-1-y: u odd, v even
    assert np.abs(ux[:, ::-1] - ux).max() < tol
    assert np.abs(uy[:, ::-1] + uy).max() < tol
    assert np.abs(ux[::-1, :] + ux).max() < tol
    assert np.abs(uy[::-1, :] - uy).max() < tol
    # the flow circulates: u changes sign between the lower and upper half
    assert ux[16, 48] * ux[48, 48] < 0 and uy[32, 24] * uy[32, 72] < 0


def test_vortex_peak_speed():
    U = 0.02
    deficits = []
    for n in (32, 64, 128, 256):
        case, phi0 = _vortex(n, U=U)
        ux, uy = _velocity(case, phi0, 0)
        peak = max(np.abs(ux).max(), np.abs(uy).max())
        assert peak < U
        deficits.append(1.0 - peak / U)
    # the maximum sits between nodes: the node value falls short at O(L^-2)
    assert deficits[-1] < 2e-4
    for a, b in zip(deficits, deficits[1:]):
        assert 3.5 < a / b < 4.5


def test_vortex_time_factor_reverses_flow():
    T = 512
    case, phi0 = _vortex(64, T=T)
    u0x, u0y = _velocity(case, phi0, 0)
    scale = np.abs(u0x).max()
    for t in (1, 37, 128, 200):
        ax, ay = _velocity(case, phi0, t)
        bx, by = _velocity(case, phi0, T - t)
        assert np.abs(ax + bx).max() < 1e-15 and np.abs(ay + by).max() < 1e-15
        assert np.abs(ax).max() > 1e-3 * scale
    hx, hy = _velocity(case, phi0, T // 2)
    assert np.abs(hx).max() < 1e-15 * scale / 1e-2 and np.abs(hy).max() < 1e-15 * scale / 1e-2
    ex, ey = _velocity(case, phi0, T)
    assert np.abs(ex + u0x).max() < 1e-15 and np.abs(ey + u0y).max() < 1e-15


def test_vortex_droplet_returns_after_one_period():
    T = 512
    case, phi0 = _vortex(64, T=T)
    o = oracle.Oracle(case, phi0)
    v0 = o.volume()[0]
    err = {}
    for t in (T // 4, T // 2, 3 * T // 4, T):
        o.step(t - o.t)
        err[t] = np.abs(o.phi() - phi0).sum() / phi0.sum()
    # stretched at half period (the droplet moves ~U T / pi = 3.3 lattice units)
    assert err[T // 2] > 0.2
    # and back at the full period, up to the interface's own relaxation
    assert err[T] < 0.05 * err[T // 2]
    # the second half of the period retraces the first
    assert abs(err[3 * T // 4] - err[T // 4]) < 0.01 * err[T // 4]
    assert err[T // 4] < err[T // 2]
    # the prescribed flow conserves sum(phi)
    assert abs(o.volume()[0] / v0 - 1.0) < 1e-13
