"""GPU parity of the moving walls (2-D, register-pipelined and persistent
kernels) against the FP64 oracle, through the C ABI: halfway bounce-back,
moving-wall term on f with rho of the receiving node, plain bounce-back of g,
mirrored ghost row for the stencils.  Tolerances as in test_gpu_parity.py:
FP64 1e-12, FP32 phi 1e-5."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_10899_gb300 import build
    build.build()
    from paper_2505_10899_gb300 import lbm
    return lbm


def md(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max())


def sheared(nx, ny, u_top=0.02, u_bot=-0.01, **kw):
    case = W.base_case(nx, ny, walls=1, u_top=u_top, u_bot=u_bot, sigma=1e-2, **kw)
    phi0 = W.tanh_disc(nx, ny, 0.4 * nx + 0.3, 5.2, 0.35 * min(nx, ny), 4.0)  # on the bottom wall
    u0 = np.zeros((2, ny, nx))
    u0[0] = u_bot + (u_top - u_bot) * (np.arange(ny)[:, None] + 0.5) / ny
    u0 += W.uniform(3, (2, ny, nx), -2e-3, 2e-3)
    return case, phi0, u0


def check(L, o, s, tol_pop, tol_phi, c=0):
    f, g, j, t = s.get_state(c)
    assert t == o.t
    assert md(f, o.f) <= tol_pop and md(g, o.g) <= tol_pop and md(j, o.j) <= tol_pop
    phi, ux, uy, p = s.fields(c)
    ophi, oux, ouy, op = o.fields()
    assert md(phi, ophi) <= tol_phi
    assert md(ux, oux) <= tol_pop and md(uy, ouy) <= tol_pop and md(p, op) <= tol_pop


@pytest.mark.parametrize("kw", [dict(), dict(rho_l=3.0, tau_f_l=0.7, tau_f_g=1.1)],
                         ids=["ratio1", "ratio3_var_tau"])
def test_fp64_walls_100_steps(L, kw):
    case, phi0, u0 = sheared(70, 36, **kw)
    o = oracle.Oracle(case, phi0, u0).step(100)
    s = L.Sim(case, phi0, u0, precision="f64")
    assert s.kernel() == 1  # walls run the register-pipelined kernel
    s.step(100)
    check(L, o, s, TOL64, TOL64)
    assert s.status() == L.LBM_OK


def test_fp64_walls_random_state(L):
    # import with walls (bounce-back positions, moving-wall term removed),
    # then 7 steps and export, against the oracle from the same state
    nx, ny = 45, 19
    case = W.base_case(nx, ny, walls=1, u_top=0.01, u_bot=-0.03, sigma=1e-2, rho_l=10.0,
                       tau_f_l=0.6, tau_f_g=1.0)
    f, g, j = W.random_state(nx, ny, seed=41)
    s = L.Sim(case, np.zeros((ny, nx)), None, precision="f64")
    s.set_state(0, f, g, j, 3)
    f2, g2, j2, t2 = s.get_state(0)
    assert md(f2, f) < 1e-15 and md(g2, g) == 0.0 and t2 == 3  # round trip
    o = oracle.Oracle(case, state=(f, g, j, 3)).step(7)
    s.step(7)
    check(L, o, s, TOL64, TOL64)


@pytest.mark.parametrize("shape", [(7, 1), (1, 5), (5, 2), (33, 3)])
def test_fp64_walls_degenerate_grids(L, shape):
    nx, ny = shape
    case = W.base_case(nx, ny, walls=1, u_top=0.02, u_bot=0.01, sigma=1e-2, rho_l=2.0,
                       tau_f_l=0.8)
    f, g, j = W.random_state(nx, ny, seed=9, phi_lo=0.2, phi_hi=0.8)
    s = L.Sim(case, np.zeros((ny, nx)), None, precision="f64")
    s.set_state(0, f, g, j, 0)
    o = oracle.Oracle(case, state=(f, g, j, 0)).step(20)
    s.step(20)
    check(L, o, s, TOL64, TOL64)


def test_fp32_walls(L):
    case, phi0, u0 = sheared(70, 36, rho_l=3.0, tau_f_l=0.7)
    o = oracle.Oracle(case, phi0, u0).step(100)
    s = L.Sim(case, phi0, u0, precision="f32").step(100)
    phi, ux, uy, p = s.fields(0)
    ophi, oux, ouy, op = o.fields()
    assert md(phi, ophi) <= 1e-5 and md(ux, oux) <= 1e-6 and md(uy, ouy) <= 1e-6


def test_walls_mixed_batch_and_persistent_kernel(L):
    # a periodic case and two wall cases in one launch; then the persistent kernel
    c1, p1, u1 = sheared(40, 24)
    c2 = W.base_case(48, 30, sigma=1e-2)
    p2, u2 = W.tanh_disc(48, 30, 20.3, 14.6, 7.0, 4.0), None
    c3, p3, u3 = sheared(33, 17, u_top=0.0, u_bot=0.015, rho_l=2.0)
    cases, phis, us = [c1, c2, c3], [p1, p2, p3], [u1, u2, u3]
    for variant in (1, 3):
        s = L.Sim(cases, phis, us, precision="f64")
        s.set_kernel(variant)
        s.step(30)
        for k in range(3):
            o = oracle.Oracle(cases[k], phis[k], us[k]).step(30)
            check(L, o, s, TOL64, TOL64, c=k)
        with pytest.raises(L.LbmError):
            s.set_kernel(2)  # the bulk-copy kernel is periodic-only


def test_couette_steady_profile_fp32(L):
    nx, ny, U = 32, 24, 0.01
    case = W.base_case(nx, ny, walls=1, u_top=U, u_bot=-U, sigma=0.0, tau_f_l=1.0,
                       tau_f_g=1.0, **{"lambda": 0.0})
    s = L.Sim(case, np.zeros((ny, nx)), None, precision="f32").step(20000)
    ux = s.fields(0)[1]
    exact = -U + 2 * U * (np.arange(ny) + 0.5) / ny
    assert np.abs(ux - exact[:, None]).max() < 1e-5 * U


def test_fp32_walls_volume_drift_1e4_steps(L):
    case, phi0, u0 = W.shear_droplet(nx=128, ny=64, R=12.0, U=0.01, Ca=0.2, Re=0.2)
    s = L.Sim(case, phi0, u0, precision="f32")
    v0 = s.volume()[0]
    s.step(10000)
    assert s.status() == L.LBM_OK
    assert abs(s.volume()[0] / v0 - 1) <= 1e-6
