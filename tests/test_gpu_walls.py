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


# ---------------------------------------------------------------- reverse mode

def _ad_modules():
    from paper_2505_10899_gb300 import adjoint
    return adjoint


def _one_step_out(A, case, state, t):
    s = A.AdjointSim(case, np.full((case["ny"], case["nx"]), 0.5))
    s.restore(state, t)
    s.step(1)
    out = s.snapshot()
    s.close()
    return out


def test_adjoint_step_with_walls_matches_fd(L):
    # one step: <lambda_t, delta> against central differences of the GPU
    # forward step, for the state and all six parameters (incl. wall speeds)
    import torch
    A = _ad_modules()
    nx, ny = 36, 20
    case = W.base_case(nx, ny, walls=1, u_top=0.02, u_bot=-0.01, sigma=5e-3, rho_l=4.0,
                       tau_f_l=0.9, tau_f_g=0.9)
    f, g, j = W.random_state(nx, ny, seed=17, coupled=True, phi_lo=0.1, phi_hi=0.9)
    base = A.AdjointSim(case, np.full((ny, nx), 0.5))
    base.sim.set_state(0, f, g, j, 5)
    S = base.snapshot()
    lam_out = torch.as_tensor(W.uniform(11, (20, ny, nx), -1, 1), device="cuda")
    delta = torch.as_tensor(W.uniform(12, (20, ny, nx), -1, 1), device="cuda")
    grads = np.zeros(6)
    lam_in = base.vjp_step(lam_out, grads)
    eps = 1e-6
    fd = float(((_one_step_out(A, case, S + eps * delta, 5)
                 - _one_step_out(A, case, S - eps * delta, 5)) * lam_out).sum()) / (2 * eps)
    ad = float((lam_in * delta).sum())
    assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-9, (ad, fd)
    th0 = np.array([case["sigma"], case["tau_g"], case["lambda"], case["tau_f_l"],
                    case["u_top"], case["u_bot"]])
    for q, h in enumerate([1e-7, 1e-6, 1e-6, 1e-6, 1e-6, 1e-6]):
        outs = []
        for sgn in (+1, -1):
            th = th0.copy()
            th[q] += sgn * h
            outs.append(_one_step_out(A, A.case_with(case, th), S, 5))
        fdq = float(((outs[0] - outs[1]) * lam_out).sum()) / (2 * h)
        assert abs(grads[q] - fdq) <= 1e-5 * abs(fdq) + 1e-7, (q, grads[q], fdq)
    assert abs(grads[4]) > 0 and abs(grads[5]) > 0
    base.close()


def _np_taylor_D(phi):
    ny, nx = phi.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    m = phi.sum()
    cx, cy = (phi * x).sum() / m, (phi * y).sum() / m
    dx, dy = x - cx, y - cy
    I = np.array([[(phi * dx * dx).sum(), (phi * dx * dy).sum()],
                  [(phi * dx * dy).sum(), (phi * dy * dy).sum()]]) / m
    ev = np.linalg.eigvalsh(I)
    return (np.sqrt(ev[1]) - np.sqrt(ev[0])) / (np.sqrt(ev[1]) + np.sqrt(ev[0]))


def test_taylor_deformation_gradient_vs_oracle_fd(L):
    # J = D(phi_T) of a sheared droplet: gradients through the checkpointed
    # reverse mode against central differences of J from the FP64 oracle
    import torch
    A = _ad_modules()
    case, phi0, u0 = W.shear_droplet(nx=48, ny=32, R=6.0, U=0.01, Ca=0.2, Re=0.5)
    T = 160
    th0 = np.array([case["sigma"], case["tau_g"], case["lambda"], case["tau_f_l"],
                    case["u_top"], case["u_bot"]])
    phi0_t = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
    th_t = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    phiT = A.coupled_run(phi0_t, th_t, case, T, ckpt_every=32, u0=u0)
    J = A.taylor_deformation(phiT)
    J.backward()
    g = th_t.grad.numpy()

    def oJ(th, p0=phi0):
        o = oracle.Oracle(A.case_with(case, th), p0, u0).step(T)
        phi = o.fields()[0]
        # the clip of Eq. 37 is touched only by round-off-size excursions
        assert phi.min() > -1e-9 and phi.max() < 1
        return _np_taylor_D(phi)

    assert abs(float(J.detach()) - oJ(th0)) < 1e-10 * abs(float(J.detach()))
    assert float(J.detach()) > 0.01  # the droplet has deformed
    for q, h in [(0, 1e-6), (1, 1e-5), (4, 1e-6), (5, 1e-6)]:
        tp, tm = th0.copy(), th0.copy()
        tp[q] += h
        tm[q] -= h
        fd = (oJ(tp) - oJ(tm)) / (2 * h)
        assert abs(g[q] - fd) <= 2e-5 * abs(fd) + 1e-9, (q, g[q], fd)
    d = W.uniform(9, phi0.shape, -1.0, 1.0) * phi0 * (1 - phi0)
    h = 1e-6
    fd = (oJ(th0, phi0 + h * d) - oJ(th0, phi0 - h * d)) / (2 * h)
    ad = float((phi0_t.grad.numpy() * d).sum())
    assert abs(ad - fd) <= 2e-5 * abs(fd) + 1e-9, (ad, fd)
