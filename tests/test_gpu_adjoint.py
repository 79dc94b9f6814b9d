"""Reverse mode of the coupled step (lbm_adjoint_step / lbm_adjoint_init).

(1) One step: the vector-Jacobian product equals the directional derivative
    of the GPU forward step by central differences, for the state and for
    (sigma, tau_g, lambda, tau_f), coupled and vortex flow.
(2) Many steps: gradients of J = sum(w * phi_T) with respect to sigma, tau_g,
    lambda, tau_f and phi0 (directional) through the torch.autograd.Function
    equal central differences of J computed with the FP64 CPU oracle, with
    the forward states recorded in device memory and with checkpoints and
    recomputation; every split between the two gives the same bits.
States stay inside (0, 1) so that the clip of Eq. 37 is not hit."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_10899_gb300 import build
    build.build()
    from paper_2505_10899_gb300 import adjoint, lbm
    return lbm, adjoint


def _rand(shape, seed, lo=-1.0, hi=1.0):
    import torch
    return torch.as_tensor(W.uniform(seed, shape, lo, hi), device="cuda")


def _one_step_out(A, case, state, t):
    s = A.AdjointSim(case, np.full((case["ny"], case["nx"]), 0.5))
    s.restore(state, t)
    s.step(1)
    out = s.snapshot()
    s.close()
    return out


@pytest.mark.parametrize("flow", ["coupled", "vortex"])
def test_adjoint_step_matches_fd(L, flow):
    import torch
    lbm, A = L
    nx, ny = 40, 28
    if flow == "coupled":
        case = W.base_case(nx, ny, sigma=5e-3, rho_l=4.0, tau_f_l=0.9, tau_f_g=0.9,
                           s_f=[1.2, 1.1, 0.9, 1, 1.3, 1, 0.8, 1, 1])
    else:
        case, _, _ = W.single_vortex(n=nx, W=3.0, U=0.02, T=64)
        case["ny"] = ny
    # random well-conditioned state in the pull layout, phi in (0.1, 0.9)
    f, g, j = W.random_state(nx, ny, seed=7, coupled=True, phi_lo=0.1, phi_hi=0.9)
    base = A.AdjointSim(case, np.full((ny, nx), 0.5))
    base.sim.set_state(0, f if flow == "coupled" else None, g, j, 5)
    S = base.snapshot()
    if flow != "coupled":
        S[:9] = 0
    lam_out = _rand((20, ny, nx), 11)
    delta = _rand((20, ny, nx), 12)
    if flow != "coupled":
        delta[:9] = 0
    grads = np.zeros(6)
    lam_in = base.vjp_step(lam_out, grads)
    assert grads[4] == 0.0 and grads[5] == 0.0  # no walls
    eps = 1e-6
    Sp = _one_step_out(A, case, S + eps * delta, 5)
    Sm = _one_step_out(A, case, S - eps * delta, 5)
    fd = float(((Sp - Sm) * lam_out).sum()) / (2 * eps)
    ad = float((lam_in * delta).sum())
    assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-9, (ad, fd)
    # parameters
    th0 = np.array([case["sigma"], case["tau_g"], case["lambda"], case["tau_f_l"]])
    for q, h in enumerate([1e-7, 1e-6, 1e-6, 1e-6]):
        if flow != "coupled" and q == 3:
            assert grads[3] == 0.0
            continue
        outs = []
        for sgn in (+1, -1):
            th = th0.copy()
            th[q] += sgn * h
            outs.append(_one_step_out(A, A.case_with(case, th), S, 5))
        fdq = float(((outs[0] - outs[1]) * lam_out).sum()) / (2 * h)
        assert abs(grads[q] - fdq) <= 1e-5 * abs(fdq) + 1e-7, (q, grads[q], fdq)
    base.close()


def _oracle_J(case, theta, phi0, w, nsteps, A):
    c = A.case_with(case, theta)
    o = oracle.Oracle(c, phi0).step(nsteps)
    return float((o.fields()[0] * w).sum())


@pytest.mark.parametrize("store_bytes", [None, 0], ids=["recorded", "recomputed"])
def test_multistep_gradient_vs_oracle_fd(L, store_bytes):
    import torch
    lbm, A = L
    nx, ny, T = 48, 40, 15
    case = W.base_case(nx, ny, sigma=4e-3, tau_g=0.8)
    # droplet small enough that phi stays inside (0, 1): no clip
    phi0 = W.tanh_disc(nx, ny, 20.0, 19.0, 5.0, 4.0, periodic=True)
    phi0 = phi0 + 0.2 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, :] * phi0 * (1 - phi0)
    assert phi0.max() < 0.999 and phi0.min() > 0
    w = W.uniform(3, (ny, nx), 0.0, 1.0)
    theta0 = np.array([case["sigma"], case["tau_g"], case["lambda"], case["tau_f_l"]])
    phi0_t = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
    theta_t = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    phiT = A.coupled_run(phi0_t, theta_t, case, T, ckpt_every=4, store_bytes=store_bytes)
    J = (phiT * torch.as_tensor(w, device=phiT.device)).sum()
    J.backward()
    g_theta = theta_t.grad.numpy()
    g_phi0 = phi0_t.grad.numpy()
    # forward value agrees with the oracle
    assert abs(float(J) - _oracle_J(case, theta0, phi0, w, T, A)) < 1e-10 * abs(float(J))
    # parameter gradients vs central differences of the oracle
    for q, h in enumerate([1e-6, 1e-5, 1e-5, 1e-5]):
        tp, tm = theta0.copy(), theta0.copy()
        tp[q] += h
        tm[q] -= h
        fd = (_oracle_J(case, tp, phi0, w, T, A) - _oracle_J(case, tm, phi0, w, T, A)) / (2 * h)
        assert abs(g_theta[q] - fd) <= 2e-5 * abs(fd) + 1e-9, (q, g_theta[q], fd)
    # initial-field gradient along a random direction
    d = W.uniform(9, (ny, nx), -1.0, 1.0) * phi0 * (1 - phi0)
    h = 1e-6
    fd = (_oracle_J(case, theta0, phi0 + h * d, w, T, A)
          - _oracle_J(case, theta0, phi0 - h * d, w, T, A)) / (2 * h)
    ad = float((g_phi0 * d).sum())
    assert abs(ad - fd) <= 2e-5 * abs(fd) + 1e-9, (ad, fd)


def test_adjoint_step_from_snapshot_equals_step_on_handle(L):
    # lbm_adjoint_step_from on a snapshot of S_t gives the bits of
    # lbm_adjoint_step with S_t in the handle, parameter derivatives included
    import torch
    lbm, A = L
    nx, ny = 40, 24
    case = W.base_case(nx, ny, walls=1, u_top=0.01, u_bot=-0.02, sigma=5e-3, rho_l=3.0,
                       tau_f_l=0.8, tau_f_g=0.8)
    f, g, j = W.random_state(nx, ny, seed=23, coupled=True, phi_lo=0.1, phi_hi=0.9)
    s = A.AdjointSim(case, np.full((ny, nx), 0.5))
    s.sim.set_state(0, f, g, j, 7)
    S = s.snapshot()
    lam = _rand((20, ny, nx), 31)
    g1, g2 = np.zeros(6), np.zeros(6)
    a1 = s.vjp_step(lam, g1)
    s.step(3)  # the handle's own state no longer matters
    a2 = s.vjp_step_from(S, 7, lam)
    s.take_grads(g2)
    assert torch.equal(a1, a2)
    assert np.array_equal(g1, g2) and np.abs(g1).max() > 0
    with pytest.raises(lbm.LbmError):
        s.vjp_step_from(S, 7, lam, lam)
    with pytest.raises(lbm.LbmError):
        s.vjp_step_from(S, 7, lam, S)
    s.close()


def test_recorded_and_recomputed_states_give_the_same_gradient(L):
    import torch
    lbm, A = L
    nx, ny, T = 36, 28, 23
    case = W.base_case(nx, ny, sigma=4e-3, rho_l=2.0, tau_f_l=0.9, tau_f_g=0.9)
    phi0 = W.tanh_disc(nx, ny, 17.3, 13.6, 6.0, 4.0, periodic=True)
    w = torch.as_tensor(W.uniform(4, (ny, nx), 0.0, 1.0), device="cuda")
    state_bytes = 20 * 8 * nx * ny
    out = {}
    for store in (0, 5 * state_bytes, T * state_bytes, None):
        phi0_t = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
        th = torch.tensor([case["sigma"], case["tau_g"], case["lambda"], case["tau_f_l"]],
                          dtype=torch.float64, requires_grad=True)
        phiT = A.coupled_run(phi0_t, th, case, T, ckpt_every=4, store_bytes=store)
        (phiT * w).sum().backward()
        out[store] = (phiT.detach().cpu().numpy(), th.grad.numpy(), phi0_t.grad.numpy())
    ref = out[0]
    for store, (p, gt, gp) in out.items():
        assert np.array_equal(p, ref[0]), store
        assert np.array_equal(gt, ref[1]) and np.array_equal(gp, ref[2]), store


def test_small_droplet_volume_gradient_vs_central_differences(L):
    # Volume objective: V = phase volume inside the disc of radius R + W = 10
    # around the small droplet of Sec. 4.1 (two droplets as printed, 128 x 64),
    # after 2000 steps of the classical model (lambda = 0), where the droplet
    # loses volume to the bulk.  dV/d(lambda, sigma) through the reverse mode
    # against central differences of GPU FP64 forward runs.  Turning on the
    # sharpening flux keeps volume in the droplet: dV/dlambda > 0.
    import torch
    lbm, A = L
    case, phi0, u0, _, _ = W.two_droplets(lam=0.0)
    ny, nx = phi0.shape
    yy, xx = np.mgrid[0:ny, 0:nx]
    disc = (((xx - 96.0) ** 2 + (yy - 32.0) ** 2) < 10.0 ** 2).astype(np.int8)
    T = 2000
    th0 = np.array([case["sigma"], case["tau_g"], case["lambda"], case["tau_f_l"]])
    th_t = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    phiT = A.coupled_run(torch.tensor(phi0), th_t, case, T, ckpt_every=64, u0=u0)
    V = A.region_volume(phiT, disc, 1)
    V.backward()
    g = th_t.grad.numpy()

    def V_of(th):
        s = lbm.Sim(A.case_with(case, th), phi0, u0, precision="f64")
        s.step(T)
        phi = s.fields(0)[0]
        s.close()
        return float((phi * disc).sum())

    assert abs(V_of(th0) - float(V.detach())) < 1e-10
    for q, h in ((2, 1e-4), (0, 1e-3 * th0[0])):  # lambda, sigma
        tp, tm = th0.copy(), th0.copy()
        tp[q] += h
        tm[q] -= h
        fd = (V_of(tp) - V_of(tm)) / (2 * h)
        assert abs(g[q] - fd) <= 1e-4 * abs(fd), (q, g[q], fd)
    assert g[2] > 0
