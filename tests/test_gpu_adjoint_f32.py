"""Reverse mode in FP32 (FP32 states, adjoints and adjoint arithmetic; FP64
parameter accumulation), against the FP64 reverse mode.

Tolerances come from the arithmetic: one FP32 step rounds each of a few
hundred operations per node at 2^-24 = 6e-8, so one vector-Jacobian product
agrees with the FP64 one to ~1e-5 of its scale (bar 1e-4); over T steps the
FP32 forward trajectory itself moves away from the FP64 one (phi by ~1e-6
after 100 steps), and the gradient of a smooth objective follows it to
~1e-4 relative (bar 2e-3).  Recorded and recomputed FP32 states give the
same bits (the FP32 snapshot carries the low part of the g_0 float pair)."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("walls", [0, 1])
def test_fp32_vjp_matches_fp64_vjp(L, walls):
    import torch
    lbm, A = L
    nx, ny = 40, 28
    kw = dict(walls=1, u_top=0.01, u_bot=-0.02) if walls else {}
    case = W.base_case(nx, ny, sigma=5e-3, rho_l=3.0, tau_f_l=0.9, tau_f_g=0.9, **kw)
    f, g, j = W.random_state(nx, ny, seed=7, coupled=True, phi_lo=0.1, phi_hi=0.9)
    lam = W.uniform(11, (20, ny, nx), -1.0, 1.0)
    out = {}
    for prec in ("f64", "f32"):
        s = A.AdjointSim(case, np.full((ny, nx), 0.5), precision=prec)
        s.sim.set_state(0, f, g, j, 5)
        lam_t = torch.as_tensor(lam, dtype=s.dtype, device="cuda")
        grads = np.zeros(6)
        adj = s.vjp_step(lam_t, grads)
        out[prec] = (adj.double().cpu().numpy(), grads)
        s.close()
    a64, g64 = out["f64"]
    a32, g32 = out["f32"]
    assert np.abs(a32 - a64).max() <= 1e-4 * np.abs(a64).max()
    for q in (0, 1, 2, 3) + ((4, 5) if walls else ()):
        assert abs(g32[q] - g64[q]) <= 1e-4 * abs(g64[q]) + 1e-6 * np.abs(g64).max(), (q, g32, g64)


def test_fp32_multistep_gradient_matches_fp64(L):
    import torch
    lbm, A = L
    nx, ny, T = 48, 40, 100
    case = W.base_case(nx, ny, sigma=4e-3, tau_g=0.8, rho_l=2.0)
    phi0 = W.tanh_disc(nx, ny, 20.0, 19.0, 6.0, 4.0, periodic=True)
    phi0 = phi0 + 0.2 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, :] * phi0 * (1 - phi0)
    w = torch.as_tensor(W.uniform(3, (ny, nx), 0.0, 1.0), device="cuda")
    res = {}
    for prec in ("f64", "f32"):
        phi0_t = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
        th = torch.tensor([case["sigma"], case["tau_g"], case["lambda"], case["tau_f_l"]],
                          dtype=torch.float64, requires_grad=True)
        phiT = A.coupled_run(phi0_t, th, case, T, ckpt_every=16, precision=prec)
        (phiT * w).sum().backward()
        res[prec] = (th.grad.numpy().copy(), phi0_t.grad.numpy().copy())
    (t64, p64), (t32, p32) = res["f64"], res["f32"]
    for q in range(4):
        assert abs(t32[q] - t64[q]) <= 2e-3 * abs(t64[q]), (q, t32[q], t64[q])
    assert np.abs(p32 - p64).max() <= 2e-3 * np.abs(p64).max()


def test_fp32_recorded_and_recomputed_states_give_the_same_gradient(L):
    import torch
    lbm, A = L
    nx, ny, T = 36, 28, 23
    case = W.base_case(nx, ny, sigma=4e-3, rho_l=2.0, tau_f_l=0.9, tau_f_g=0.9)
    phi0 = W.tanh_disc(nx, ny, 17.3, 13.6, 6.0, 4.0, periodic=True)
    w = torch.as_tensor(W.uniform(4, (ny, nx), 0.0, 1.0), device="cuda")
    state_bytes = 21 * 4 * nx * ny
    out = {}
    for store in (0, 5 * state_bytes, T * state_bytes):
        phi0_t = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
        th = torch.tensor([case["sigma"], case["tau_g"], case["lambda"], case["tau_f_l"]],
                          dtype=torch.float64, requires_grad=True)
        phiT = A.coupled_run(phi0_t, th, case, T, ckpt_every=4, store_bytes=store,
                             precision="f32")
        (phiT * w).sum().backward()
        out[store] = (phiT.detach().cpu().numpy(), th.grad.numpy(), phi0_t.grad.numpy())
    ref = out[0]
    for store, (p, gt, gp) in out.items():
        assert np.array_equal(p, ref[0]), store
        assert np.array_equal(gt, ref[1]) and np.array_equal(gp, ref[2]), store
    # the snapshot of an FP32 handle restores the step bit for bit
    s = A.AdjointSim(case, phi0, precision="f32")
    s.step(7)
    S = s.snapshot()
    s.step(5)
    a = s.snapshot()
    s.restore(S, 7)
    s.step(5)
    assert torch.equal(a, s.snapshot())
    s.close()
