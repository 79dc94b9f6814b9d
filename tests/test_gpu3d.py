"""GPU parity of the three-dimensional step (D3Q19 flow, D3Q7 phase field)
through the C ABI of include/lbm3_api.h, against the FP64 3-D oracle on the
same seeded inputs.

Tolerances (as for the 2-D path):
  * FP64 storage: max |GPU - oracle| <= 1e-12 on populations, phi*u, phi, u
    and p after 100 steps;
  * FP32 storage: <= 1e-5 on phi after 100 steps, 1e-6 on u;
  * FP16 storage (FP32 arithmetic): <= 2e-3 on phi after 100 steps, and the
    phase volume kept to 1e-6 relative (g_0 absorbs the FP16 rounding of the
    moving populations).
Grids span several CTA tiles in x and y, several z chunks, and ragged tails.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def L3():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_10899_gb300 import build
    build.build()
    from paper_2505_10899_gb300 import lbm3
    return lbm3


def md(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max())


def two_phase(nx, ny, nz, seed=5, **kw):
    case = W.base_case3(nx, ny, nz, sigma=1e-2, **kw)
    phi0 = W.tanh_ball(nx, ny, nz, 0.45 * nx, 0.55 * ny, 0.5 * nz, 0.3 * min(nx, ny, nz) + 1.5, 4.0)
    u0 = W.uniform(seed, (3, nz, ny, nx), -0.01, 0.01)
    return case, phi0, u0


def pair(L3, case, phi0, u0, nsteps, precision, tiling=None, state=None):
    o = oracle.Oracle3(case, phi0, u0) if state is None else oracle.Oracle3(case, state=state)
    s = L3.Sim3(case, phi0 if phi0 is not None else np.zeros((case["nz"], case["ny"], case["nx"])),
                u0, precision=precision)
    if tiling:
        s.set_tiling(*tiling)
    if state is not None:
        f, g, j, t = state
        s.set_state(f, g, j, t)
    o.step(nsteps)
    s.step(nsteps)
    return o, s


def check_all(o, s, tol_pop, tol_phi, tol_u, tol_p):
    f, g, j, t = s.get_state()
    assert t == o.t
    assert md(f, o.f) <= tol_pop
    assert md(g, o.g) <= tol_pop
    assert md(j, o.j) <= tol_pop
    phi, u, p = s.fields()
    ophi, ou, op = o.fields()
    assert md(phi, ophi) <= tol_phi
    assert md(u, ou) <= tol_u
    assert md(p, op) <= tol_p
    assert s.status() == 0


@pytest.mark.parametrize("var", ["equal_nu", "ratio3_var_tau"])
def test_fp64_parity_100_steps(L3, var):
    kw = dict(rho_l=1.0) if var == "equal_nu" else dict(rho_l=3.0, tau_f_l=0.7, tau_f_g=1.1)
    case, phi0, u0 = two_phase(40, 24, 20, **kw)
    o, s = pair(L3, case, phi0, u0, 100, "f64")
    check_all(o, s, TOL64, TOL64, TOL64, TOL64)


def test_fp64_parity_random_state_with_clip(L3):
    # phi outside [0, 1] exercises the clip of Eq. 37; random f, phi*u
    case = W.base_case3(37, 19, 11, sigma=1e-2, rho_l=10.0, tau_f_l=0.6, tau_f_g=1.0)
    state = (*W.random_state3(37, 19, 11, seed=77), 5)
    o, s = pair(L3, case, None, None, 7, "f64", state=state)
    check_all(o, s, TOL64, TOL64, TOL64, TOL64)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 9), (2, 3, 1), (33, 1, 5), (1, 17, 3),
                                   (5, 4, 3)])
def test_fp64_degenerate_grids(L3, shape):
    nx, ny, nz = shape
    case = W.base_case3(nx, ny, nz, sigma=1e-2, rho_l=2.0, tau_f_l=0.8)
    state = (*W.random_state3(nx, ny, nz, seed=11, phi_lo=0.2, phi_hi=0.8), 0)
    o, s = pair(L3, case, None, None, 20, "f64", state=state)
    check_all(o, s, TOL64, TOL64, TOL64, TOL64)


@pytest.mark.parametrize("tiling", [(32, 4, 8), (32, 16, 8), (64, 4, 13), (32, 8, 20)])
def test_fp64_every_tiling(L3, tiling):
    case, phi0, u0 = two_phase(70, 21, 20, rho_l=3.0, tau_f_l=0.7)
    o, s = pair(L3, case, phi0, u0, 30, "f64", tiling=tiling)
    check_all(o, s, TOL64, TOL64, TOL64, TOL64)


def test_fp32_parity_100_steps(L3):
    case, phi0, u0 = two_phase(40, 24, 20, rho_l=3.0, tau_f_l=0.7)
    o, s = pair(L3, case, phi0, u0, 100, "f32")
    phi, u, p = s.fields()
    ophi, ou, op = o.fields()
    assert md(phi, ophi) <= 1e-5
    assert md(u, ou) <= 1e-6
    assert s.status() == 0


@pytest.mark.parametrize("variant,tiling", [(2, (32, 4, 8)), (2, (32, 8, 13)), (3, (64, 4, 8)),
                                            (3, (32, 4, 20))])
def test_fp32_async_copy_variants(L3, variant, tiling):
    # the cp.async kernel runs the same per-node arithmetic as the register
    # kernel: equal up to FMA contraction, and within the FP32 bar of the oracle
    case, phi0, u0 = two_phase(70, 21, 20, rho_l=3.0, tau_f_l=0.7)
    a = L3.Sim3(case, phi0, u0, precision="f32")
    a.set_tiling(*tiling)
    a.set_kernel(variant)
    assert a.kernel() == variant
    b = L3.Sim3(case, phi0, u0, precision="f32")
    b.set_tiling(*tiling)
    b.set_kernel(1)
    a.step(100)
    b.step(100)
    fa, fb = a.get_state(), b.get_state()
    for x, y in zip(fa[:3], fb[:3]):
        assert md(x, y) <= 2e-6
    o = oracle.Oracle3(case, phi0, u0).step(100)
    assert md(a.fields()[0], o.fields()[0]) <= 1e-5
    assert a.status() == 0


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("shape,tiling", [((40, 21, 20), (128, 4, 8)),
                                          ((200, 7, 15), (256, 2, 13)),
                                          ((8, 3, 5), (128, 4, 5))])
def test_bulk_row_variant(L3, prec, shape, tiling):
    # Whole-row bulk copies (variant 4): the same per-node arithmetic as the
    # register kernel, so equal to it up to FMA contraction, and within the
    # precision's bar of the oracle; ragged row blocks and z chunks, and a
    # box thinner than the rows a CTA touches (ny = 3 < 4 + 2, nz = 5).
    nx, ny, nz = shape
    case, phi0, u0 = two_phase(nx, ny, nz, rho_l=3.0, tau_f_l=0.7)
    a = L3.Sim3(case, phi0, u0, precision=prec)
    a.set_tiling(*tiling)
    assert a.kernel() == 4  # the tile selects the variant made for it
    b = L3.Sim3(case, phi0, u0, precision=prec)
    b.set_kernel(1)
    tr = a.track_volume(True)
    a.step(100)
    b.step(100)
    assert a.status() == 0 and b.status() == 0
    fa, fb = a.get_state(), b.get_state()
    tol = 2e-6 if prec == "f32" else 2e-3
    for x, y in zip(fa[:3], fb[:3]):
        assert md(x, y) <= tol
    o = oracle.Oracle3(case, phi0, u0).step(99)
    # tracked: the volume of the state entering the last step
    assert abs(float(tr.cpu().numpy()[0]) / o.volume()[0] - 1) < (1e-6 if prec == "f32" else 1e-5)
    o.step(1)
    assert md(a.fields()[0], o.fields()[0]) <= (1e-5 if prec == "f32" else 2e-3)


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("variant,shape,tiling", [(5, (64, 21, 20), (32, 8, 8)),
                                                  (5, (128, 10, 13), (64, 4, 8)),
                                                  (5, (192, 17, 9), (64, 4, 9)),
                                                  (5, (64, 3, 5), (32, 8, 5)),
                                                  (6, (128, 21, 20), (64, 4, 8)),
                                                  (6, (192, 9, 13), (64, 2, 8)),
                                                  (6, (128, 3, 5), (64, 2, 5))])
def test_strip_bulk_variant(L3, prec, variant, shape, tiling):
    # Strip-row bulk copies (variants 5 and 6, the second with two stages and
    # more CTAs per SM): the same per-node arithmetic as the
    # register kernel, so equal to it up to FMA contraction, and within the
    # precision's bar of the oracle.  Several strips with periodic wrap pieces
    # at x = 0 and x = nx, ragged row blocks and z chunks, and a box of two
    # strips thinner than the rows a CTA touches (ny = 3).
    nx, ny, nz = shape
    case, phi0, u0 = two_phase(nx, ny, nz, rho_l=3.0, tau_f_l=0.7)
    a = L3.Sim3(case, phi0, u0, precision=prec)
    a.set_tiling(*tiling)
    a.set_kernel(variant)
    assert a.kernel() == variant and a.tiling()[:3] == tiling
    b = L3.Sim3(case, phi0, u0, precision=prec)
    b.set_kernel(1)
    tr = a.track_volume(True)
    a.step(100)
    b.step(100)
    assert a.status() == 0 and b.status() == 0
    fa, fb = a.get_state(), b.get_state()
    tol = 2e-6 if prec == "f32" else 2e-3
    for x, y in zip(fa[:3], fb[:3]):
        assert md(x, y) <= tol
    o = oracle.Oracle3(case, phi0, u0).step(99)
    assert abs(float(tr.cpu().numpy()[0]) / o.volume()[0] - 1) < (1e-6 if prec == "f32" else 1e-5)
    o.step(1)
    assert md(a.fields()[0], o.fields()[0]) <= (1e-5 if prec == "f32" else 2e-3)


def test_strip_variant_rejected_where_unavailable(L3):
    case, phi0, u0 = two_phase(64, 8, 8)
    s = L3.Sim3(case, phi0, u0, precision="f64")
    with pytest.raises(L3.LbmError):
        s.set_kernel(5)
    case, phi0, u0 = two_phase(40, 8, 8)  # nx not a multiple of the strip width
    t = L3.Sim3(case, phi0, u0, precision="f16")
    with pytest.raises(L3.LbmError):
        t.set_kernel(5)
    t.set_kernel(0)
    case, phi0, u0 = two_phase(32, 8, 8)  # one strip: both pads would wrap
    t = L3.Sim3(case, phi0, u0, precision="f32")
    with pytest.raises(L3.LbmError):
        t.set_kernel(5)
    # automatic selection keeps a tile the register kernel runs, and leaves a
    # tile only the whole-row kernel runs for the default tile
    case, phi0, u0 = two_phase(128, 8, 8)
    u = L3.Sim3(case, phi0, u0, precision="f32")
    u.set_tiling(64, 4, 8)
    u.set_kernel(5)
    u.set_kernel(0)
    assert u.kernel() == 1 and u.tiling()[:2] == (64, 4)
    u.set_tiling(128, 4, 8)
    assert u.kernel() == 4
    u.set_kernel(0)
    assert u.kernel() == 1 and u.tiling()[:2] == (32, 8)


def test_bulk_row_variant_rejected_where_unavailable(L3):
    case, phi0, u0 = two_phase(40, 24, 20)
    s = L3.Sim3(case, phi0, u0, precision="f64")
    with pytest.raises(L3.LbmError):
        s.set_kernel(4)
    with pytest.raises(L3.LbmError):
        s.set_tiling(128, 4, 8)
    case, phi0, u0 = two_phase(44, 8, 8)  # FP16 rows of 88 bytes: not 16-byte multiples
    t = L3.Sim3(case, phi0, u0, precision="f16")
    with pytest.raises(L3.LbmError):
        t.set_kernel(4)
    case, phi0, u0 = two_phase(264, 4, 8)  # rows longer than 256
    t = L3.Sim3(case, phi0, u0, precision="f32")
    with pytest.raises(L3.LbmError):
        t.set_kernel(4)
    t.set_kernel(0)


def test_async_variant_rejected_where_unavailable(L3):
    case, phi0, u0 = two_phase(40, 24, 20)
    s = L3.Sim3(case, phi0, u0, precision="f64")
    with pytest.raises(L3.LbmError):
        s.set_kernel(2)
    t = L3.Sim3(case, phi0, u0, precision="f32")
    t.set_tiling(32, 16, 8)
    with pytest.raises(L3.LbmError):
        t.set_kernel(3)


def test_fp16_storage_parity_and_volume(L3):
    case, phi0, u0 = two_phase(40, 24, 20, rho_l=3.0, tau_f_l=0.7)
    o, s = pair(L3, case, phi0, u0, 100, "f16")
    phi, u, p = s.fields()
    ophi, ou, op = o.fields()
    assert md(phi, ophi) <= 2e-3
    assert abs(s.volume()[0] / phi0.sum() - 1) <= 1e-6
    assert s.status() == 0


def test_volume_regions_and_tracking(L3):
    case, phi0, u0 = two_phase(40, 24, 20, rho_l=3.0)
    s = L3.Sim3(case, phi0, u0, precision="f64")
    o = oracle.Oracle3(case, phi0, u0)
    lab = np.zeros((20, 24, 40), np.int8)
    lab[10:] = 1
    lab[:, :, :3] = -1
    s.set_regions(lab, 2)
    tr = s.track_volume(True)
    s.step(40)
    o.step(39)
    v_before_last = o.volume()[0]
    o.step(1)
    assert abs(float(tr.cpu().numpy()[0]) / v_before_last - 1) < 1e-13
    v = s.volume()
    ov = o.volume(lab, 2)
    assert np.abs(v / ov - 1).max() < 1e-13
    assert abs(v.sum() + o.phi()[:, :, :3].sum() - phi0.sum()) < 1e-10


def test_graph_replay_matches_direct_steps(L3):
    # 64-step graphs plus a remainder: same result as 130 single launches
    case, phi0, u0 = two_phase(40, 24, 20, rho_l=3.0)
    a = L3.Sim3(case, phi0, u0, precision="f32")
    b = L3.Sim3(case, phi0, u0, precision="f32")
    a.step(130)
    for _ in range(130):
        b.step(1)
    fa = a.get_state()
    fb = b.get_state()
    for x, y in zip(fa[:3], fb[:3]):
        assert np.array_equal(x, y)
    assert fa[3] == fb[3] == 130


def test_fp32_volume_drift_1e4_steps(L3):
    # phase volume over 10^4 steps stays within 1e-6 relative in FP32 storage
    n = 48
    case = W.base_case3(n, n, n, sigma=1e-3, rho_l=3.0)
    phi0 = W.tanh_ball(n, n, n, n / 2, n / 2, n / 2, 12.0, 4.0)
    s = L3.Sim3(case, phi0, None, precision="f32")
    v0 = s.volume()[0]
    s.step(10000)
    v1 = s.volume()[0]
    assert abs(v1 / v0 - 1) <= 1e-6
    assert s.status() == 0


def test_autotune_keeps_state(L3):
    case, phi0, u0 = two_phase(40, 24, 20, rho_l=3.0)
    s = L3.Sim3(case, phi0, u0, precision="f32")
    s.step(3)
    before = s.get_state()
    best = s.autotune(2)
    after = s.get_state()
    for x, y in zip(before[:3], after[:3]):
        assert np.array_equal(x, y)
    assert s.tiling()[:3] == (best["bx"], best["by"], best["zc"])
    assert s.kernel() == best["kernel"] in (1, 2, 3)
    s.step(5)
    o = oracle.Oracle3(case, phi0, u0).step(8)
    assert md(s.fields()[0], o.fields()[0]) <= 1e-5


def test_nonfinite_is_flagged(L3):
    case = W.base_case3(8, 8, 8)
    f, g, j = W.random_state3(8, 8, 8, seed=3)
    g[0, 2, 3, 4] = np.inf
    s = L3.Sim3(case, np.full((8, 8, 8), 0.5), None, precision="f32")
    s.set_state(f, g, j, 0)
    s.step(1)
    assert s.status() == -4
