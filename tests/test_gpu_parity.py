"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Tolerances:
  * FP64 path: max |GPU - oracle| <= 1e-12 on populations, phi*u and the
    macroscopic fields after 100 steps (both sides differ only in rounding
    order and FMA contraction);
  * FP32 path: <= 1e-5 on phi after 100 steps; u and p (values ~1e-4..1e-2)
    to 1e-6 absolute.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_PHI = 1e-5


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_10899_gb300 import build
    build.build()
    from paper_2505_10899_gb300 import lbm
    return lbm


def maxdiff(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max())


def run_pair(L, case, phi0, u0, nsteps, precision, state=None, variant=0):
    o = oracle.Oracle(case, phi0, u0) if state is None else oracle.Oracle(case, state=state)
    s = L.Sim(case, phi0 if phi0 is not None else np.zeros((case["ny"], case["nx"])),
              u0, precision=precision)
    s.set_kernel(variant)
    if state is not None:
        f, g, j, t = state
        s.set_state(0, f, g, j, t)
    o.step(nsteps)
    s.step(nsteps)
    return o, s


def compare_full(o, s, tol_pop, tol_phi, tol_u, tol_p):
    f, g, j, t = s.get_state(0)
    assert t == o.t
    if o.coupled:
        assert maxdiff(f, o.f) <= tol_pop
    assert maxdiff(g, o.g) <= tol_pop
    assert maxdiff(j, o.j) <= tol_pop
    phi, ux, uy, p = s.fields(0)
    ophi, oux, ouy, op = o.fields()
    assert maxdiff(phi, ophi) <= tol_phi
    assert maxdiff(ux, oux) <= tol_u and maxdiff(uy, ouy) <= tol_u
    assert maxdiff(p, op) <= tol_p
    assert s.status() == L_OK


L_OK = 0


VARIANTS = pytest.mark.parametrize("variant", [1, 2], ids=["regs", "tma"])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_full_row_and_edge_strips_match_oracle(L, prec):
    # Bulk-copy kernel, strips of 128 columns: rows no wider than a strip are
    # staged whole and read their periodic neighbours from the same copy;
    # wider rows split into strips whose edge strips copy the wrap columns.
    # Widths 4 (the narrowest), 12, 100, 128 (one strip) and 132, 260 (a
    # ragged last strip), several runs of rows each, 40 steps.
    for nx in (4, 12, 100, 128, 132, 260):
        ny = 26
        case = W.base_case(nx, ny, rho_l=3.0, tau_f_l=0.8, tau_f_g=1.1)
        phi0 = W.tanh_disc(nx, ny, 0.4 * nx, 11.0, min(0.3 * nx, 8.0), 3.0, periodic=True)
        phi0 = phi0 + W.uniform(nx, phi0.shape, -1e-3, 1e-3)
        u0 = np.zeros((2, ny, nx))
        u0[0], u0[1] = 0.013, -0.007
        o = oracle.Oracle(case, phi0, u0)
        s = L.Sim(case, phi0, u0, precision=prec)
        s.set_kernel(2)
        s.set_tiling(128, 8)
        o.step(40)
        s.step(40)
        if prec == "f64":
            compare_full(o, s, TOL64, TOL64, TOL64, TOL64)
        else:
            phi, ux, uy, p = s.fields(0)
            ophi, oux, ouy, op = o.fields()
            assert maxdiff(phi, ophi) <= TOL32_PHI, nx
            assert maxdiff(ux, oux) <= 1e-6 and maxdiff(uy, ouy) <= 1e-6, nx
        assert s.status() == L.LBM_OK
        s.close()


@VARIANTS
@pytest.mark.parametrize("lam", [0.5, 0.0])
def test_two_droplets_fp64(L, lam, variant):
    case, phi0, u0, lab, _ = W.two_droplets(noise=1e-3, lam=lam)
    o, s = run_pair(L, case, phi0, u0, 100, "f64", variant=variant)
    compare_full(o, s, TOL64, TOL64, TOL64, TOL64)
    s.set_regions(0, lab, 2)
    v = s.volume()
    assert np.abs(v / o.volume(lab, 2) - 1).max() < 1e-13


@VARIANTS
def test_two_droplets_fp32(L, variant):
    case, phi0, u0, lab, _ = W.two_droplets(noise=1e-3)
    o, s = run_pair(L, case, phi0, u0, 100, "f32", variant=variant)
    phi, ux, uy, p = s.fields(0)
    ophi, oux, ouy, op = o.fields()
    assert maxdiff(phi, ophi) <= TOL32_PHI
    assert maxdiff(ux, oux) <= 1e-6 and maxdiff(uy, ouy) <= 1e-6
    assert maxdiff(p, op) <= 1e-6
    s.set_regions(0, lab, 2)
    assert np.abs(s.volume() / o.volume(lab, 2) - 1).max() < 1e-6


@VARIANTS
def test_variable_density_random_state_fp64(L, variant):
    # ragged grid (several strips and a partial one), density ratio 10,
    # unequal viscosities, non-default free rates, random non-equilibrium state
    case = W.base_case(300, 70, sigma=5e-3, rho_l=10.0, rho_g=1.0, tau_f_l=0.7,
                       tau_f_g=1.2, s_f=[1.1, 1.3, 0.9, 1.0, 1.2, 1.0, 1.4, 1.0, 1.0],
                       s_g=[1.0, 1.2, 1.3, 1.0, 0.8, 1.0, 0.9, 1.1, 1.5])
    f, g, j = W.random_state(300, 70, seed=77)
    o, s = run_pair(L, case, None, None, 30, "f64", state=(f, g, j, 5), variant=variant)
    compare_full(o, s, TOL64, TOL64, TOL64, TOL64)


@VARIANTS
def test_translating_droplet_fp64(L, variant):
    case = W.base_case(96, 80, rho_l=3.0, tau_f_l=0.9, tau_f_g=0.9)
    phi0 = W.tanh_disc(96, 80, 40.0, 37.0, 15.0, 4.0, periodic=True)
    phi0 += W.uniform(5, phi0.shape, -1e-3, 1e-3)
    u0 = np.zeros((2, 80, 96))
    u0[0], u0[1] = 0.013, -0.008
    o, s = run_pair(L, case, phi0, u0, 100, "f64", variant=variant)
    compare_full(o, s, TOL64, TOL64, TOL64, TOL64)


@pytest.mark.parametrize("shape", [(1, 1), (3, 3), (1, 5), (4, 1), (2, 7), (33, 5), (129, 3),
                                   (5, 4), (3, 8), (7, 36), (2, 132)])
def test_degenerate_grids_fp64(L, shape):
    ny, nx = shape
    case = W.base_case(nx, ny, sigma=1e-2)
    f, g, j = W.random_state(nx, ny, seed=nx * 100 + ny)
    o, s = run_pair(L, case, None, None, 7, "f64", state=(f, g, j, 0))
    compare_full(o, s, TOL64, TOL64, TOL64, TOL64)
    if nx % 4 == 0:   # also through the bulk-copy kernel (periodic-wrap pieces)
        o, s = run_pair(L, case, None, None, 7, "f64", state=(f, g, j, 0), variant=2)
        compare_full(o, s, TOL64, TOL64, TOL64, TOL64)
        o, s = run_pair(L, case, None, None, 7, "f32", state=(f, g, j, 0), variant=2)
        assert maxdiff(s.fields(0)[0], o.fields()[0]) <= TOL32_PHI


@VARIANTS
def test_vortex_fp64(L, variant):
    case, phi0, _ = W.single_vortex(n=64, W=3.0, U=0.02, T=256)
    phi0 = phi0 + W.uniform(9, phi0.shape, -1e-3, 1e-3)
    o, s = run_pair(L, case, phi0, None, 100, "f64", variant=variant)
    compare_full(o, s, TOL64, TOL64, TOL64, 0.0)


@VARIANTS
def test_vortex_fp32(L, variant):
    case, phi0, _ = W.single_vortex(n=64, W=3.0, U=0.02, T=256)
    o, s = run_pair(L, case, phi0, None, 100, "f32", variant=variant)
    phi = s.fields(0)[0]
    assert maxdiff(phi, o.fields()[0]) <= TOL32_PHI


def test_graph_replay_and_parity_realignment_fp64(L):
    # 1 + 64 + 65 + 20 steps: a direct step, a graph replay, a realigning step
    # plus a replay, and a remainder; must equal 150 oracle steps.
    case, phi0, u0, _, _ = W.two_droplets(noise=1e-3)
    o = oracle.Oracle(case, phi0, u0).step(150)
    s = L.Sim(case, phi0, u0, precision="f64")
    for n in (1, 64, 65, 20):
        s.step(n)
    assert s.t == 150
    f, g, j, t = s.get_state(0)
    assert maxdiff(f, o.f) <= TOL64 and maxdiff(g, o.g) <= TOL64


@pytest.mark.parametrize("specs", [[(64, 64, 1.0), (96, 40, 4.0), (37, 51, 10.0)],
                                   [(64, 64, 1.0), (192, 40, 4.0), (36, 52, 10.0)]],
                         ids=["regs-only", "tma-eligible"])
def test_batch_of_uneven_cases_fp64(L, specs):
    cases, phis, us, oracles = [], [], [], []
    for k, (nx, ny, ratio) in enumerate(specs):
        c = W.base_case(nx, ny, rho_l=ratio, tau_f_l=0.8, tau_f_g=0.8)
        phi = W.tanh_disc(nx, ny, nx / 2, ny / 2, min(nx, ny) / 4, 4.0, periodic=True)
        phi += W.uniform(k, phi.shape, -1e-3, 1e-3)
        u = np.zeros((2, ny, nx))
        u[0] = 0.01 * (k + 1)
        cases.append(c), phis.append(phi), us.append(u)
        oracles.append(oracle.Oracle(c, phi, u).step(40))
    s = L.Sim(cases, phis, us, precision="f64")
    s.step(40)
    for k, o in enumerate(oracles):
        f, g, j, t = s.get_state(k)
        assert maxdiff(f, o.f) <= TOL64 and maxdiff(g, o.g) <= TOL64
        assert maxdiff(j, o.j) <= TOL64
    v = s.volume()
    for k, o in enumerate(oracles):
        assert abs(v[k] / o.volume()[0] - 1) < 1e-13


def _chain_batch():
    cases, phis, us = [], [], []
    for k, (nx, ny, ratio) in enumerate([(64, 64, 1.0), (96, 40, 4.0), (128, 52, 10.0),
                                         (32, 48, 2.0), (160, 36, 1.0)]):
        cases.append(W.base_case(nx, ny, rho_l=ratio, tau_f_l=0.8, tau_f_g=0.9))
        phi = W.tanh_disc(nx, ny, nx / 2, ny / 2, min(nx, ny) / 4, 4.0, periodic=True)
        phis.append(phi + W.uniform(20 + k, phi.shape, -1e-3, 1e-3))
        u = np.zeros((2, ny, nx))
        u[k % 2] = 0.01 * (k + 1) * (-1) ** k
        us.append(u)
    return cases, phis, us


def test_chains_do_not_change_results(L):
    # The chains split the cases into groups whose steps run as parallel
    # branches of the step graph; the kernels and their per-node arithmetic
    # are the same, so states and fused volumes are bitwise equal for any
    # chain count and any chunking of the steps into graphs.
    cases, phis, us = _chain_batch()
    ref = None
    for nch in (1, 2, 3, 4):
        s = L.Sim(cases, phis, us, precision="f32")
        s.set_tiling(32, 8)
        s.set_chains(nch)
        assert s.chains() == nch
        vol = s.track_volume(True)
        s.prepare(7)
        for n in (1, 5, 64, 7):  # graphs of both parities, the 64-step graph and a remainder
            s.step(n)
        assert s.t == 77 and s.status() == L.LBM_OK
        out = [s.get_state(k)[:3] for k in range(len(cases))] + [vol.cpu().numpy()]
        if ref is None:
            ref = out
        else:
            for a, b in zip(ref[:-1], out[:-1]):
                for x, y in zip(a, b):
                    assert np.array_equal(x, y)
            assert np.array_equal(ref[-1], out[-1])
        s.close()
    s = L.Sim(cases[:2], phis[:2], us[:2], precision="f32")
    s.set_chains(4)
    assert s.chains() == 2  # at most one chain per case
    with pytest.raises(L.LbmError):
        s.set_chains(5)


def test_whole_row_chains_fp32(L):
    # FP32, bulk-copy kernel, 128-column strips: cases whose row fits 64, 96,
    # 192 or 256 columns run whole-row strips in chains of their own (four
    # here); the others form the requested chains.  Every case matches the
    # oracle, the states agree with the same batch on 64-column strips (no
    # whole-row chains) up to FMA contraction, and the fused volumes with
    # lbm_volume.
    import torch
    widths = [(64, 40), (96, 36), (100, 30), (128, 33), (192, 28), (200, 26), (256, 24), (384, 20)]
    cases, phis, us = [], [], []
    for k, (nx, ny) in enumerate(widths):
        cases.append(W.base_case(nx, ny, rho_l=1.0 + k, tau_f_l=0.8, tau_f_g=0.9))
        phi = W.tanh_disc(nx, ny, 0.45 * nx, 0.5 * ny, min(nx, ny) / 4, 4.0, periodic=True)
        phis.append(phi + W.uniform(40 + k, phi.shape, -1e-3, 1e-3))
        u = np.zeros((2, ny, nx))
        u[k % 2] = 0.01 * (-1) ** k
        us.append(u)
    a = L.Sim(cases, phis, us, precision="f32")
    a.set_kernel(2)
    a.set_tiling(128, 16)
    a.set_chains(2)
    assert a.chains() == 2 and not a.row_chains()  # off by default
    a.set_row_chains(True)
    assert a.row_chains()
    assert a.chains() == 2 + 4  # widths 64, 96, 192 and 256 (the 200-wide row included)
    vol = a.track_volume(True)
    b = L.Sim(cases, phis, us, precision="f32")
    b.set_kernel(2)
    b.set_tiling(64, 16)
    assert b.chains() == 2
    a.step(50)
    b.step(50)
    assert a.status() == L.LBM_OK and b.status() == L.LBM_OK
    torch.cuda.synchronize()
    fused = vol.cpu().numpy().copy()
    for k, (c, p0, u0) in enumerate(zip(cases, phis, us)):
        o = oracle.Oracle(c, p0, u0).step(50)
        phi, ux, uy, p = a.fields(k)
        ophi, oux, ouy, op = o.fields()
        assert maxdiff(phi, ophi) <= TOL32_PHI, k
        assert maxdiff(ux, oux) <= 1e-6 and maxdiff(uy, ouy) <= 1e-6, k
        for x, y in zip(a.get_state(k)[:3], b.get_state(k)[:3]):
            assert maxdiff(x, y) <= 2e-6, k
    # the fused volumes of the last step: the state at t = 49, up to the low
    # part of g_0 that the fused FP32 sum leaves out
    r = L.Sim(cases, phis, us, precision="f32")
    r.set_kernel(2)
    r.set_tiling(128, 16)
    r.set_row_chains(True)
    r.step(49)
    assert np.abs(fused / r.volume() - 1).max() < 1e-7
    # the register kernel runs no whole-row chains; the request comes back
    # with the bulk-copy kernel
    r.set_kernel(1)
    assert not r.row_chains() and r.chains() == 2
    r.set_kernel(2)
    assert r.row_chains() and r.chains() == 6
    for s in (a, b, r):
        s.close()


def test_three_chains_match_oracle_fp64(L):
    cases, phis, us = _chain_batch()
    oracles = [oracle.Oracle(c, p, u).step(30) for c, p, u in zip(cases, phis, us)]
    s = L.Sim(cases, phis, us, precision="f64")
    s.set_chains(3)
    s.step(30)
    for k, o in enumerate(oracles):
        f, g, j, t = s.get_state(k)
        assert maxdiff(f, o.f) <= TOL64 and maxdiff(g, o.g) <= TOL64
        assert maxdiff(j, o.j) <= TOL64


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_init_from_device_and_pinned_inputs(L, prec):
    # lbm_init copies pageable arrays and reads device and page-locked arrays
    # in place: all three give the same state, bit for bit, after 5 steps
    import torch
    cases = W.batched_droplets(6, seed=99)
    fields = [W.case_fields(c) for c in cases]
    phis = [np.ascontiguousarray(p) for p, _ in fields]
    us = [np.ascontiguousarray(u) for _, u in fields]
    ref = L.Sim(cases, phis, us, precision=prec)
    dev = [torch.from_numpy(a).cuda() for a in phis + us]
    pin = [torch.from_numpy(a).pin_memory() for a in phis + us]
    n = len(cases)
    torch.cuda.synchronize()
    sims = [L.Sim(cases, [t.data_ptr() for t in ts[:n]], [t.data_ptr() for t in ts[n:]],
                  precision=prec) for ts in (dev, pin)]
    for s in [ref] + sims:
        s.step(5)
    for c in range(n):
        a = ref.get_state(c)
        for s in sims:
            b = s.get_state(c)
            for x, y in zip(a[:3], b[:3]):
                assert np.array_equal(x, y)
    assert all(s.status() == L_OK for s in [ref] + sims)


def test_checkpoint_roundtrip_bitwise(L):
    case, phi0, u0, _, _ = W.two_droplets(noise=1e-3)
    for prec in ("f32", "f64"):
        s = L.Sim(case, phi0, u0, precision=prec)
        s.step(37)
        blob = s.save()
        s.step(70)
        a = s.get_state(0)
        s.load(blob)
        assert s.t == 37
        s.step(70)
        b = s.get_state(0)
        for x, y in zip(a[:3], b[:3]):
            assert np.array_equal(x, y)


def test_nonfinite_is_reported(L):
    case = W.base_case(40, 20)
    f, g, j = W.random_state(40, 20, seed=3)
    g[0, 5, 7] = np.nan
    s = L.Sim(case, np.zeros((20, 40)), None, precision="f32")
    s.set_state(0, f, g, j, 0)
    s.step(2)
    assert s.status() == L.LBM_ERR_NONFINITE
    assert s.status() == L.LBM_OK  # flags were cleared


def test_zero_steps_and_bad_calls(L):
    case, phi0, u0, _, _ = W.two_droplets()
    s = L.Sim(case, phi0, u0, precision="f32")
    f0 = s.get_state(0)
    s.step(0)
    assert all(np.array_equal(a, b) for a, b in zip(f0[:3], s.get_state(0)[:3]))
    with pytest.raises(L.LbmError):
        s.step(-1)
    with pytest.raises(L.LbmError):
        L.lbm_fields(s.h, 1, (64, 128))   # no case 1: rejected by the ABI
    with pytest.raises(L.LbmError):
        s.set_regions(0, None, 9)


@VARIANTS
def test_tiling_does_not_change_results(L, variant):
    # per-node arithmetic is independent of the work tiling; separate kernel
    # instantiations may contract multiply-adds differently, so results agree
    # to FP32 rounding (values are O(1) for g, O(1e-3) for f)
    case = W.base_case(200, 90, rho_l=5.0, tau_f_l=0.7, tau_f_g=1.1)
    phi0 = W.tanh_disc(200, 90, 90.0, 40.0, 25.0, 4.0, periodic=True)
    u0 = np.zeros((2, 90, 200))
    u0[0] = 0.01
    ref = None
    for bx, rows in [(32, 2), (64, 17), (128, 64), (128, 3), (128, 2), (64, 2)]:
        for prec in ("f32",):
            s = L.Sim(case, phi0, u0, precision=prec)
            s.set_kernel(variant)
            s.set_tiling(bx, rows)
            assert s.tiling()[:2] == (bx, rows)
            s.step(33)
            st = s.get_state(0)
            if ref is None:
                ref = st
            else:
                for x, y in zip(ref[:3], st[:3]):
                    assert maxdiff(x, y) <= 2e-6
    with pytest.raises(L.LbmError):
        s.set_tiling(48, 8)


def test_fused_volume_tracking(L):
    import torch
    cases = [W.base_case(64, 48), W.base_case(100, 30, rho_l=3.0)]
    phis = [W.tanh_disc(64, 48, 30, 20, 10, 4.0, True), W.tanh_disc(100, 30, 50, 15, 8, 4.0, True)]
    s = L.Sim(cases, phis, None, precision="f64")
    vol = s.track_volume(True)
    s.step(10)
    torch.cuda.synchronize()
    # tracked value = volume of the state entering the last step (t = 9)
    s2 = L.Sim(cases, phis, None, precision="f64")
    s2.step(9)
    ref = s2.volume()
    assert np.array_equal(vol.cpu().numpy(), ref) or np.abs(vol.cpu().numpy() / ref - 1).max() < 1e-14
    with pytest.raises(L.LbmError):
        s.set_regions(0, np.zeros((48, 64), np.int8), 2)
    s.track_volume(False)
    s.set_regions(0, np.zeros((48, 64), np.int8), 2)
    with pytest.raises(L.LbmError):
        s.track_volume(True)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("host", [True, False])
def test_fused_volume_history(L, prec, host):
    # Slot t mod nslots holds the fused volumes of the state at time t, for
    # every step, whether the steps ran directly, from a graph, or in chains;
    # a page-locked host history is written by the kernels themselves.  The
    # values are those of plain tracking read after every single step, bit
    # for bit (same tiling, same chains, deterministic reductions).
    import torch
    cases, phis, us = _chain_batch()
    T = 13
    r = L.Sim(cases, phis, us, precision=prec)
    r.set_chains(2)
    vol = r.track_volume(True)
    rec = []
    for t in range(T):
        r.step(1)
        torch.cuda.synchronize()
        rec.append(vol.cpu().numpy().copy())
    r.close()
    for nslots in (16, 8):
        s = L.Sim(cases, phis, us, precision=prec)
        s.set_chains(2)
        hist = s.track_volume_history(nslots, host=host)
        for n in (2, 5, 5, 1):  # direct, first-seen chunk direct, then its graph, direct
            s.step(n)
        assert s.t == T
        torch.cuda.synchronize()
        got = hist.cpu().numpy()
        for t in range(max(0, T - nslots), T):
            assert np.array_equal(got[t % nslots], rec[t]), (nslots, t)
        if nslots > T:
            assert not got[T:].any()  # slots of later times untouched
        with pytest.raises(L.LbmError):
            L.lbm_track_volume_history(s.h, hist.data_ptr(), 0)
        pageable = np.zeros((nslots, len(cases)))
        with pytest.raises(L.LbmError):
            L.lbm_track_volume_history(s.h, pageable.ctypes.data, nslots)
        s.close()


def test_kernel_variants_agree_fp32(L):
    # both load paths feed the same per-node arithmetic: equal to FP32 rounding
    case = W.base_case(160, 72, rho_l=4.0, tau_f_l=0.8, tau_f_g=1.2)
    phi0 = W.tanh_disc(160, 72, 70.0, 30.0, 20.0, 4.0, periodic=True)
    u0 = np.zeros((2, 72, 160))
    u0[1] = -0.012
    out = []
    for variant in (1, 2):
        s = L.Sim(case, phi0, u0, precision="f32")
        s.set_kernel(variant)
        assert s.kernel() == variant
        s.step(50)
        out.append(s.get_state(0))
    for x, y in zip(out[0][:3], out[1][:3]):
        assert maxdiff(x, y) <= 2e-6
    s = L.Sim(W.base_case(30, 8), np.zeros((8, 30)), None, precision="f32")
    with pytest.raises(L.LbmError):
        s.set_kernel(2)          # 30 is not a multiple of 4


def test_autotune_keeps_state_and_parity(L):
    case, phi0, u0, _, _ = W.two_droplets(noise=1e-3)
    o = oracle.Oracle(case, phi0, u0).step(30)
    s = L.Sim(case, phi0, u0, precision="f64")
    s.step(10)
    before = s.get_state(0)
    best = s.autotune(1)
    assert best["kernel"] in (1, 2, 3) and best["bx"] in (32, 64, 128) and best["ms"] > 0
    assert s.tiling()[:2] == (best["bx"], best["rows"]) and s.kernel() == best["kernel"]
    after = s.get_state(0)
    assert after[3] == before[3] == 10
    for x, y in zip(before[:3], after[:3]):
        assert np.array_equal(x, y)
    s.step(20)
    f, g, j, t = s.get_state(0)
    assert maxdiff(f, o.f) <= TOL64 and maxdiff(g, o.g) <= TOL64 and maxdiff(j, o.j) <= TOL64


@pytest.mark.parametrize("ratio", [1.0, 3.0, 10.0])
def test_translating_droplet_fp32(L, ratio):
    # FP32 storage and arithmetic against the FP64 oracle: phi to 1e-5 after
    # 100 steps for a droplet moving at 0.02 lu/step, density ratio 1..10
    case = W.base_case(96, 80, rho_l=ratio, tau_f_l=1.0, tau_f_g=1.0)
    phi0 = W.tanh_disc(96, 80, 40.0, 37.0, 15.0, 4.0, periodic=True)
    u0 = np.zeros((2, 80, 96))
    u0[0], u0[1] = 0.016, -0.012
    o, s = run_pair(L, case, phi0, u0, 100, "f32")
    err = maxdiff(s.fields(0)[0], o.fields()[0])
    print(f"ratio {ratio}: max |phi_f32 - phi_oracle| = {err:.3e}")
    assert err <= TOL32_PHI


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_persistent_kernel(L, prec):
    # one cooperative launch for all steps, grid barrier between steps
    case, phi0, u0, _, _ = W.two_droplets(noise=1e-3)
    o = oracle.Oracle(case, phi0, u0).step(150)
    s = L.Sim(case, phi0, u0, precision=prec)
    s.set_kernel(3)
    assert s.kernel() == 3
    s.step(77)
    s.step(73)
    tol = TOL64 if prec == "f64" else TOL32_PHI
    assert maxdiff(s.fields(0)[0], o.fields()[0]) <= tol
    assert s.status() == L.LBM_OK
    # vortex flow: the step clock advances inside the launch
    vcase, vphi0, _ = W.single_vortex(n=64, W=3.0, U=0.02, T=256)
    vphi0 = vphi0 + W.uniform(9, vphi0.shape, -1e-3, 1e-3)
    ov = oracle.Oracle(vcase, vphi0).step(100)
    sv = L.Sim(vcase, vphi0, None, precision=prec)
    sv.set_kernel(3)
    sv.step(100)
    assert maxdiff(sv.fields(0)[0], ov.fields()[0]) <= tol
    # autotuning may pick the persistent kernel; it must not change the state
    before = sv.get_state(0)
    sv.autotune(1)
    after = sv.get_state(0)
    for x, y in zip(before[:3], after[:3]):
        assert np.array_equal(x, y)
