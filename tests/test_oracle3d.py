"""Pins of the 3-D oracle (D3Q19 flow, D3Q7 phase field, SRT limit).

The paper fixes the method in two dimensions; its three-dimensional form here
is the single-relaxation-time limit (Sec. 3.1, all MRT rates equal) of
Eqs. 20-37 written on the textbook D3Q19 and D3Q7 lattices.  Each test checks
a fact that the lattices, the Chapman-Enskog limits of Eqs. 18 and 17, or
symmetry fix independently of the oracle's code:
  * the velocity sets and weights, their isotropy, and that D3Q19 summed over
    c_z is the D2Q9 lattice of Eq. 19;
  * the moments of f_eq, F_i, g_eq and G_i (Eqs. 21-23, 31-32);
  * the stencils of Sec. 3.2 against their plane-wave symbols;
  * conservation of sum(phi), fixed points, equivariance under the cube's
    symmetries;
  * the shear-wave viscosity (Eq. 27), the phase-field mobility (Eq. 34 with
    c_s^2 = 1/4), pure advection, a steady flat interface and Laplace's law
    dp = 2 sigma / R for a sphere.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads as W

CS2F, CS2G = 1.0 / 3.0, 0.25


def _rng(seed):
    return np.random.default_rng(seed)


def test_velocity_sets(lattice_golden):
    c19, w19, c7, w7 = oracle.lattices3()
    # D3Q19: the rest vector, the 6 axis vectors, the 12 face diagonals
    want19 = {(0, 0, 0)}
    for a in range(3):
        for s in (1, -1):
            e = [0, 0, 0]
            e[a] = s
            want19.add(tuple(e))
    for a, b in itertools.combinations(range(3), 2):
        for sa, sb in itertools.product((1, -1), repeat=2):
            e = [0, 0, 0]
            e[a], e[b] = sa, sb
            want19.add(tuple(e))
    assert {tuple(v) for v in c19} == want19 and len(c19) == 19
    assert c7.tolist()[0] == [0, 0, 0]
    assert {tuple(v) for v in c7} == {v for v in want19 if sum(map(abs, v)) <= 1}
    # weights by speed class (textbook D3Q19: 1/3, 1/18, 1/36; D3Q7 here 1/4, 1/8)
    sp19 = (c19 ** 2).sum(1)
    assert np.allclose(w19, np.select([sp19 == 0, sp19 == 1, sp19 == 2], [1 / 3, 1 / 18, 1 / 36]),
                       rtol=0, atol=1e-16)
    assert np.allclose(w7, np.where((c7 ** 2).sum(1) == 0, 0.25, 0.125), rtol=0, atol=1e-16)
    # projecting D3Q19 on the xy-plane (summing over c_z) gives D2Q9, Eq. 19
    c2, w2 = lattice_golden
    for (cx, cy), w in zip(c2.astype(int), w2):
        sel = (c19[:, 0] == cx) & (c19[:, 1] == cy)
        assert abs(w19[sel].sum() - w) < 1e-16


def test_isotropy():
    c19, w19, c7, w7 = oracle.lattices3()
    d = np.eye(3)
    for c, w, cs2 in ((c19, w19, CS2F), (c7, w7, CS2G)):
        assert abs(w.sum() - 1) < 1e-15
        assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-16
        assert np.abs(np.einsum("i,ia,ib->ab", w, c, c) - cs2 * d).max() < 4e-16
        assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-16
    four = np.einsum("i,ia,ib,ic,id->abcd", w19, c19, c19, c19, c19)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) * CS2F ** 2
    assert np.abs(four - iso).max() < 4e-16


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_feq_moments(seed):
    r = _rng(seed)
    c19, _, _, _ = oracle.lattices3()
    p, rho, u = r.uniform(-1e-2, 1e-2), r.uniform(0.5, 10), r.uniform(-0.05, 0.05, 3)
    f = oracle.feq3(p, rho, u)
    assert abs(f.sum()) < 1e-15 * rho
    assert np.abs(c19.T @ f - rho * u).max() < 1e-15 * rho
    P = np.einsum("i,ia,ib->ab", f, c19, c19)
    assert np.abs(P - (p * np.eye(3) + rho * np.outer(u, u))).max() < 1e-15 * rho


@pytest.mark.parametrize("seed", [4, 5])
def test_force_moments(seed):
    r = _rng(seed)
    c19, _, _, _ = oracle.lattices3()
    u, F, gr = r.uniform(-0.05, 0.05, 3), r.uniform(-1e-3, 1e-3, 3), r.uniform(-1, 1, 3)
    Fi = oracle.force3(u, F, gr)
    assert abs(Fi.sum() - u @ gr) < 1e-16
    assert np.abs(c19.T @ Fi - F).max() < 1e-16
    P = np.einsum("i,ia,ib->ab", Fi, c19, c19)
    want = CS2F * ((u @ gr) * np.eye(3) + np.outer(u, gr) + np.outer(gr, u))
    assert np.abs(P - want).max() < 1e-16


@pytest.mark.parametrize("seed", [6, 7])
def test_geq_moments(seed):
    r = _rng(seed)
    _, _, c7, _ = oracle.lattices3()
    phi, mu, lam, u = r.uniform(0, 1), r.uniform(-1e-3, 1e-3), 0.5, r.uniform(-0.05, 0.05, 3)
    g = oracle.geq3(phi, mu, lam, u)
    assert abs(g.sum() - phi) < 1e-16
    assert np.abs(c7.T @ g - phi * u).max() < 1e-17
    P = np.einsum("i,ia,ib->ab", g, c7, c7)
    assert np.abs(P - CS2G * (mu + lam * phi) * np.eye(3)).max() < 1e-16


@pytest.mark.parametrize("seed", [8, 9])
def test_gsrc_moments(seed):
    r = _rng(seed)
    _, _, c7, _ = oracle.lattices3()
    dJ, lam, Wd, psi = r.uniform(-1e-4, 1e-4, 3), 0.5, 4.0, r.uniform(-3, 3)
    n = r.normal(size=3)
    n /= np.linalg.norm(n)
    G = oracle.gsrc3(dJ, lam, Wd, psi, n)
    assert abs(G.sum()) < 1e-18
    # first moment: c_s^2 times the braced vector of Eq. 32
    sharp = (lam / Wd) * (1 - np.tanh(2 * psi / Wd) ** 2)
    assert np.abs(c7.T @ G - (dJ + CS2G * sharp * n)).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ib->ab", G, c7, c7)).max() < 1e-18


def _plane_wave(shape, k, theta=0.3):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = k[0] * x + k[1] * y + k[2] * z + theta
    return np.cos(ph), np.sin(ph)


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 1), (3, -1, 2)])
def test_stencil_plane_wave_symbols(m):
    shape = (12, 10, 16)
    k = 2 * np.pi * np.array([m[0] / shape[2], m[1] / shape[1], m[2] / shape[0]])
    cos, sin = _plane_wave(shape, k)
    gx, gy, gz, lap = oracle.stencil3(cos)
    ck, sk = np.cos(k), np.sin(k)
    # symbols of the D3Q19 weights (1/18 axis, 1/36 face diagonals) / c_s^2
    S = [sk[a] * (1 + ck[(a + 1) % 3] + ck[(a + 2) % 3]) / 3 for a in range(3)]
    L = (2 / 3) * (ck.sum() + ck[0] * ck[1] + ck[0] * ck[2] + ck[1] * ck[2] - 6)
    for g, s in zip((gx, gy, gz), S):
        assert np.abs(g + s * sin).max() < 1e-14
    assert np.abs(lap - L * cos).max() < 1e-14


def test_stencil_second_order():
    errs = []
    for n in (16, 32):
        k = 2 * np.pi / n * np.array([1.0, 1.0, 1.0])
        cos, sin = _plane_wave((n, n, n), k)
        gx, _, _, lap = oracle.stencil3(cos)
        errs.append((np.abs(gx + k[0] * sin).max() / k[0],
                     np.abs(lap + 3 * k[0] ** 2 * cos).max() / (3 * k[0] ** 2)))
    for a, b in zip(*errs):
        assert 3.5 < a / b < 4.5


def test_init_moments():
    r = _rng(11)
    case = W.base_case3(5, 4, 3, rho_l=3.0)
    phi0 = r.uniform(0, 1, (3, 4, 5))
    u0 = r.uniform(-0.02, 0.02, (3, 3, 4, 5))
    o = oracle.Oracle3(case, phi0, u0)
    c19, _, _, _ = oracle.lattices3()
    rho = 1.0 + 2.0 * phi0
    assert np.abs(o.g.sum(0) - phi0).max() < 1e-15
    assert np.abs(o.f.sum(0)).max() < 1e-15
    assert np.abs(np.einsum("ia,izyx->azyx", c19, o.f) - rho * u0).max() < 1e-15
    assert np.abs(o.j - phi0 * u0).max() == 0.0


def test_global_phi_conserved():
    case = W.base_case3(12, 10, 14, sigma=1e-2, rho_l=5.0, tau_f_l=0.7)
    phi0 = W.tanh_ball(12, 10, 14, 6, 5, 7, 3.5, 4.0) + 1e-3 * W.uniform(3, (14, 10, 12), -1, 1)
    o = oracle.Oracle3(case, phi0)
    v0 = o.volume()[0]
    o.step(200)
    assert np.isfinite(o.f).all()
    assert abs(o.volume()[0] / v0 - 1) < 1e-13


def test_uniform_translation_is_fixed_point():
    case = W.base_case3(4, 5, 3, sigma=1e-2, rho_l=2.0)
    phi0 = np.full((3, 5, 4), 0.4)
    u0 = np.zeros((3, 3, 5, 4))
    u0[0], u0[1], u0[2] = 0.03, -0.02, 0.01
    o = oracle.Oracle3(case, phi0, u0)
    f0, g0 = o.f.copy(), o.g.copy()
    o.step(20)
    phi, u, p = o.fields()
    assert np.abs(p).max() < 1e-15
    assert np.abs(u - u0).max() < 1e-15
    assert np.abs(o.f - f0).max() < 1e-15 and np.abs(o.g - g0).max() < 1e-15


def _run(case, phi0, u0, n):
    o = oracle.Oracle3(case, phi0, u0).step(n)
    return o.fields()


def test_cube_symmetry_equivariance():
    # A cyclic permutation of the axes and a mirror x -> -x map solutions onto
    # solutions: any axis-specific slip (a sign, a weight, an index) breaks it.
    n = 8
    r = _rng(21)
    case = W.base_case3(n, n, n, sigma=1e-2, rho_l=4.0, tau_f_l=0.7)
    phi0 = W.tanh_ball(n, n, n, 3.3, 4.1, 4.6, 2.6, 3.0)
    u0 = r.uniform(-0.01, 0.01, (3, n, n, n))
    phi, u, p = _run(case, phi0, u0, 30)
    # axes of arrays: [z][y][x]; new x = old y, new y = old z, new z = old x
    perm = lambda a: np.transpose(a, (2, 0, 1))
    phi_c, u_c, p_c = _run(case, perm(phi0), np.stack([perm(u0[1]), perm(u0[2]), perm(u0[0])]), 30)
    assert np.abs(phi_c - perm(phi)).max() < 1e-13
    assert np.abs(p_c - perm(p)).max() < 1e-15
    for a, b in ((0, 1), (1, 2), (2, 0)):
        assert np.abs(u_c[a] - perm(u[b])).max() < 1e-15
    # mirror in x about a node: index i -> (-i) mod n
    mir = lambda a: np.roll(a[..., ::-1], 1, axis=-1)
    phi_m, u_m, p_m = _run(case, mir(phi0), np.stack([-mir(u0[0]), mir(u0[1]), mir(u0[2])]), 30)
    assert np.abs(phi_m - mir(phi)).max() < 1e-13
    assert np.abs(u_m[0] + mir(u[0])).max() < 1e-15
    assert np.abs(u_m[2] - mir(u[2])).max() < 1e-15


def test_translation_equivariance():
    n = 6
    case = W.base_case3(n, n + 1, n + 2, sigma=1e-2, rho_l=2.0)
    phi0 = W.tanh_ball(n, n + 1, n + 2, 2.0, 3.0, 4.0, 2.0, 3.0)
    phi, u, p = _run(case, phi0, None, 15)
    sh = (2, -3, 1)
    phi_s, u_s, p_s = _run(case, np.roll(phi0, sh, axis=(0, 1, 2)), None, 15)
    assert np.abs(phi_s - np.roll(phi, sh, axis=(0, 1, 2))).max() < 1e-14
    assert np.abs(u_s - np.roll(u, sh, axis=(1, 2, 3))).max() < 1e-16


@pytest.mark.parametrize("tau,phase", [(0.7, 1.0), (1.3, 0.0)])
def test_shear_wave_viscosity(tau, phase):
    # Bulk of one fluid (phi = 1 liquid, phi = 0 gas), density ratio 3 and the
    # other fluid's tau_f different: the wave decays at nu = c_s^2 (tau_f - 1/2)
    # of that fluid (Eq. 27 with mu and rho of the bulk).
    n, U = 48, 1e-3
    other = 0.9
    tl, tg = (tau, other) if phase == 1.0 else (other, tau)
    case = W.base_case3(2, 2, n, sigma=0.0, rho_l=3.0, tau_f_l=tl, tau_f_g=tg,
                        **{"lambda": 0.0})
    z = np.arange(n)[:, None, None] * np.ones((1, 2, 2))
    u0 = np.zeros((3, n, 2, 2))
    u0[0] = U * np.sin(2 * np.pi * z / n)
    o = oracle.Oracle3(case, np.full((n, 2, 2), phase), u0)
    amps = []
    for t in (100, 700):
        o.step(t - o.t)
        ux = o.fields()[1][0, :, 0, 0]
        amps.append((ux * np.sin(2 * np.pi * np.arange(n) / n)).sum() * 2 / n)
    k = 2 * np.pi / n
    nu = -np.log(amps[1] / amps[0]) / (600 * k * k)
    assert abs(nu / ((tau - 0.5) / 3.0) - 1.0) < 5e-3


@pytest.mark.parametrize("axis", [0, 2])
def test_phase_mobility(axis):
    # lambda = 0, small amplitude about phi = 0: Eq. 3 linearises to
    # d_t phi = M lap(2 beta phi - kappa lap phi), M = c_s^2 (tau_g - 1/2)
    # with c_s^2 = 1/4 on D3Q7 (Eq. 34).  Mode decay rate M k^2 (2 beta + kappa k^2).
    n, tau, sigma, Wd = 48, 0.8, 1e-2, 4.0
    shape = [2, 2, 2]
    shape[axis] = n
    case = W.base_case3(shape[2], shape[1], shape[0], sigma=sigma, W=Wd, tau_g=tau,
                        **{"lambda": 0.0})
    s = np.arange(n).reshape([n if a == axis else 1 for a in range(3)])
    phi0 = 1e-4 * np.cos(2 * np.pi * s / n) * np.ones(shape)
    o = oracle.Oracle3(case, phi0)
    amps = []
    for t in (200, 2200):
        o.step(t - o.t)
        line = np.moveaxis(o.phi(), axis, 0)[:, 0, 0]
        amps.append((line * np.cos(2 * np.pi * np.arange(n) / n)).sum() * 2 / n)
    k = 2 * np.pi / n
    beta, kappa = 12 * sigma / Wd, 1.5 * sigma * Wd
    rate = -np.log(amps[1] / amps[0]) / 2000
    want = CS2G * (tau - 0.5) * k * k * (2 * beta + kappa * k * k)
    assert abs(rate / want - 1) < 5e-3


def test_pure_advection():
    # sigma = lambda = 0: Eq. 17 reduces to d_t phi + div(phi u) = 0
    n, N = 32, 600
    case = W.base_case3(n, 4, 4, sigma=0.0, **{"lambda": 0.0})
    x = np.arange(n)[None, None, :] * np.ones((4, 4, 1))
    phi0 = 0.5 + 0.3 * np.sin(2 * np.pi * x / n)
    u = (0.015, 0.01, -0.008)
    u0 = np.zeros((3, 4, 4, n))
    for a in range(3):
        u0[a] = u[a]
    o = oracle.Oracle3(case, phi0, u0).step(N)
    line = o.phi()[0, 0]
    c, c0 = np.fft.fft(line)[1], np.fft.fft(phi0[0, 0])[1]
    shift = -np.angle(c / c0) / (2 * np.pi / n)
    assert abs(shift / (u[0] * N) - 1.0) < 3e-3
    assert abs(abs(c) / abs(c0) - 1.0) < 1e-4


def test_flat_interface_is_steady():
    n, Wd = 64, 4.0
    case = W.base_case3(2, 2, n, sigma=1e-2, W=Wd, rho_l=3.0, tau_f_l=0.8)
    line = W.flat_slab(n, 1, n / 4, 3 * n / 4, Wd)[0]
    phi0 = np.ascontiguousarray(np.broadcast_to(line[:, None, None], (n, 2, 2)))
    o = oracle.Oracle3(case, phi0).step(2000)
    phi, u, p = o.fields()
    col = phi[:, 0, 0]
    i = int(n / 4) - 3
    while col[i + 1] < 0.5:
        i += 1
    pos = i + (0.5 - col[i]) / (col[i + 1] - col[i])
    assert abs(pos - n / 4) < 0.01
    assert np.abs(u).max() < 1e-6
    assert np.abs(phi - phi0).max() < 1e-2


@pytest.mark.slow
def test_laplace_law_sphere():
    # Eq. 18 with F_s = hbar grad phi: dp = 2 sigma / R for a sphere.
    n, R, sigma = 40, 10.0, 1e-2
    case = W.base_case3(n, n, n, sigma=sigma)
    o = oracle.Oracle3(case, W.tanh_ball(n, n, n, n / 2, n / 2, n / 2, R, case["W"]))
    o.step(1500)
    phi, u, p = o.fields()
    R_eff = (3 * phi.sum() / (4 * np.pi)) ** (1 / 3)
    dp = p[n // 2, n // 2, n // 2] - p[0, 0, 0]
    assert abs(dp / (2 * sigma / R_eff) - 1) < 0.05
    assert np.abs(u).max() < 5e-5


def test_dependency_radius_of_k_steps():
    # phi after k steps at a node depends on phi0 within 1 + 2k nodes: a
    # periodic block of phi0 reproduces the whole-box result exactly there
    # (the basis of the sampled full-size parity test)
    case, phi0 = W.rayleigh_plateau(24, 24, 32, R=6.0)
    k, half = 2, 8
    r = 1 + 2 * k
    phi = oracle.Oracle3(case, phi0).step(k).fields()[0]
    for (cz, cy, cx) in [(0, 12, 18), (20, 6, 12), (31, 23, 0)]:
        iz, iy, ix = (np.arange(c - half, c + half) % n for c, n in ((cz, 32), (cy, 24), (cx, 24)))
        bc = dict(case, nx=2 * half, ny=2 * half, nz=2 * half)
        o = oracle.Oracle3(bc, phi0[np.ix_(iz, iy, ix)]).step(k)
        inner = o.fields()[0][r:-r, r:-r, r:-r]
        assert np.array_equal(inner, phi[np.ix_(iz[r:-r], iy[r:-r], ix[r:-r])])
        # the bound is nearly tight: two nodes closer to the block face the
        # block result differs somewhere (one closer still agrees here, as the
        # initial Laplacian reaches phi only through the rounding of sum g_eq)
        e = r - 2
        edge = o.fields()[0][e:-e, e:-e, e:-e]
        assert not np.array_equal(edge, phi[np.ix_(iz[e:-e], iy[e:-e], ix[e:-e])])


def test_normal_vanishes_on_ridges_of_psi():
    # Eq. 17's unit normal grad(psi)/|grad(psi)| has no direction on a ridge
    # of psi (here the axis of the Eq. 45 thread, through nodes in x and y),
    # and a small |grad(psi)| amplifies perturbations by 1/|grad(psi)|.  With
    # n = 0 where |grad(psi)| < 0.1 the mirror-symmetric thread stays
    # symmetric to rounding with the sharpening flux on (lambda = 0.5) as
    # with it off, with the axis on nodes or between them.
    mz = lambda a: np.roll(a[::-1], 1, axis=0)   # z -> -z about a node
    for lam, side in ((0.0, 24), (0.5, 24), (0.5, 25)):
        case, phi0 = W.column_eq45(n=64, lam=lam, n_side=side)
        assert np.abs(phi0 - mz(phi0)).max() < 1e-15
        phi = oracle.Oracle3(case, phi0).step(40).fields()[0]
        assert np.abs(phi - mz(phi)).max() < 1e-13, (lam, side)
