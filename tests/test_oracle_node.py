"""Per-node pins of the oracle: moments of the equilibria and sources
(Eqs. 21-23, 31-32), the level-set map (Eqs. 13-16, 37), the MRT collision
(Eqs. 25, 33) reducing to BGK for equal rates (Sec. 3.1, after Eq. 26).

Moments are taken with the golden lattice (typed from Eq. 19); the expected
values are the closed forms that the Chapman-Enskog recovery of Eqs. 17-18
requires, not the oracle's own formulas.
"""
import numpy as np
import pytest

import oracle
import workloads

CS2 = 1.0 / 3.0


def moments(c, v):
    return v.sum(), np.einsum("ia,i->a", c, v), np.einsum("ia,ib,i->ab", c, c, v)


def rand(seed, n, lo=-1.0, hi=1.0):
    return workloads.uniform(seed, (n,), lo, hi)


@pytest.mark.parametrize("seed", range(8))
def test_feq_moments(lattice_golden, seed):
    c, _ = lattice_golden
    p, ux, uy = rand(seed, 3, -0.05, 0.05)
    rho = rand(seed + 100, 1, 0.5, 10.0)[0]
    m0, m1, m2 = moments(c, oracle.feq(p, rho, ux, uy))
    u = np.array([ux, uy])
    assert abs(m0) < 1e-15                                 # sum f_eq = 0
    assert np.abs(m1 - rho * u).max() < 1e-15              # = rho u
    assert np.abs(m2 - (p * np.eye(2) + rho * np.outer(u, u))).max() < 1e-15


@pytest.mark.parametrize("seed", range(8))
def test_force_moments(lattice_golden, seed):
    c, _ = lattice_golden
    ux, uy, Fx, Fy, grx, gry = rand(seed, 6, -0.1, 0.1)
    m0, m1, m2 = moments(c, oracle.force(ux, uy, Fx, Fy, grx, gry))
    u, F, gr = np.array([ux, uy]), np.array([Fx, Fy]), np.array([grx, gry])
    assert abs(m0 - u @ gr) < 1e-16                        # u . grad rho
    assert np.abs(m1 - F).max() < 1e-16                    # the force
    ref = CS2 * ((u @ gr) * np.eye(2) + np.outer(u, gr) + np.outer(gr, u))
    assert np.abs(m2 - ref).max() < 1e-16


@pytest.mark.parametrize("seed", range(8))
def test_geq_moments(lattice_golden, seed):
    c, _ = lattice_golden
    phi, mu, ux, uy = rand(seed, 4, -0.1, 1.1)
    lam = 0.5
    m0, m1, m2 = moments(c, oracle.geq(phi, mu, lam, ux, uy))
    assert abs(m0 - phi) < 1e-15                           # conserves phi
    assert np.abs(m1 - phi * np.array([ux, uy])).max() < 1e-15
    # second moment c_s^2 (hbar + lambda phi) I gives M lap(hbar + lambda phi)
    assert np.abs(m2 - CS2 * (mu + lam * phi) * np.eye(2)).max() < 1e-15


@pytest.mark.parametrize("seed", range(8))
def test_gsrc_moments(lattice_golden, seed):
    c, _ = lattice_golden
    dJx, dJy = rand(seed, 2, -1e-3, 1e-3)
    phi = rand(seed + 7, 1, 1e-4, 1 - 1e-4)[0]
    W, lam = 4.0, 0.5
    ang = rand(seed + 9, 1, 0, 2 * np.pi)[0]
    n = np.array([np.cos(ang), np.sin(ang)])
    ps = oracle.psi(phi, W)
    m0, m1, m2 = moments(c, oracle.gsrc(dJx, dJy, lam, W, ps, n[0], n[1]))
    assert abs(m0) < 1e-17                                 # sum G_i = 0
    assert np.abs(m2).max() < 1e-17
    # first moment d_t(phi u) + c_s^2 (lambda/W) [1 - tanh^2(2 psi/W)] n, where by
    # Eqs. 13-15 applied to the regularised psi of Eq. 37 (a = phi + xi,
    # b = 1 - phi + xi) the bracket is 4ab/(a+b)^2, i.e. 4 phi (1 - phi) up to xi.
    a, b = phi + 1e-10, 1 - phi + 1e-10
    ref = np.array([dJx, dJy]) + CS2 * (lam / W) * 4 * a * b / (a + b) ** 2 * n
    assert np.abs(m1 - ref).max() < 1e-15
    ref15 = np.array([dJx, dJy]) + CS2 * (lam / W) * 4 * phi * (1 - phi) * n
    assert np.abs(m1 - ref15).max() < 1e-10


def test_psi_level_set_map():
    W, xi = 3.0, 1e-10
    assert oracle.psi(0.5, W, xi) == 0.0
    for phi in [2.0 ** -20, 2.0 ** -7, 0.1875, 0.375, 0.75, 1 - 2.0 ** -20]:  # 1-phi exact
        ps = oracle.psi(phi, W, xi)
        # antisymmetry about the interface and Eq. 13 (inverse map)
        assert abs(oracle.psi(1 - phi, W, xi) + ps) < 1e-12 * max(1, abs(ps))
        # (with xi the inverse returns (phi + xi)/(1 + 2 xi), within xi of phi)
        assert abs(0.5 * (1 + np.tanh(2 * ps / W)) - phi) < xi + 1e-15
    # clip of phi to [0,1] before Eq. 37; xi keeps psi finite at the bounds
    lo = 0.25 * W * np.log(xi / (1 + xi))
    for phi in [-0.3, -1e-12, 0.0]:
        assert oracle.psi(phi, W, xi) == pytest.approx(lo, rel=1e-15)
    for phi in [1.0, 1 + 1e-12, 1.7]:
        assert oracle.psi(phi, W, xi) == pytest.approx(-lo, rel=1e-15)
    # psi is the signed distance for the equilibrium profile (Eq. 4 / Eq. 14)
    for s in [-2.5, -0.7, 0.3, 1.9]:
        phi = 0.5 * (1 + np.tanh(2 * s / W))
        assert abs(oracle.psi(phi, W, 0.0) - s) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_mrt_equal_rates_is_bgk(seed):
    # All rates equal: M^-1 S M = s I, so Eq. 25 is the BGK update
    # f - s (f - feq) + (1 - s/2) F (the SRT limit stated after Eq. 26).
    f, fe, F = (rand(seed * 3 + k, 9) for k in range(3))
    s = rand(seed + 50, 1, 0.1, 1.9)[0]
    out = oracle.mrt(f, fe, F, np.full(9, s))
    assert np.abs(out - (f - s * (f - fe) + (1 - s / 2) * F)).max() < 1e-14


def test_mrt_rate_selects_moment():
    # With S = diag(e_k) only moment k relaxes: every other moment of f*
    # equals m + F-bar (forcing with weight 1) and moment k equals
    # m_eq + F-bar/2.  Checks each row of M and M^-1 separately.
    M, _ = oracle.matrices()
    f, fe, F = (rand(200 + k, 9) for k in range(3))
    for k in range(9):
        s = np.zeros(9)
        s[k] = 1.0
        ms = M @ oracle.mrt(f, fe, F, s)
        ref = M @ f + M @ F
        ref[k] = (M @ fe)[k] + 0.5 * (M @ F)[k]
        assert np.abs(ms - ref).max() < 1e-13
