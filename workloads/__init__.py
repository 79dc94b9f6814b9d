"""Seeded synthetic inputs shared by the oracle-side tests, the GPU tests and the bench.

This module holds no arithmetic of the lattice Boltzmann method itself: it builds
initial order-parameter fields (the tanh profiles of the paper's Sec. 4 set-ups),
region labels for the droplet volumes of Fig. 3b, seeded noise and random
population states, and the parameter dictionaries of the benchmark workloads.
Both the CPU oracle and the CUDA library receive exactly these arrays.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), a
counter-based generator, so a field is a pure function of (seed, index).
"""
from __future__ import annotations

import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive SplitMix64 outputs for the stream starting at ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, shape, lo=0.0, hi=1.0) -> np.ndarray:
    """Uniform doubles in [lo, hi) from the top 53 bits of SplitMix64."""
    n = int(np.prod(shape)) if len(shape) else 1
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (lo + (hi - lo) * u).reshape(shape)


# ---------------------------------------------------------------------------
# Initial fields (Sec. 4 set-ups)
# ---------------------------------------------------------------------------

def tanh_disc(nx, ny, cx, cy, R, W, periodic=False):
    """0.5[1 + tanh(2(R - d)/W)] on node coordinates (i, j); d Euclidean.

    With periodic=True the distance is taken to the nearest periodic image."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    dx = x - cx
    dy = y - cy
    if periodic:
        dx = dx - nx * np.round(dx / nx)
        dy = dy - ny * np.round(dy / ny)
    d = np.sqrt(dx * dx + dy * dy)
    return 0.5 * (1.0 + np.tanh(2.0 * (R - d) / W))


def droplets_field(nx, ny, drops, W, periodic=False):
    """Sum of tanh discs, as in the two-droplet set-up of Sec. 4.1."""
    phi = np.zeros((ny, nx))
    for (cx, cy, R) in drops:
        phi += tanh_disc(nx, ny, cx, cy, R, W, periodic)
    return phi


def nearest_surface_labels(nx, ny, drops, periodic=True):
    """Region of each node: the droplet whose surface is nearest (|x-c|-R minimal)."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    best = np.full((ny, nx), np.inf)
    lab = np.zeros((ny, nx), dtype=np.int8)
    for k, (cx, cy, R) in enumerate(drops):
        dx = x - cx
        dy = y - cy
        if periodic:
            dx = dx - nx * np.round(dx / nx)
            dy = dy - ny * np.round(dy / ny)
        s = np.sqrt(dx * dx + dy * dy) - R
        sel = s < best
        best = np.where(sel, s, best)
        lab = np.where(sel, np.int8(k), lab)
    return lab


def flat_slab(nx, ny, x1, x2, W):
    """A periodic slab phi(x) = 1 between x1 < x < x2 with two tanh interfaces."""
    x = np.arange(nx, dtype=np.float64)
    phi = 0.5 * (np.tanh(2.0 * (x - x1) / W) - np.tanh(2.0 * (x - x2) / W))
    return np.broadcast_to(phi[None, :], (ny, nx)).copy()


# ---------------------------------------------------------------------------
# Parameter sets
# ---------------------------------------------------------------------------

def base_case(nx, ny, **kw):
    c = dict(nx=int(nx), ny=int(ny), flow="coupled", W=4.0, sigma=1e-3,
             **{"lambda": 0.5}, xi=1e-10, tau_g=0.8, rho_l=1.0, rho_g=1.0,
             tau_f_l=1.0, tau_f_g=1.0, s_f=[1.0] * 9, s_g=[1.0] * 9,
             vortex_U=0.0, vortex_T=1.0)
    c.update(kw)
    return c


def two_droplets(noise=0.0, seed=12345, lam=0.5):
    """Two stationary droplets in gas: 128x64 periodic, R=12 at (40,32) and
    R=6 at (96,32), W=4, ratios 1:1, tau_g=0.8, tau_f=1.0, sigma=1e-3, at rest.
    ``noise`` adds a seeded uniform perturbation in [-noise, noise) to phi0."""
    nx, ny = 128, 64
    drops = [(40.0, 32.0, 12.0), (96.0, 32.0, 6.0)]
    case = base_case(nx, ny, **{"lambda": lam})
    phi0 = droplets_field(nx, ny, drops, case["W"])
    if noise:
        phi0 = phi0 + uniform(seed, (ny, nx), -noise, noise)
    labels = nearest_surface_labels(nx, ny, drops)
    return case, phi0, None, labels, drops


def single_vortex(n=256, W=3.0, U=0.02, T=16384, lam=0.5, sigma=0.01, tau_g=0.8):
    """Time-reversed single vortex, phase field only: n x n, disc of radius 0.15n
    at (0.5n, 0.75n), prescribed velocity with amplitude U and period T steps."""
    case = base_case(n, n, flow="vortex", W=W, sigma=sigma, tau_g=tau_g,
                     vortex_U=U, vortex_T=float(T), **{"lambda": lam})
    phi0 = tanh_disc(n, n, 0.5 * n, 0.75 * n, 0.15 * n, W)
    return case, phi0, None


def random_state(nx, ny, seed, coupled=True, phi_lo=-0.05, phi_hi=1.05):
    """A random but well-conditioned post-streaming state for parity tests:
    g_i = w_i * phi_i-ish positive pieces plus noise, f_i small, phi*u small."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    phi = uniform(seed, (ny, nx), phi_lo, phi_hi)
    g = w[:, None, None] * phi[None] + uniform(seed + 1, (9, ny, nx), -2e-3, 2e-3)
    f = uniform(seed + 2, (9, ny, nx), -2e-3, 2e-3) if coupled else None
    j = uniform(seed + 3, (2, ny, nx), -1e-3, 1e-3)
    return f, g, j


EDGES = (64, 96, 128, 192, 256, 384, 512)


def batched_droplets(ncases=512, seed=2026, W=4.0, sigma=1e-3, tau_g=0.8,
                     tau_f=1.0, lam=0.5):
    """Independent 2-D droplet cases: square edge uniform in EDGES, radius
    uniform in [0.05, 0.3]*edge, centred, translation speed uniform in
    [0, 0.02] in a uniform random direction, density ratio log-uniform in
    [1, 10] (rho_g = 1), equal kinematic viscosity (tau_f) in both phases."""
    r = uniform(seed, (ncases, 5))
    cases = []
    for c in range(ncases):
        edge = EDGES[min(int(r[c, 0] * len(EDGES)), len(EDGES) - 1)]
        R = (0.05 + 0.25 * r[c, 1]) * edge
        speed = 0.02 * r[c, 2]
        ang = 2.0 * math.pi * r[c, 3]
        ratio = math.exp(math.log(10.0) * r[c, 4])
        case = base_case(edge, edge, W=W, sigma=sigma, tau_g=tau_g,
                         rho_l=ratio, rho_g=1.0, tau_f_l=tau_f, tau_f_g=tau_f,
                         **{"lambda": lam})
        case["R"] = R
        case["u0"] = (speed * math.cos(ang), speed * math.sin(ang))
        cases.append(case)
    return cases


def case_fields(case):
    """phi0 and u0 (2, ny, nx) of a batched droplet case."""
    nx, ny = case["nx"], case["ny"]
    phi0 = tanh_disc(nx, ny, 0.5 * nx, 0.5 * ny, case["R"], case["W"], periodic=True)
    u0 = np.empty((2, ny, nx))
    u0[0] = case["u0"][0]
    u0[1] = case["u0"][1]
    return phi0, u0


# ---------------------------------------------------------------------------
# Three-dimensional inputs ([z][y][x] fields, x fastest).

def base_case3(nx, ny, nz, **kw):
    c = dict(nx=int(nx), ny=int(ny), nz=int(nz), W=4.0, sigma=1e-3,
             **{"lambda": 0.5}, xi=1e-10, tau_g=0.8, rho_l=1.0, rho_g=1.0,
             tau_f_l=1.0, tau_f_g=1.0)
    c.update(kw)
    return c


def tanh_ball(nx, ny, nz, cx, cy, cz, R, W):
    """0.5[1 + tanh(2(R - d)/W)], d the distance from (cx, cy, cz) to the
    nearest periodic image of node (i, j, k)."""
    def axis(n, c):
        d = np.arange(n, dtype=np.float64) - c
        return d - n * np.round(d / n)
    dx = axis(nx, cx)[None, None, :]
    dy = axis(ny, cy)[None, :, None]
    dz = axis(nz, cz)[:, None, None]
    d = np.sqrt(dx * dx + dy * dy + dz * dz)
    return 0.5 * (1.0 + np.tanh(2.0 * (R - d) / W))


def liquid_column(nx, ny, nz, R, W, eps=0.0, wavelength=None):
    """A liquid column along z, centred at (nx/2, ny/2), of radius
    R (1 + eps cos(2 pi z / wavelength)): the perturbed column of the
    Rayleigh-Plateau set-up (Sec. 4.3, here in three dimensions)."""
    wl = float(nz if wavelength is None else wavelength)
    dx = np.arange(nx, dtype=np.float64)[None, :] - 0.5 * nx
    dy = np.arange(ny, dtype=np.float64)[:, None] - 0.5 * ny
    r = np.sqrt(dx * dx + dy * dy)[None, :, :]
    Rz = R * (1.0 + eps * np.cos(2.0 * np.pi * np.arange(nz) / wl))[:, None, None]
    return 0.5 * (1.0 + np.tanh(2.0 * (Rz - r) / W))


def rayleigh_plateau(nx=256, ny=256, nz=1024, R=32.0, eps=0.05, W=4.0,
                     rho_ratio=10.0, sigma=1e-3, tau_g=0.8, tau_f=1.0, lam=0.5):
    """Periodic box with a sinusoidally perturbed liquid column, at rest.
    Returns (case, phi0)."""
    case = base_case3(nx, ny, nz, W=W, sigma=sigma, tau_g=tau_g, rho_l=rho_ratio,
                      rho_g=1.0, tau_f_l=tau_f, tau_f_g=tau_f, **{"lambda": lam})
    return case, liquid_column(nx, ny, nz, R, W, eps)


def random_state3(nx, ny, nz, seed, phi_lo=-0.05, phi_hi=1.05):
    """A random, well-conditioned post-streaming 3-D state for parity tests:
    g_i = (D3Q7 weight) * phi plus noise, f_i small, phi*u small."""
    w7 = np.array([0.25] + [0.125] * 6)
    phi = uniform(seed, (nz, ny, nx), phi_lo, phi_hi)
    g = w7[:, None, None, None] * phi[None] + uniform(seed + 1, (7, nz, ny, nx), -2e-3, 2e-3)
    f = uniform(seed + 2, (19, nz, ny, nx), -2e-3, 2e-3)
    j = uniform(seed + 3, (3, nz, ny, nx), -1e-3, 1e-3)
    return f, g, j


def shear_droplet(nx=512, ny=256, R=40.0, U=0.01, Ca=0.1, Re=0.1, W=4.0, tau_g=0.8,
                  lam=0.5, rho_ratio=1.0):
    """A droplet in the sheared cavity of Sec. 4.4 (the 512 x 256 channel by
    default): walls below
    y = 0 and above y = ny - 1 moving at -U and +U, droplet of radius R at the
    centre, equal kinematic viscosities.  Shear rate G = 2U/ny; the viscosity
    and surface tension follow from Re = G R^2 / nu and Ca = rho nu G R / sigma.
    The fluid starts on the linear Couette profile through the wall positions
    (walls half a node outside the end rows).  Returns (case, phi0, u0)."""
    G = 2.0 * U / ny
    nu = G * R * R / Re
    tau_f = 3.0 * nu + 0.5
    sigma = nu * G * R / Ca
    case = base_case(nx, ny, W=W, sigma=sigma, tau_g=tau_g, rho_l=rho_ratio, rho_g=1.0,
                     tau_f_l=tau_f, tau_f_g=tau_f, walls=1, u_top=U, u_bot=-U,
                     **{"lambda": lam})
    phi0 = tanh_disc(nx, ny, 0.5 * nx, 0.5 * ny - 0.5, R, W)
    u0 = np.zeros((2, ny, nx))
    u0[0] = -U + 2.0 * U * (np.arange(ny, dtype=np.float64)[:, None] + 0.5) / ny
    return case, phi0, u0


def coarse_sheared_droplet(lam=0.5, U=0.01, Ca=0.1, Re=0.1, W=4.0, tau_g=0.8):
    """The sheared droplet of Sec. 4.4 on the grid given there: a 128 x 64
    cavity between walls moving at -U (below) and +U (above), one droplet of
    radius 8 (Eq. 46) at the cavity centre, fluid on the Couette profile.  The
    wall speed, Ca, Re, W and tau_g are not given with the experiment; these
    defaults are the values chosen for it.  Returns (case, phi0, u0)."""
    return shear_droplet(nx=128, ny=64, R=8.0, U=U, Ca=Ca, Re=Re, W=W, tau_g=tau_g, lam=lam)


def film_eq45(nx=256, ny=128, a=0.15, amp=0.05, W=4.0, sigma=1e-3, tau_f=0.6, lam=0.5):
    """Eq. 45 on the two-dimensional grid as printed: the domain
    (0, 2 pi) x (0, pi) on nx x ny nodes (spacing pi / ny), a liquid layer of
    height a + amp cos(x) (in the domain's units) on a resting wall below
    y = 0, a resting wall above y = pi, fluid at rest.  Node (i, j) sits at
    x = i h, y = (j + 1/2) h, the walls half a node outside the end rows; W is
    in lattice units.  Returns (case, phi0)."""
    h = np.pi / ny
    x = np.arange(nx, dtype=np.float64)[None, :] * (2.0 * np.pi / nx)
    y = (np.arange(ny, dtype=np.float64)[:, None] + 0.5) * h
    phi0 = 0.5 * (1.0 + np.tanh(2.0 * (a - y + amp * np.cos(x)) / (W * h)))
    case = base_case(nx, ny, W=W, sigma=sigma, tau_f_l=tau_f, tau_f_g=tau_f, walls=1,
                     u_top=0.0, u_bot=0.0, **{"lambda": lam})
    return case, phi0


def column_eq45(n=256, a=0.15, amp=0.05, W=4.0, sigma=1e-3, tau_f=0.6, lam=0.5,
                tau_g=0.8, rho_ratio=1.0, n_side=None):
    """Eq. 45 read as a section through an axisymmetric liquid thread (y the
    distance from the axis, x along it) and run as a three-dimensional column
    on a periodic box: the axis along z over one period 2 pi (n nodes,
    spacing h = 2 pi / n), radius a + amp cos(z) in those units, i.e. a / h
    lattice units with a relative perturbation amp / a, fluid at rest.  The
    transverse box has side 2 pi (n_side = n nodes: the radial extent pi on
    each side of the axis) unless n_side says otherwise.  Returns (case, phi0)."""
    h = 2.0 * np.pi / n
    m = n if n_side is None else int(n_side)
    case = base_case3(m, m, n, W=W, sigma=sigma, tau_g=tau_g, rho_l=rho_ratio, rho_g=1.0,
                      tau_f_l=tau_f, tau_f_g=tau_f, **{"lambda": lam})
    return case, liquid_column(m, m, n, a / h, W, eps=amp / a, wavelength=n)


def droplet_lattice(nx=16384, ny=8192, mx=64, my=32, R=24.0, W=4.0, lam=0.5):
    """One large periodic grid holding an mx x my lattice of equal droplets of
    radius R (tanh profile), each centred in its (nx/mx) x (ny/my) cell, with
    the physics of the two-droplet set-up of Sec. 4.1 (sigma = 1e-3,
    tau_g = 0.8, tau_f = 1, density ratio 1), fluid at rest.  The field is
    one cell repeated, so a run of the whole grid equals, cell by cell, a run
    of one periodic cell.  Returns (case, phi0, cell)."""
    cx, cy = nx // mx, ny // my
    assert cx * mx == nx and cy * my == ny
    cell = tanh_disc(cx, cy, 0.5 * cx, 0.5 * cy, R, W, periodic=True)
    case = base_case(nx, ny, W=W, sigma=1e-3, tau_g=0.8, **{"lambda": lam})
    return case, np.tile(cell, (my, mx)), cell
