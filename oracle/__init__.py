"""FP64 CPU oracle of the coupled volume-conserving LB step -- TEST INFRASTRUCTURE.

This package is not the product.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It wraps
``lbm_oracle.c`` (a plain C restatement of Secs. 3.1-3.2 of Xiong, Wang & Liu,
arXiv 2505.10899) through ctypes and shares no code with the CUDA library.

Every function here is argument marshalling; the arithmetic is in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, plant: int = 0) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP).

    plant > 0 builds a copy with one deliberately wrong formula (ORC_PLANT in
    lbm_oracle.c), used only by the mutation test of the pins."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO if plant == 0 else _SO.replace(".so", f"_plant{plant}.so")
    if (not force and os.path.exists(so)
            and os.path.getmtime(so) >= os.path.getmtime(_SRC)):
        return so
    tmp = so + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           f"-DORC_PLANT={int(plant)}", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in lbm_oracle.c."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("flow", ctypes.c_int32), ("walls", ctypes.c_int32),
        ("W", ctypes.c_double), ("sigma", ctypes.c_double),
        ("lam", ctypes.c_double), ("xi", ctypes.c_double),
        ("tau_g", ctypes.c_double),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("tau_f_l", ctypes.c_double), ("tau_f_g", ctypes.c_double),
        ("s_f", ctypes.c_double * 9), ("s_g", ctypes.c_double * 9),
        ("vortex_U", ctypes.c_double), ("vortex_T", ctypes.c_double),
        ("u_top", ctypes.c_double), ("u_bot", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I8 = ctypes.POINTER(ctypes.c_int8)
_I32 = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = build(plant=int(os.environ.get("ORACLE_PLANT", "0")))
            L = ctypes.CDLL(so)
            P = ctypes.POINTER(Params)
            L.orc_lattice.argtypes = [_I32, _I32, _D]
            L.orc_matrices.argtypes = [_D, _D]
            L.orc_feq.argtypes = [ctypes.c_double] * 4 + [_D]
            L.orc_force.argtypes = [ctypes.c_double] * 6 + [_D]
            L.orc_geq.argtypes = [ctypes.c_double] * 5 + [_D]
            L.orc_gsrc.argtypes = [ctypes.c_double] * 7 + [_D]
            L.orc_psi.argtypes = [ctypes.c_double] * 3
            L.orc_psi.restype = ctypes.c_double
            L.orc_chem.argtypes = [ctypes.c_double] * 4
            L.orc_chem.restype = ctypes.c_double
            L.orc_mrt.argtypes = [_D, _D, _D, _D, _D]
            L.orc_stencil.argtypes = [_D, ctypes.c_int32, ctypes.c_int32, _D, _D, _D]
            L.orc_init.argtypes = [P, _D, _D, _D, _D, _D]
            L.orc_step.argtypes = [P, _D, _D, _D, ctypes.c_int64, ctypes.c_int64]
            L.orc_fields.argtypes = [P, _D, _D, ctypes.c_int64, _D, _D, _D, _D]
            L.orc_collide.argtypes = [P, _D, _D, _D, ctypes.c_int64, _D, _D, _D]
            L.orc_volume.argtypes = [P, _D, _I8, ctypes.c_int32, _D]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def make_params(case: dict) -> Params:
    """Build the oracle's parameter struct from a plain case dictionary."""
    p = Params()
    p.nx, p.ny = int(case["nx"]), int(case["ny"])
    p.flow = {"coupled": 0, "vortex": 1}[case.get("flow", "coupled")]
    p.W = case["W"]
    p.sigma = case["sigma"]
    p.lam = case.get("lambda", 0.5)
    p.xi = case.get("xi", 1e-10)
    p.tau_g = case["tau_g"]
    p.rho_l = case.get("rho_l", 1.0)
    p.rho_g = case.get("rho_g", 1.0)
    p.tau_f_l = case.get("tau_f_l", 1.0)
    p.tau_f_g = case.get("tau_f_g", case.get("tau_f_l", 1.0))
    sf = case.get("s_f", [1.0] * 9)
    sg = case.get("s_g", [1.0] * 9)
    for k in range(9):
        p.s_f[k] = sf[k]
        p.s_g[k] = sg[k]
    p.vortex_U = case.get("vortex_U", 0.0)
    p.vortex_T = case.get("vortex_T", 1.0)
    p.walls = int(case.get("walls", 0))
    p.u_top = case.get("u_top", 0.0)
    p.u_bot = case.get("u_bot", 0.0)
    return p


def lattice():
    cx = (ctypes.c_int32 * 9)()
    cy = (ctypes.c_int32 * 9)()
    w = (ctypes.c_double * 9)()
    lib().orc_lattice(cx, cy, w)
    return np.array(cx[:]), np.array(cy[:]), np.array(w[:])


def matrices():
    m = np.zeros(81)
    mi = np.zeros(81)
    lib().orc_matrices(_dp(m), _dp(mi))
    return m.reshape(9, 9), mi.reshape(9, 9)


def feq(p, rho, ux, uy):
    out = np.zeros(9)
    lib().orc_feq(p, rho, ux, uy, _dp(out))
    return out


def force(ux, uy, Fx, Fy, grx, gry):
    out = np.zeros(9)
    lib().orc_force(ux, uy, Fx, Fy, grx, gry, _dp(out))
    return out


def geq(phi, mu, lam, ux, uy):
    out = np.zeros(9)
    lib().orc_geq(phi, mu, lam, ux, uy, _dp(out))
    return out


def gsrc(dJx, dJy, lam, W, psi, nx_, ny_):
    out = np.zeros(9)
    lib().orc_gsrc(dJx, dJy, lam, W, psi, nx_, ny_, _dp(out))
    return out


def psi(phi, W, xi=1e-10):
    return lib().orc_psi(phi, W, xi)


def chem(phi, lap, W, sigma):
    return lib().orc_chem(phi, lap, W, sigma)


def mrt(f, fe, F, s):
    out = np.zeros(9)
    f, fe, F, s = (np.ascontiguousarray(a, dtype=np.float64) for a in (f, fe, F, s))
    lib().orc_mrt(_dp(f), _dp(fe), _dp(F), _dp(s), _dp(out))
    return out


def stencil(chi):
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    ny, nx = chi.shape
    gx, gy, lap = (np.zeros_like(chi) for _ in range(3))
    lib().orc_stencil(_dp(chi), nx, ny, _dp(gx), _dp(gy), _dp(lap))
    return gx, gy, lap


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracles' OpenMP loops (process-wide)."""
    lib().orc_set_num_threads(int(n))


class Oracle:
    """State holder around the C oracle: populations after streaming at time t."""

    def __init__(self, case: dict, phi0=None, u0=None, state=None):
        self.case = dict(case)
        self.p = make_params(case)
        nx, ny = self.p.nx, self.p.ny
        self.n = nx * ny
        self.shape = (ny, nx)
        self.coupled = self.p.flow == 0
        if state is not None:
            f, g, j, t = state
            self.f = None if f is None else np.ascontiguousarray(f, np.float64).copy()
            self.g = np.ascontiguousarray(g, np.float64).copy()
            self.j = np.ascontiguousarray(j, np.float64).copy()
            self.t = int(t)
            return
        self.f = np.zeros((9, ny, nx)) if self.coupled else None
        self.g = np.zeros((9, ny, nx))
        self.j = np.zeros((2, ny, nx))
        self.t = 0
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
        assert phi0.shape == self.shape
        u0p = None
        if u0 is not None:
            u0 = np.ascontiguousarray(u0, dtype=np.float64)
            assert u0.shape == (2, ny, nx)
            u0p = _dp(u0)
        _check(lib().orc_init(ctypes.byref(self.p), _dp(phi0), u0p,
                              _dp(self.f), _dp(self.g), _dp(self.j)), "init")

    def step(self, nsteps: int):
        _check(lib().orc_step(ctypes.byref(self.p), _dp(self.f), _dp(self.g),
                              _dp(self.j), self.t, int(nsteps)), "step")
        self.t += int(nsteps)
        return self

    def fields(self):
        ny, nx = self.shape
        phi, ux, uy, pr = (np.zeros((ny, nx)) for _ in range(4))
        _check(lib().orc_fields(ctypes.byref(self.p), _dp(self.f), _dp(self.g),
                                self.t, _dp(phi), _dp(ux), _dp(uy), _dp(pr)), "fields")
        return phi, ux, uy, pr

    def collide(self):
        ny, nx = self.shape
        fs = np.zeros((9, ny, nx)) if self.coupled else None
        gs = np.zeros((9, ny, nx))
        jn = np.zeros((2, ny, nx))
        _check(lib().orc_collide(ctypes.byref(self.p), _dp(self.f), _dp(self.g),
                                 _dp(self.j), self.t, _dp(fs), _dp(gs), _dp(jn)),
               "collide")
        return fs, gs, jn

    def volume(self, labels=None, nregions=1):
        out = np.zeros(int(nregions))
        lp = None
        if labels is not None:
            labels = np.ascontiguousarray(labels, dtype=np.int8)
            assert labels.shape == self.shape
            lp = labels.ctypes.data_as(_I8)
        _check(lib().orc_volume(ctypes.byref(self.p), _dp(self.g), lp,
                                int(nregions), _dp(out)), "volume")
        return out

    def phi(self):
        return self.g.sum(axis=0)


# ---------------------------------------------------------------------------
# Three-dimensional extension (D3Q19 flow, D3Q7 phase field, SRT limit of
# Eqs. 25 and 33); arithmetic in lbm_oracle3d.c.

_SRC3 = os.path.join(_HERE, "lbm_oracle3d.c")
_SO3 = os.path.join(_BUILD, "liblbm_oracle3d.so")
_lib3 = None


def build3(force: bool = False, plant: int = 0) -> str:
    """Compile the 3-D oracle (same flags as build())."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO3 if plant == 0 else _SO3.replace(".so", f"_plant{plant}.so")
    if (not force and os.path.exists(so)
            and os.path.getmtime(so) >= os.path.getmtime(_SRC3)):
        return so
    tmp = so + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           f"-DORC_PLANT={int(plant)}", "-fPIC", "-shared", "-o", tmp, _SRC3, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


class Params3(ctypes.Structure):
    """Mirror of ``orc3_params`` in lbm_oracle3d.c."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("W", ctypes.c_double), ("sigma", ctypes.c_double),
        ("lam", ctypes.c_double), ("xi", ctypes.c_double),
        ("tau_g", ctypes.c_double),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("tau_f_l", ctypes.c_double), ("tau_f_g", ctypes.c_double),
    ]


def lib3():
    global _lib3
    with _lock:
        if _lib3 is None:
            L = ctypes.CDLL(build3(plant=int(os.environ.get("ORACLE_PLANT", "0"))))
            P = ctypes.POINTER(Params3)
            L.orc3_lattices.argtypes = [_I32, _D, _I32, _D]
            L.orc3_feq.argtypes = [ctypes.c_double, ctypes.c_double, _D, _D]
            L.orc3_force.argtypes = [_D, _D, _D, _D]
            L.orc3_geq.argtypes = [ctypes.c_double] * 3 + [_D, _D]
            L.orc3_gsrc.argtypes = [_D, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, _D, _D]
            L.orc3_stencil.argtypes = [P, _D, _D, _D, _D, _D]
            L.orc3_init.argtypes = [P, _D, _D, _D, _D, _D]
            L.orc3_step.argtypes = [P, _D, _D, _D, ctypes.c_int64]
            L.orc3_fields.argtypes = [P, _D, _D, _D, _D, _D]
            _lib3 = L
    return _lib3


def make_params3(case: dict) -> Params3:
    p = Params3()
    p.nx, p.ny, p.nz = int(case["nx"]), int(case["ny"]), int(case["nz"])
    p.W = case["W"]
    p.sigma = case["sigma"]
    p.lam = case.get("lambda", 0.5)
    p.xi = case.get("xi", 1e-10)
    p.tau_g = case["tau_g"]
    p.rho_l = case.get("rho_l", 1.0)
    p.rho_g = case.get("rho_g", 1.0)
    p.tau_f_l = case.get("tau_f_l", 1.0)
    p.tau_f_g = case.get("tau_f_g", case.get("tau_f_l", 1.0))
    return p


def _vec(v, n):
    return np.ascontiguousarray(np.broadcast_to(np.asarray(v, np.float64), (n,)))


def lattices3():
    """(c19 [19,3], w19 [19], c7 [7,3], w7 [7]) as the 3-D oracle uses them."""
    c19 = (ctypes.c_int32 * 57)()
    w19 = (ctypes.c_double * 19)()
    c7 = (ctypes.c_int32 * 21)()
    w7 = (ctypes.c_double * 7)()
    lib3().orc3_lattices(c19, w19, c7, w7)
    return (np.array(c19[:]).reshape(19, 3), np.array(w19[:]),
            np.array(c7[:]).reshape(7, 3), np.array(w7[:]))


def feq3(p, rho, u):
    out = np.zeros(19)
    lib3().orc3_feq(p, rho, _dp(_vec(u, 3)), _dp(out))
    return out


def force3(u, F, grad_rho):
    out = np.zeros(19)
    lib3().orc3_force(_dp(_vec(u, 3)), _dp(_vec(F, 3)), _dp(_vec(grad_rho, 3)), _dp(out))
    return out


def geq3(phi, mu, lam, u):
    out = np.zeros(7)
    lib3().orc3_geq(phi, mu, lam, _dp(_vec(u, 3)), _dp(out))
    return out


def gsrc3(dJ, lam, W, psi, n):
    out = np.zeros(7)
    lib3().orc3_gsrc(_dp(_vec(dJ, 3)), lam, W, psi, _dp(_vec(n, 3)), _dp(out))
    return out


def stencil3(chi):
    """Isotropic D3Q19 gradient and Laplacian of a periodic [nz][ny][nx] field."""
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    nz, ny, nx = chi.shape
    p = Params3()
    p.nx, p.ny, p.nz = nx, ny, nz
    p.W, p.tau_g, p.rho_l, p.rho_g, p.tau_f_l, p.tau_f_g = 4.0, 1.0, 1.0, 1.0, 1.0, 1.0
    gx, gy, gz, lap = (np.zeros_like(chi) for _ in range(4))
    _check(lib3().orc3_stencil(ctypes.byref(p), _dp(chi), _dp(gx), _dp(gy), _dp(gz),
                               _dp(lap)), "stencil3")
    return gx, gy, gz, lap


class Oracle3:
    """State holder around the 3-D oracle: f [19][z][y][x], g [7][z][y][x],
    phi*u of the previous step [3][z][y][x], after streaming at step t."""

    def __init__(self, case: dict, phi0=None, u0=None, state=None):
        self.case = dict(case)
        self.p = make_params3(case)
        nx, ny, nz = self.p.nx, self.p.ny, self.p.nz
        self.shape = (nz, ny, nx)
        if state is not None:
            f, g, j, t = state
            self.f = np.ascontiguousarray(f, np.float64).copy()
            self.g = np.ascontiguousarray(g, np.float64).copy()
            self.j = np.ascontiguousarray(j, np.float64).copy()
            self.t = int(t)
            return
        self.f = np.zeros((19,) + self.shape)
        self.g = np.zeros((7,) + self.shape)
        self.j = np.zeros((3,) + self.shape)
        self.t = 0
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
        assert phi0.shape == self.shape
        u0p = None
        if u0 is not None:
            u0 = np.ascontiguousarray(u0, dtype=np.float64)
            assert u0.shape == (3,) + self.shape
            u0p = _dp(u0)
        _check(lib3().orc3_init(ctypes.byref(self.p), _dp(phi0), u0p, _dp(self.f),
                                _dp(self.g), _dp(self.j)), "init3")

    def step(self, nsteps: int):
        _check(lib3().orc3_step(ctypes.byref(self.p), _dp(self.f), _dp(self.g),
                                _dp(self.j), int(nsteps)), "step3")
        self.t += int(nsteps)
        return self

    def fields(self):
        """phi [z][y][x], u [3][z][y][x], p [z][y][x] (Eqs. 28, 29, 35)."""
        phi = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        pr = np.zeros(self.shape)
        _check(lib3().orc3_fields(ctypes.byref(self.p), _dp(self.f), _dp(self.g),
                                  _dp(phi), _dp(u), _dp(pr)), "fields3")
        return phi, u, pr

    def phi(self):
        return self.g.sum(axis=0)

    def volume(self, labels=None, nregions=1):
        """Phase volumes sum(phi) per label (FP64), Eq. 35 summed over nodes."""
        phi = self.phi().ravel()
        if labels is None:
            return np.array([phi.sum()])
        lab = np.asarray(labels).ravel()
        return np.array([phi[lab == k].sum() for k in range(int(nregions))])
