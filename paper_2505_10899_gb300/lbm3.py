"""ctypes binding of the three-dimensional entry points (include/lbm3_api.h) of
liblbm_gb300.so: argument marshalling only, same names as the C ABI.

``Sim3`` wraps a handle with its device workspace (a torch uint8 tensor on the
current CUDA device).  There is no CPU fallback: importing this module fails
when the library has not been built.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .lbm import LBM_ABI_VERSION, LBM_ERR_ARG, LBM_OK, LbmError, lib as _lib2

LBM3_F64, LBM3_F32, LBM3_F16 = 0, 1, 2
PRECISIONS = {"f64": LBM3_F64, "f32": LBM3_F32, "f16": LBM3_F16}


class lbm3_params(ctypes.Structure):
    _fields_ = [
        ("abi_version", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32), ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("W", ctypes.c_double), ("sigma", ctypes.c_double), ("lam", ctypes.c_double),
        ("xi", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("tau_f_l", ctypes.c_double), ("tau_f_g", ctypes.c_double),
    ]


_P = ctypes.POINTER(lbm3_params)
_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_H = ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)

_lib = _lib2()
for _name, (_args, _res) in {
    "lbm3_workspace_bytes": ([_P], ctypes.c_size_t),
    "lbm3_init": ([_P, _VP, ctypes.c_size_t, _D, _D, _VP, ctypes.POINTER(_H)], ctypes.c_int),
    "lbm3_step": ([_H, ctypes.c_int64], ctypes.c_int),
    "lbm3_set_regions": ([_H, ctypes.POINTER(ctypes.c_int8), ctypes.c_int32], ctypes.c_int),
    "lbm3_volume": ([_H, _D], ctypes.c_int),
    "lbm3_track_volume": ([_H, _VP], ctypes.c_int),
    "lbm3_fields": ([_H, _D, _D, _D], ctypes.c_int),
    "lbm3_get_state": ([_H, _D, _D, _D, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "lbm3_set_state": ([_H, _D, _D, _D, ctypes.c_int64], ctypes.c_int),
    "lbm3_time": ([_H], ctypes.c_int64),
    "lbm3_set_tiling": ([_H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "lbm3_get_tiling": ([_H, _I32P, _I32P, _I32P, _I32P], ctypes.c_int),
    "lbm3_autotune": ([_H, ctypes.c_int32, _I32P, _I32P, _I32P, _I32P, _D], ctypes.c_int),
    "lbm3_set_kernel": ([_H, ctypes.c_int32], ctypes.c_int),
    "lbm3_set_wait_limit": ([_H, ctypes.c_int64], ctypes.c_int),
    "lbm3_get_kernel": ([_H], ctypes.c_int32),
    "lbm3_status": ([_H], ctypes.c_int),
    "lbm3_destroy": ([_H], None),
}.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


def _check(rc, where):
    if rc != LBM_OK:
        raise LbmError(rc, where, _lib.lbm_last_error().decode(errors="replace"))
    return rc


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def make_params(case: dict, precision: str = "f32") -> lbm3_params:
    """lbm3_params from a plain case dictionary (see workloads.base_case3)."""
    p = lbm3_params()
    p.abi_version = LBM_ABI_VERSION
    p.nx, p.ny, p.nz = int(case["nx"]), int(case["ny"]), int(case["nz"])
    p.precision = PRECISIONS[precision]
    p.reserved = 0
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


def lbm3_workspace_bytes(p: lbm3_params) -> int:
    return int(_lib.lbm3_workspace_bytes(ctypes.byref(p)))


def lbm3_init(p: lbm3_params, d_workspace: int, ws_bytes: int, phi0, u0=None, stream: int = 0):
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
    h = _H()
    _check(_lib.lbm3_init(ctypes.byref(p), ctypes.c_void_p(d_workspace), ws_bytes, _dp(phi0),
                          _dp(u0), ctypes.c_void_p(stream), ctypes.byref(h)), "lbm3_init")
    return h


def lbm3_step(h, nsteps: int):
    return _check(_lib.lbm3_step(h, int(nsteps)), "lbm3_step")


def lbm3_set_regions(h, labels, nregions: int):
    lp = None
    if labels is not None:
        labels = np.ascontiguousarray(labels, dtype=np.int8)
        lp = labels.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    return _check(_lib.lbm3_set_regions(h, lp, int(nregions)), "lbm3_set_regions")


def lbm3_volume(h, nregions: int = 1):
    out = np.zeros(int(nregions))
    _check(_lib.lbm3_volume(h, _dp(out)), "lbm3_volume")
    return out


def lbm3_track_volume(h, d_out: int):
    return _check(_lib.lbm3_track_volume(h, ctypes.c_void_p(d_out) if d_out else None),
                  "lbm3_track_volume")


def lbm3_fields(h, shape):
    phi, p = np.zeros(shape), np.zeros(shape)
    u = np.zeros((3,) + tuple(shape))
    _check(_lib.lbm3_fields(h, _dp(phi), _dp(u), _dp(p)), "lbm3_fields")
    return phi, u, p


def lbm3_get_state(h, shape):
    f = np.zeros((19,) + tuple(shape))
    g = np.zeros((7,) + tuple(shape))
    j = np.zeros((3,) + tuple(shape))
    t = ctypes.c_int64(0)
    _check(_lib.lbm3_get_state(h, _dp(f), _dp(g), _dp(j), ctypes.byref(t)), "lbm3_get_state")
    return f, g, j, int(t.value)


def lbm3_set_state(h, f, g, j, t: int):
    f, g, j = (None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (f, g, j))
    return _check(_lib.lbm3_set_state(h, _dp(f), _dp(g), _dp(j), int(t)), "lbm3_set_state")


def lbm3_time(h) -> int:
    return int(_lib.lbm3_time(h))


def lbm3_set_tiling(h, bx: int, by: int, zc: int):
    return _check(_lib.lbm3_set_tiling(h, int(bx), int(by), int(zc)), "lbm3_set_tiling")


def lbm3_get_tiling(h):
    v = [ctypes.c_int32() for _ in range(4)]
    _check(_lib.lbm3_get_tiling(h, *[ctypes.byref(x) for x in v]), "lbm3_get_tiling")
    return tuple(int(x.value) for x in v)


def lbm3_autotune(h, trials: int = 3):
    var, bx, by, zc = (ctypes.c_int32() for _ in range(4))
    ms = ctypes.c_double()
    _check(_lib.lbm3_autotune(h, int(trials), ctypes.byref(var), ctypes.byref(bx),
                              ctypes.byref(by), ctypes.byref(zc), ctypes.byref(ms)),
           "lbm3_autotune")
    return {"kernel": int(var.value), "bx": int(bx.value), "by": int(by.value),
            "zc": int(zc.value), "ms": float(ms.value)}


def lbm3_set_kernel(h, variant: int):
    return _check(_lib.lbm3_set_kernel(h, int(variant)), "lbm3_set_kernel")


def lbm3_set_wait_limit(h, cycles: int):
    return _check(_lib.lbm3_set_wait_limit(h, int(cycles)), "lbm3_set_wait_limit")


def lbm3_get_kernel(h) -> int:
    return int(_lib.lbm3_get_kernel(h))


def lbm3_status(h) -> int:
    return int(_lib.lbm3_status(h))


def lbm3_destroy(h):
    if h:
        _lib.lbm3_destroy(h)


class Sim3:
    """One periodic 3-D box advanced on the current CUDA device."""

    def __init__(self, case, phi0, u0=None, precision="f32", stream=None, device=None):
        import torch  # device memory and streams only

        if not torch.cuda.is_available():
            raise RuntimeError("Sim3 needs a CUDA device")
        self.case = dict(case)
        self.params = make_params(case, precision)
        self.precision = precision
        self.shape = (self.params.nz, self.params.ny, self.params.nx)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = lbm3_workspace_bytes(self.params)
        if nbytes == 0:
            raise LbmError(LBM_ERR_ARG, "lbm3_workspace_bytes",
                           _lib.lbm_last_error().decode(errors="replace"))
        self.ws_bytes = nbytes
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = (self.workspace.data_ptr() + 255) // 256 * 256
        self.nregions = 1
        self.h = lbm3_init(self.params, self.ws_ptr, nbytes, phi0, u0, self.stream.cuda_stream)

    def step(self, n):
        lbm3_step(self.h, n)
        return self

    def set_regions(self, labels, nregions):
        lbm3_set_regions(self.h, labels, nregions)
        self.nregions = int(nregions)

    def volume(self):
        return lbm3_volume(self.h, self.nregions)

    def track_volume(self, enable=True):
        import torch
        if enable:
            self.vol_track = torch.zeros(1, dtype=torch.float64, device=self.device)
            lbm3_track_volume(self.h, self.vol_track.data_ptr())
            return self.vol_track
        lbm3_track_volume(self.h, 0)
        self.vol_track = None
        return None

    def fields(self):
        return lbm3_fields(self.h, self.shape)

    def get_state(self):
        return lbm3_get_state(self.h, self.shape)

    def set_state(self, f, g, j, t):
        lbm3_set_state(self.h, f, g, j, t)

    def tiling(self):
        return lbm3_get_tiling(self.h)

    def set_tiling(self, bx, by, zc):
        lbm3_set_tiling(self.h, bx, by, zc)

    def autotune(self, trials=3):
        return lbm3_autotune(self.h, trials)

    def set_kernel(self, variant):
        lbm3_set_kernel(self.h, variant)

    def kernel(self):
        return lbm3_get_kernel(self.h)

    def set_wait_limit(self, cycles):
        lbm3_set_wait_limit(self.h, cycles)

    @property
    def t(self):
        return lbm3_time(self.h)

    def status(self):
        return lbm3_status(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
