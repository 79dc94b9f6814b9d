"""ctypes binding of liblbm_gb300.so (include/lbm_api.h): argument marshalling only.

Every entry point of the C ABI is exposed under the same name.  ``Sim`` wraps a
handle together with its device workspace, which is a torch uint8 tensor on
the current CUDA device (torch provides device memory and the stream; all
arithmetic runs in the library's CUDA kernels).  There is no CPU fallback:
importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_GB300_CHECKED=1 selects the debug build with index checks in the step
# kernels (build.build(checked=True)), which reports LBM_ERR_BOUNDS
LIB_PATH = os.path.join(_HERE, "_lib", "liblbm_gb300_checked.so"
                        if os.environ.get("LBM_GB300_CHECKED") == "1" else "liblbm_gb300.so")

LBM_ABI_VERSION = 2
LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_WORKSPACE = 0, -1, -2, -3
LBM_ERR_NONFINITE, LBM_ERR_TIMEOUT, LBM_ERR_UNIMPLEMENTED = -4, -5, -6
LBM_ERR_BOUNDS = -7
LBM_F64, LBM_F32 = 0, 1
LBM_FLOW_COUPLED, LBM_FLOW_VORTEX = 0, 1


class LbmError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("abi_version", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("flow", ctypes.c_int32), ("walls", ctypes.c_int32),
        ("W", ctypes.c_double), ("sigma", ctypes.c_double), ("lam", ctypes.c_double),
        ("xi", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("tau_f_l", ctypes.c_double), ("tau_f_g", ctypes.c_double),
        ("s_f", ctypes.c_double * 9), ("s_g", ctypes.c_double * 9),
        ("vortex_U", ctypes.c_double), ("vortex_T", ctypes.c_double),
        ("u_wall_top", ctypes.c_double), ("u_wall_bottom", ctypes.c_double),
    ]


_P = ctypes.POINTER(lbm_params)
_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_H = ctypes.c_void_p


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -m paper_2505_10899_gb300.build or __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "lbm_abi_version": ([], ctypes.c_int32),
        "lbm_last_error": ([], ctypes.c_char_p),
        "lbm_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "lbm_workspace_bytes": ([_P, ctypes.c_int32], ctypes.c_size_t),
        "lbm_init": ([_P, ctypes.c_int32, _VP, ctypes.c_size_t, ctypes.POINTER(_D),
                      ctypes.POINTER(_D), _VP, ctypes.POINTER(_H)], ctypes.c_int),
        "lbm_step": ([_H, ctypes.c_int64], ctypes.c_int),
        "lbm_prepare_steps": ([_H, ctypes.c_int64], ctypes.c_int),
        "lbm_set_chains": ([_H, ctypes.c_int32], ctypes.c_int),
        "lbm_get_chains": ([_H], ctypes.c_int32),
        "lbm_set_row_chains": ([_H, ctypes.c_int32], ctypes.c_int),
        "lbm_get_row_chains": ([_H], ctypes.c_int32),
        "lbm_set_wait_limit": ([_H, ctypes.c_int64], ctypes.c_int),
        "lbm_fp64_fma_rate": ([ctypes.c_int64, ctypes.c_int32, _D, _D], ctypes.c_int),
        "lbm_record_steps": ([_H, ctypes.c_int64, _VP, ctypes.c_int64], ctypes.c_int),
        "lbm_adjoint_sweep": ([_H, _VP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _VP,
                               _VP], ctypes.c_int),
        "lbm_set_regions": ([_H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int8), ctypes.c_int32],
                            ctypes.c_int),
        "lbm_volume": ([_H, _D], ctypes.c_int),
        "lbm_volume_async": ([_H, _VP], ctypes.c_int),
        "lbm_num_regions": ([_H], ctypes.c_int32),
        "lbm_track_volume": ([_H, _VP], ctypes.c_int),
        "lbm_track_volume_history": ([_H, _VP, ctypes.c_int64], ctypes.c_int),
        "lbm_get_tiling": ([_H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "lbm_set_tiling": ([_H, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
        "lbm_set_kernel": ([_H, ctypes.c_int32], ctypes.c_int),
        "lbm_autotune": ([_H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), _D],
                         ctypes.c_int),
        "lbm_get_kernel": ([_H], ctypes.c_int32),
        "lbm_fields": ([_H, ctypes.c_int32, _D, _D, _D, _D], ctypes.c_int),
        "lbm_get_state": ([_H, ctypes.c_int32, _D, _D, _D, ctypes.POINTER(ctypes.c_int64)],
                          ctypes.c_int),
        "lbm_set_state": ([_H, ctypes.c_int32, _D, _D, _D, ctypes.c_int64], ctypes.c_int),
        "lbm_time": ([_H], ctypes.c_int64),
        "lbm_checkpoint_bytes": ([_H], ctypes.c_size_t),
        "lbm_save": ([_H, _VP, ctypes.c_size_t], ctypes.c_int),
        "lbm_load": ([_H, _VP, ctypes.c_size_t], ctypes.c_int),
        "lbm_status": ([_H], ctypes.c_int),
        "lbm_adjoint_step": ([_H, _VP, _VP, _D], ctypes.c_int),
        "lbm_adjoint_step_from": ([_H, _VP, ctypes.c_int64, _VP, _VP, _D], ctypes.c_int),
        "lbm_adjoint_workspace_bytes": ([_H], ctypes.c_size_t),
        "lbm_adjoint_attach": ([_H, _VP, ctypes.c_size_t], ctypes.c_int),
        "lbm_adjoint_seed_phi": ([_H, _VP, _VP], ctypes.c_int),
        "lbm_adjoint_init": ([_H, _VP, _VP, _VP, _VP, _D], ctypes.c_int),
        "lbm_adjoint_take_param_grads": ([_H, _D], ctypes.c_int),
        "lbm_snapshot_bytes": ([_H, ctypes.c_int32], ctypes.c_size_t),
        "lbm_snapshot": ([_H, ctypes.c_int32, _VP], ctypes.c_int),
        "lbm_restore": ([_H, ctypes.c_int32, _VP], ctypes.c_int),
        "lbm_set_time": ([_H, ctypes.c_int64], ctypes.c_int),
        "lbm_destroy": ([_H], None),
        "lbm_phase_volume_noalloc": ([_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int64, _VP, ctypes.c_int32, _VP, _VP],
                                     ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


_lib = _load()


def lib():
    return _lib


def _check(rc, where):
    if rc != LBM_OK:
        msg = _lib.lbm_last_error().decode(errors="replace")
        raise LbmError(rc, where, msg)
    return rc


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def make_params(case: dict, precision: str = "f32") -> lbm_params:
    """lbm_params from a plain case dictionary (see workloads.base_case)."""
    p = lbm_params()
    p.abi_version = LBM_ABI_VERSION
    p.nx, p.ny = int(case["nx"]), int(case["ny"])
    p.precision = {"f64": LBM_F64, "f32": LBM_F32}[precision]
    p.flow = {"coupled": LBM_FLOW_COUPLED, "vortex": LBM_FLOW_VORTEX}[case.get("flow", "coupled")]
    p.walls = int(case.get("walls", 0))
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
    p.u_wall_top = case.get("u_top", 0.0)
    p.u_wall_bottom = case.get("u_bot", 0.0)
    return p


# --- thin same-name wrappers -------------------------------------------------

def lbm_workspace_bytes(params) -> int:
    arr = (lbm_params * len(params))(*params)
    return int(_lib.lbm_workspace_bytes(arr, len(params)))


def _init_ptr(a):
    """An initial field for lbm_init: a host array (FP64, [ny][nx] or
    [2][ny][nx]), or an int, the address of such an array in device or
    page-locked host memory that the caller keeps alive until lbm_init
    returns."""
    if isinstance(a, (int, np.integer)):
        return ctypes.cast(ctypes.c_void_p(int(a)), _D)
    return _dp(np.ascontiguousarray(a, dtype=np.float64))


def lbm_init(params, d_workspace: int, ws_bytes: int, phi0s, u0s=None, stream: int = 0):
    n = len(params)
    arr = (lbm_params * n)(*params)
    phis = [p if isinstance(p, (int, np.integer)) else np.ascontiguousarray(p, dtype=np.float64)
            for p in phi0s]
    us = [None if u is None else (u if isinstance(u, (int, np.integer))
                                  else np.ascontiguousarray(u, dtype=np.float64))
          for u in (u0s if u0s is not None else [None] * n)]
    phi_ptrs = (_D * n)(*[_init_ptr(p) for p in phis])
    u_ptrs = (_D * n)(*[_init_ptr(u) if u is not None else _D() for u in us])
    h = _H()
    _check(_lib.lbm_init(arr, n, ctypes.c_void_p(d_workspace), ws_bytes, phi_ptrs, u_ptrs,
                         ctypes.c_void_p(stream), ctypes.byref(h)), "lbm_init")
    return h


def lbm_step(h, nsteps: int):
    return _check(_lib.lbm_step(h, int(nsteps)), "lbm_step")


def lbm_prepare_steps(h, nsteps: int):
    return _check(_lib.lbm_prepare_steps(h, int(nsteps)), "lbm_prepare_steps")


def lbm_set_chains(h, nchains: int):
    return _check(_lib.lbm_set_chains(h, int(nchains)), "lbm_set_chains")


def lbm_get_chains(h) -> int:
    return int(_lib.lbm_get_chains(h))


def lbm_fp64_fma_rate(trips: int = 40000, blocks_per_sm: int = 4):
    """FP64 FMAs per second of the current device and the timed milliseconds."""
    r, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.lbm_fp64_fma_rate(int(trips), int(blocks_per_sm), ctypes.byref(r),
                                  ctypes.byref(ms)), "lbm_fp64_fma_rate")
    return float(r.value), float(ms.value)


def lbm_record_steps(h, count: int, d_states: int, stride_bytes: int):
    return _check(_lib.lbm_record_steps(h, int(count), ctypes.c_void_p(d_states),
                                        int(stride_bytes)), "lbm_record_steps")


def lbm_adjoint_sweep(h, d_states: int, stride_bytes: int, t0: int, count: int, d_adj: int,
                      d_spare: int):
    return _check(_lib.lbm_adjoint_sweep(h, ctypes.c_void_p(d_states), int(stride_bytes),
                                         int(t0), int(count), ctypes.c_void_p(d_adj),
                                         ctypes.c_void_p(d_spare)), "lbm_adjoint_sweep")


def lbm_set_wait_limit(h, cycles: int):
    return _check(_lib.lbm_set_wait_limit(h, int(cycles)), "lbm_set_wait_limit")


def lbm_set_regions(h, c: int, labels, nregions: int):
    lp = None
    if labels is not None:
        labels = np.ascontiguousarray(labels, dtype=np.int8)
        lp = labels.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    return _check(_lib.lbm_set_regions(h, int(c), lp, int(nregions)), "lbm_set_regions")


def lbm_track_volume(h, d_out: int):
    return _check(_lib.lbm_track_volume(h, ctypes.c_void_p(d_out) if d_out else None),
                  "lbm_track_volume")


def lbm_track_volume_history(h, out: int, nslots: int):
    """out: address of device or page-locked host memory, nslots * ncases FP64."""
    return _check(_lib.lbm_track_volume_history(h, ctypes.c_void_p(out) if out else None,
                                                int(nslots)), "lbm_track_volume_history")


def lbm_get_tiling(h):
    bx, rows, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.lbm_get_tiling(h, ctypes.byref(bx), ctypes.byref(rows), ctypes.byref(n)),
           "lbm_get_tiling")
    return int(bx.value), int(rows.value), int(n.value)


def lbm_set_tiling(h, bx: int, rows: int):
    return _check(_lib.lbm_set_tiling(h, int(bx), int(rows)), "lbm_set_tiling")


def lbm_autotune(h, trials: int = 3):
    k, bx, rows = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ms = ctypes.c_double()
    _check(_lib.lbm_autotune(h, int(trials), ctypes.byref(k), ctypes.byref(bx),
                             ctypes.byref(rows), ctypes.byref(ms)), "lbm_autotune")
    return {"kernel": int(k.value), "bx": int(bx.value), "rows": int(rows.value),
            "ms": float(ms.value)}


def lbm_set_kernel(h, variant: int):
    return _check(_lib.lbm_set_kernel(h, int(variant)), "lbm_set_kernel")


def lbm_get_kernel(h) -> int:
    return int(_lib.lbm_get_kernel(h))


def lbm_num_regions(h) -> int:
    return int(_lib.lbm_num_regions(h))


def lbm_volume(h, out=None):
    if out is None:
        out = np.zeros(lbm_num_regions(h))
    _check(_lib.lbm_volume(h, _dp(out)), "lbm_volume")
    return out


def lbm_volume_async(h, d_out: int):
    return _check(_lib.lbm_volume_async(h, ctypes.c_void_p(d_out)), "lbm_volume_async")


def lbm_fields(h, c: int, shape):
    phi, ux, uy, p = (np.zeros(shape) for _ in range(4))
    _check(_lib.lbm_fields(h, int(c), _dp(phi), _dp(ux), _dp(uy), _dp(p)), "lbm_fields")
    return phi, ux, uy, p


def lbm_get_state(h, c: int, shape, coupled=True):
    ny, nx = shape
    f = np.zeros((9, ny, nx)) if coupled else None
    g = np.zeros((9, ny, nx))
    j = np.zeros((2, ny, nx))
    t = ctypes.c_int64(0)
    _check(_lib.lbm_get_state(h, int(c), _dp(f), _dp(g), _dp(j), ctypes.byref(t)),
           "lbm_get_state")
    return f, g, j, int(t.value)


def lbm_set_state(h, c: int, f, g, j, t: int):
    f = None if f is None else np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    j = np.ascontiguousarray(j, dtype=np.float64)
    return _check(_lib.lbm_set_state(h, int(c), _dp(f), _dp(g), _dp(j), int(t)),
                  "lbm_set_state")


def lbm_time(h) -> int:
    return int(_lib.lbm_time(h))


def lbm_checkpoint_bytes(h) -> int:
    return int(_lib.lbm_checkpoint_bytes(h))


def lbm_save(h) -> bytes:
    n = lbm_checkpoint_bytes(h)
    buf = ctypes.create_string_buffer(n)
    _check(_lib.lbm_save(h, buf, n), "lbm_save")
    return buf.raw


def lbm_load(h, data: bytes):
    buf = ctypes.create_string_buffer(data, len(data))
    return _check(_lib.lbm_load(h, buf, len(data)), "lbm_load")


def lbm_status(h) -> int:
    return int(_lib.lbm_status(h))


def lbm_snapshot_bytes(h, c: int = 0) -> int:
    return int(_lib.lbm_snapshot_bytes(h, int(c)))


def lbm_snapshot(h, c: int, d_buf: int):
    return _check(_lib.lbm_snapshot(h, int(c), ctypes.c_void_p(d_buf)), "lbm_snapshot")


def lbm_restore(h, c: int, d_buf: int):
    return _check(_lib.lbm_restore(h, int(c), ctypes.c_void_p(d_buf)), "lbm_restore")


def lbm_set_time(h, t: int):
    return _check(_lib.lbm_set_time(h, int(t)), "lbm_set_time")


def lbm_adjoint_workspace_bytes(h) -> int:
    return int(_lib.lbm_adjoint_workspace_bytes(h))


def lbm_adjoint_attach(h, d_scratch: int, nbytes: int):
    return _check(_lib.lbm_adjoint_attach(h, ctypes.c_void_p(d_scratch), int(nbytes)),
                  "lbm_adjoint_attach")


def lbm_adjoint_seed_phi(h, d_dphi: int, d_adj: int):
    return _check(_lib.lbm_adjoint_seed_phi(h, ctypes.c_void_p(d_dphi), ctypes.c_void_p(d_adj)),
                  "lbm_adjoint_seed_phi")


def lbm_adjoint_step(h, d_in: int, d_out: int, grads=None):
    """Returns the status; adds d/d(sigma, tau_g, lambda, tau_f, u_wall_top,
    u_wall_bottom) into grads (numpy[6])."""
    gp = _dp(grads) if grads is not None else None
    return int(_lib.lbm_adjoint_step(h, ctypes.c_void_p(d_in), ctypes.c_void_p(d_out), gp))


def lbm_adjoint_step_from(h, d_state: int, t: int, d_in: int, d_out: int, grads=None):
    """As lbm_adjoint_step, for the FP64 snapshot d_state of S_t; returns the
    status."""
    gp = _dp(grads) if grads is not None else None
    return int(_lib.lbm_adjoint_step_from(h, ctypes.c_void_p(d_state), int(t),
                                          ctypes.c_void_p(d_in), ctypes.c_void_p(d_out), gp))


def lbm_adjoint_take_param_grads(h, grads):
    return _check(_lib.lbm_adjoint_take_param_grads(h, _dp(grads)), "lbm_adjoint_take_param_grads")


def lbm_adjoint_init(h, d_phi0: int, d_u0: int, d_adj: int, d_out: int, grads=None):
    gp = _dp(grads) if grads is not None else None
    return _check(_lib.lbm_adjoint_init(h, ctypes.c_void_p(d_phi0),
                                        ctypes.c_void_p(d_u0) if d_u0 else None,
                                        ctypes.c_void_p(d_adj), ctypes.c_void_p(d_out), gp),
                  "lbm_adjoint_init")


def lbm_phase_volume_noalloc(d_g: int, precision: str, nx: int, ny: int, plane_stride: int,
                             d_labels: int, nregions: int, d_out: int, stream: int = 0):
    """Phase volumes of device populations without any device allocation."""
    prec = {"f64": LBM_F64, "f32": LBM_F32}[precision]
    return _check(_lib.lbm_phase_volume_noalloc(
        ctypes.c_void_p(d_g), prec, int(nx), int(ny), int(plane_stride),
        ctypes.c_void_p(d_labels) if d_labels else None, int(nregions),
        ctypes.c_void_p(d_out), ctypes.c_void_p(stream)), "lbm_phase_volume_noalloc")


def lbm_destroy(h):
    if h:
        _lib.lbm_destroy(h)


# --- convenience wrapper --------------------------------------------------------

class Sim:
    """A batch of cases advanced together on the current CUDA device."""

    def __init__(self, cases, phi0s, u0s=None, precision="f32", stream=None, device=None):
        import torch  # device memory and streams only

        if not torch.cuda.is_available():
            raise RuntimeError("Sim needs a CUDA device")
        if isinstance(cases, dict):
            cases, phi0s = [cases], [phi0s]
            u0s = None if u0s is None else [u0s]
        self.cases = [dict(c) for c in cases]
        self.params = [make_params(c, precision) for c in cases]
        self.precision = precision
        self.coupled = self.params[0].flow == LBM_FLOW_COUPLED
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = lbm_workspace_bytes(self.params)
        if nbytes == 0:
            raise LbmError(LBM_ERR_ARG, "lbm_workspace_bytes",
                           _lib.lbm_last_error().decode(errors="replace"))
        self.ws_bytes = nbytes
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self.ws_ptr = (base + 255) // 256 * 256
        self.h = lbm_init(self.params, self.ws_ptr, nbytes, phi0s, u0s, self.stream.cuda_stream)

    def shape(self, c=0):
        return (self.cases[c]["ny"], self.cases[c]["nx"])

    def step(self, n):
        lbm_step(self.h, n)
        return self

    def prepare(self, n):
        lbm_prepare_steps(self.h, n)

    def set_chains(self, n):
        lbm_set_chains(self.h, n)

    def set_row_chains(self, on=True):
        """Whole-row chains for cases whose rows fit 64, 96, 192 or 256 columns."""
        _check(_lib.lbm_set_row_chains(self.h, 1 if on else 0), "lbm_set_row_chains")

    def row_chains(self):
        return bool(_lib.lbm_get_row_chains(self.h))

    def chains(self):
        return lbm_get_chains(self.h)

    def set_regions(self, c, labels, nregions):
        lbm_set_regions(self.h, c, labels, nregions)

    def volume(self):
        return lbm_volume(self.h)

    def tiling(self):
        return lbm_get_tiling(self.h)

    def set_tiling(self, bx, rows):
        lbm_set_tiling(self.h, bx, rows)

    def autotune(self, trials=3):
        return lbm_autotune(self.h, trials)

    def set_kernel(self, variant):
        lbm_set_kernel(self.h, variant)

    def kernel(self):
        return lbm_get_kernel(self.h)

    def track_volume(self, enable=True):
        """Fused per-step volumes into a device tensor (one FP64 per case)."""
        import torch
        if enable:
            self.vol_track = torch.zeros(len(self.cases), dtype=torch.float64, device=self.device)
            lbm_track_volume(self.h, self.vol_track.data_ptr())
            return self.vol_track
        lbm_track_volume(self.h, 0)
        self.vol_track = None
        return None

    def track_volume_history(self, nslots, host=True):
        """Fused per-step volumes into an [nslots][ncases] FP64 tensor, slot
        t mod nslots for the state at time t: page-locked host memory that
        the step kernels write directly (host=True), or device memory."""
        import torch
        shape = (int(nslots), len(self.cases))
        if host:
            buf = torch.zeros(shape, dtype=torch.float64).pin_memory()
        else:
            buf = torch.zeros(shape, dtype=torch.float64, device=self.device)
        lbm_track_volume_history(self.h, buf.data_ptr(), nslots)
        self.vol_track = buf
        return buf

    def fields(self, c=0):
        return lbm_fields(self.h, c, self.shape(c))

    def get_state(self, c=0):
        return lbm_get_state(self.h, c, self.shape(c), self.coupled)

    def set_state(self, c, f, g, j, t):
        lbm_set_state(self.h, c, f, g, j, t)

    @property
    def t(self):
        return lbm_time(self.h)

    def save(self):
        return lbm_save(self.h)

    def load(self, data):
        lbm_load(self.h, data)

    def status(self):
        return lbm_status(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
