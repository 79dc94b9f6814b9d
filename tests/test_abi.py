"""The C ABI library loads on a machine without a GPU and exports every entry
point that the headers under include/ declare; parameter validation needs no
device."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT

HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


@pytest.fixture(scope="module")
def L():
    from paper_2505_10899_gb300 import build
    build.build()
    from paper_2505_10899_gb300 import lbm
    return lbm


def declared_symbols(path=None):
    names = set()
    for h in ([path] if path else HEADERS):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"^\s*[\w\s\*]+?\b(lbm3?_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("lbm_init", "lbm_step", "lbm_volume", "lbm_adjoint_step",
                     "lbm_workspace_bytes", "lbm_destroy"):
        assert required in names
    assert len(names) >= 20
    names3 = declared_symbols(os.path.join(ROOT, "include", "lbm3_api.h"))
    for required in ("lbm3_init", "lbm3_step", "lbm3_volume", "lbm3_workspace_bytes",
                     "lbm3_destroy"):
        assert required in names3


def test_library_exports_every_declared_symbol(L):
    so = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(so, n)]
    assert not missing, missing


def test_params_struct_layout(L):
    # 6 int32 + 9 doubles + 2x9 rates + 2 vortex + 2 wall doubles, no padding
    assert ctypes.sizeof(L.lbm_params) == 6 * 4 + 9 * 8 + 18 * 8 + 2 * 8 + 2 * 8
    assert L.lib().lbm_abi_version() == L.LBM_ABI_VERSION


def _case(**kw):
    import workloads as W
    return W.base_case(64, 32, **kw)


def test_workspace_bytes_and_validation(L):
    good = L.make_params(_case(), "f32")
    n32 = L.lbm_workspace_bytes([good])
    n64 = L.lbm_workspace_bytes([L.make_params(_case(), "f64")])
    assert n32 > 64 * 32 * (38 * 4) and n64 > n32
    for bad in (dict(tau_g=0.5), dict(W=0.0), dict(rho_l=-1.0), dict(tau_f_l=0.4),
                dict(s_f=[0.0] + [1.0] * 8),
                dict(s_g=[1.0, 2.0] + [1.0] * 7), dict(walls=2),
                dict(walls=1, flow="vortex", vortex_U=0.02, vortex_T=100.0),
                dict(walls=1, u_top=float("nan"))):
        assert L.lbm_workspace_bytes([L.make_params(_case(**bad), "f32")]) == 0
    # tied rates may hold anything (they are replaced by 1/tau)
    ok = L.make_params(_case(s_f=[1.0] * 7 + [9.0, 9.0], s_g=[1, 1, 1, 7.0, 1, 7.0, 1, 1, 1]))
    assert L.lbm_workspace_bytes([ok]) > 0
    # a batch must agree on launch-uniform fields
    other = L.make_params(_case(sigma=2e-3), "f32")
    assert L.lbm_workspace_bytes([good, other]) == 0
    assert b"launch-uniform" in L.lib().lbm_last_error()
    bigger = L.make_params(dict(_case(), nx=96, ny=80, rho_l=5.0), "f32")
    assert L.lbm_workspace_bytes([good, bigger]) > n32
    p = L.make_params(_case(), "f32")
    p.abi_version = 99
    assert L.lbm_workspace_bytes([p]) == 0


def test_init_rejects_bad_workspace_without_touching_the_device(L):
    p = L.make_params(_case(), "f32")
    import numpy as np
    phi = np.zeros((32, 64))
    with pytest.raises(L.LbmError) as e:
        L.lbm_init([p], 0, 10, [phi])
    assert e.value.status == L.LBM_ERR_WORKSPACE
    with pytest.raises(L.LbmError) as e:
        L.lbm_init([p], 0x1000 + 8, 1 << 30, [phi])   # misaligned pointer
    assert e.value.status == L.LBM_ERR_WORKSPACE
    with pytest.raises(L.LbmError) as e:
        L.lbm_init([p], 0x1000, 16, [phi])            # too small
    assert e.value.status == L.LBM_ERR_WORKSPACE
    # the message states the size that is needed
    assert f"need {L.lbm_workspace_bytes([p])}" in str(e.value)


def test_status_strings(L):
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert L.lib().lbm_status_string(s)


def test_params3_layout_and_validation(L):
    from paper_2505_10899_gb300 import lbm3
    import workloads as W
    assert ctypes.sizeof(lbm3.lbm3_params) == 6 * 4 + 9 * 8
    good = lbm3.make_params(W.base_case3(40, 24, 20), "f32")
    n32 = lbm3.lbm3_workspace_bytes(good)
    n16 = lbm3.lbm3_workspace_bytes(lbm3.make_params(W.base_case3(40, 24, 20), "f16"))
    n64 = lbm3.lbm3_workspace_bytes(lbm3.make_params(W.base_case3(40, 24, 20), "f64"))
    n = 40 * 24 * 20
    assert n16 < n32 < n64 and n32 > n * (2 * 26 * 4 + 2 * 3 * 4)
    for bad in (dict(tau_g=0.5), dict(W=0.0), dict(rho_l=-1.0), dict(tau_f_l=0.4),
                dict(nz=0), dict(nx=1 << 16, ny=1 << 16, nz=2)):
        case = {**W.base_case3(40, 24, 20), **bad}
        assert lbm3.lbm3_workspace_bytes(lbm3.make_params(case, "f32")) == 0
