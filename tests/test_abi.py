"""The C ABI library loads on a machine without a GPU and exports every entry
point that include/lbm_api.h declares; parameter validation needs no device."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "lbm_api.h")


@pytest.fixture(scope="module")
def L():
    from paper_2505_10899_gb300 import build
    build.build()
    from paper_2505_10899_gb300 import lbm
    return lbm


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*[\w\s\*]+?\b(lbm_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("lbm_init", "lbm_step", "lbm_volume", "lbm_adjoint_step",
                     "lbm_workspace_bytes", "lbm_destroy"):
        assert required in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(L):
    so = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(so, n)]
    assert not missing, missing


def test_params_struct_layout(L):
    # 6 int32 + 9 doubles + 2x9 rates + 2 doubles, no padding
    assert ctypes.sizeof(L.lbm_params) == 6 * 4 + 9 * 8 + 18 * 8 + 2 * 8
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
                dict(s_g=[1.0, 2.0] + [1.0] * 7)):
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


def test_status_strings(L):
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert L.lib().lbm_status_string(s)
