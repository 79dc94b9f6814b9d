"""The debug build with index checks (LBM_CHECK_BOUNDS) compiles and exports
the same entry points as the normal library (CPU: nvcc cross-compiles)."""
import ctypes
import os
import shutil

import pytest

from conftest import ROOT

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and
                                not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not found")


def _exports(path):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                         text=True).stdout
    return {ln.split()[-1] for ln in out.splitlines() if " T " in ln}


def test_checked_build_compiles_and_exports_the_abi():
    from paper_2505_10899_gb300 import build
    normal = build.build()
    checked = build.build(checked=True)
    assert os.path.basename(checked) == "liblbm_gb300_checked.so"
    a = {s for s in _exports(normal) if s.startswith("lbm")}
    b = {s for s in _exports(checked) if s.startswith("lbm")}
    assert a and a == b
