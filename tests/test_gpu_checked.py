"""GPU runs of the debug build with index checks (liblbm_gb300_checked.so):
every load and store of the 2-D step kernels and the range of every bulk copy
is checked against its array.  Runs of each kernel variant (bulk-copy,
register-pipelined, persistent; walls; vortex; a batch of uneven cases and
ragged strips) must raise no index flag and still match the FP64 oracle.
The checked library is loaded in a child process (LBM_GB300_CHECKED=1)."""
import os
import subprocess
import sys

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, ROOT)
import oracle
import workloads as W
from paper_2505_10899_gb300 import lbm
assert lbm.LIB_PATH.endswith("liblbm_gb300_checked.so")

def check(case, phi0, u0, n, prec, variant, tiling=None, tol=1e-12):
    s = lbm.Sim(case, phi0, u0, precision=prec)
    s.set_kernel(variant)
    if tiling:
        s.set_tiling(*tiling)
    s.step(n)
    assert s.status() == lbm.LBM_OK, "index flag raised"
    o = oracle.Oracle(case, phi0, u0).step(n)
    err = float(np.abs(s.fields(0)[0] - o.fields()[0]).max())
    assert err <= tol, (case["nx"], case["ny"], variant, err)
    s.close()

case, phi0, u0, _, _ = W.two_droplets(noise=1e-3)
for v in (1, 2):
    check(case, phi0, u0, 20, "f64", v)
    check(case, phi0, u0, 20, "f32", v, tol=1e-5)
check(case, phi0, u0, 12, "f64", 3)                      # persistent kernel
check(W.base_case(132, 37, rho_l=3.0), W.tanh_disc(132, 37, 60, 18, 9, 4.0, True), None,
      15, "f64", 2, (128, 5))                             # ragged strip and rows
check(W.base_case(36, 20, walls=1, u_top=0.01, u_bot=-0.01),
      W.tanh_disc(36, 20, 18, 10, 5, 4.0), None, 15, "f64", 1)
vc, vphi, _ = W.single_vortex(n=64, W=3.0, U=0.02, T=64)
check(vc, vphi, None, 16, "f64", 2)
specs = [(64, 64, 1.0), (192, 40, 4.0), (36, 52, 10.0), (4, 9, 2.0)]
cases, phis = [], []
for nx, ny, r in specs:
    cases.append(W.base_case(nx, ny, rho_l=r))
    phis.append(W.tanh_disc(nx, ny, nx / 2, ny / 2, min(nx, ny) / 4, 4.0, True))
s = lbm.Sim(cases, phis, None, precision="f32")
s.set_chains(2)
s.step(25)
assert s.status() == lbm.LBM_OK
for k, (c, p) in enumerate(zip(cases, phis)):
    o = oracle.Oracle(c, p).step(25)
    assert float(np.abs(s.fields(k)[0] - o.fields()[0]).max()) <= 1e-5
print("checked ok")
'''


def test_checked_build_raises_no_index_flag_and_matches_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_10899_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, LBM_GB300_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + SCRIPT], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]
