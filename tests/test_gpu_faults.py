"""Failure detection without a GPU fault: bounded device waits that run out.

With the wait limit set to 0 cycles (lbm_set_wait_limit), the bulk-copy
kernel's first wait for a staged row and the persistent kernel's grid
barrier give up at their first poll.  The kernels raise LBM_ERR_TIMEOUT,
wait (with the default bound) for the copies they issued, and return; no
wait is left unbounded and nothing faults.  The status is reported once and
cleared, and the context stays usable: with the default limit restored and
the checkpoint reloaded, the run reproduces the reference bit for bit.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_10899_gb300 import build
    build.build()
    from paper_2505_10899_gb300 import lbm
    return lbm


@pytest.mark.parametrize("variant,shape", [(2, (256, 128)), (3, (128, 64))],
                         ids=["bulk-copy-waits", "persistent-grid-barrier"])
def test_device_wait_timeout_is_reported_and_recoverable(L, variant, shape):
    nx, ny = shape
    case = W.base_case(nx, ny, rho_l=2.0)
    phi0 = W.tanh_disc(nx, ny, nx / 2, ny / 2, ny / 4, 4.0, periodic=True)
    s = L.Sim(case, phi0, None, precision="f32")
    s.set_kernel(variant)
    assert s.kernel() == variant
    # four warps per CTA: warps 1-3 test the first staged row while warp 0
    # is still issuing its copies
    s.set_tiling(128, 16)
    s.step(3)
    blob = s.save()
    s.step(6)
    ref = s.get_state(0)
    assert s.status() == L.LBM_OK

    s.load(blob)
    L.lbm_set_wait_limit(s.h, 0)
    s.step(6)
    assert s.status() == L.LBM_ERR_TIMEOUT
    assert s.status() == L.LBM_OK  # reported once, then cleared

    L.lbm_set_wait_limit(s.h, -1)  # default bound
    s.load(blob)
    s.step(6)
    assert s.status() == L.LBM_OK
    out = s.get_state(0)
    for a, b in zip(ref[:3], out[:3]):
        assert np.array_equal(a, b)
    s.close()
