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


@pytest.mark.parametrize("variant,prec,shape,tiling",
                         [(5, "f16", (256, 64, 32), (64, 4, 8)),
                          (5, "f32", (128, 64, 32), (32, 8, 8)),
                          (4, "f32", (128, 16, 24), (128, 4, 8))],
                         ids=["strip-f16", "strip-f32", "whole-row-f32"])
def test_3d_bulk_copy_wait_timeout_is_reported_and_recoverable(variant, prec, shape, tiling):
    # The 3-D bulk-copy kernels wait for their staged planes with the same
    # bound.  At 0 cycles a CTA whose first stage has not landed when it
    # first polls gives up (hundreds of CTAs race their own copies there),
    # waits for its copies with the default bound and returns.  The status is
    # reported once; with the default bound and the saved state restored, the
    # run matches a reference run from the same state bit for bit.
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_10899_gb300 import build
    build.build()
    from paper_2505_10899_gb300 import lbm3
    nx, ny, nz = shape
    case = W.base_case3(nx, ny, nz, sigma=1e-2, rho_l=3.0, tau_f_l=0.7)
    phi0 = W.tanh_ball(nx, ny, nz, 0.5 * nx, 0.5 * ny, 0.5 * nz, 0.3 * min(nx, ny, nz), 4.0)
    s = lbm3.Sim3(case, phi0, None, precision=prec)
    s.set_tiling(*tiling)
    s.set_kernel(variant)
    assert s.kernel() == variant
    s.step(3)
    saved = s.get_state()
    s.set_state(*saved)
    s.step(6)
    ref = s.get_state()
    assert s.status() == lbm3.LBM_OK

    s.set_wait_limit(0)
    s.step(6)
    assert s.status() == L_ERR_TIMEOUT
    assert s.status() == lbm3.LBM_OK  # reported once, then cleared

    s.set_wait_limit(-1)  # default bound
    s.set_state(*saved)
    s.step(6)
    assert s.status() == lbm3.LBM_OK
    out = s.get_state()
    for a, b in zip(ref[:3], out[:3]):
        assert np.array_equal(a, b)
    s.close()


L_ERR_TIMEOUT = -5
