"""GPU test of lbm_phase_volume_noalloc, the phase-volume entry point for callers
that cannot allocate device memory (its scratch is a fixed static device array).

It must agree with the workspace-based lbm_volume, through the C ABI, on two
calls in a row with different region sets, and reject sizes beyond its limit.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL_VOL = 1e-13  # relative, as for the other FP64 volume comparisons


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_10899_gb300 import build
    build.build()
    from paper_2505_10899_gb300 import lbm
    return lbm


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_volume_matches_lbm_volume(L, prec):
    import torch
    case, phi0, u0, labels, _ = W.two_droplets(noise=1e-3)
    ny, nx = phi0.shape
    s = L.Sim(case, phi0, u0, precision=prec)
    s.step(37)
    f, g, j, t = s.get_state(0)  # post-streaming g_i(x, t), exact device values
    dtype = torch.float32 if prec == "f32" else torch.float64
    g_dev = torch.from_numpy(g).to(device="cuda", dtype=dtype).contiguous()
    lab_dev = torch.from_numpy(np.ascontiguousarray(labels)).to("cuda")
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    # call 1: two labelled droplet regions
    s.set_regions(0, labels, 2)
    ref1 = s.volume()
    out.fill_(float("nan"))
    L.lbm_phase_volume_noalloc(g_dev.data_ptr(), prec, nx, ny, nx * ny, lab_dev.data_ptr(), 2,
                               out.data_ptr(), stream)
    torch.cuda.synchronize()
    v1 = out[:2].cpu().numpy()
    # the planes as passed, summed in FP64 on the host
    gp = g_dev.double().cpu().numpy().sum(axis=0)
    exact1 = np.array([gp[labels == r].sum() for r in range(2)])
    assert np.all(np.abs(v1 / exact1 - 1.0) < TOL_VOL), (v1, exact1)
    # lbm_volume also counts the low part of the FP32 float pair g_0, which
    # the nine FP32 planes cannot carry: at most half an ulp of g_0 per node
    tol = TOL_VOL if prec == "f64" else 1e-6
    assert np.all(np.abs(v1 / ref1 - 1.0) < tol), (v1, ref1)

    # call 2, right after: one region (no labels), other output slot sizes
    s.set_regions(0, None, 1)
    ref2 = s.volume()
    out.fill_(float("nan"))
    L.lbm_phase_volume_noalloc(g_dev.data_ptr(), prec, nx, ny, nx * ny, 0, 1,
                               out.data_ptr(), stream)
    torch.cuda.synchronize()
    v2 = out[:1].cpu().numpy()
    assert abs(v2[0] / gp.sum() - 1.0) < TOL_VOL
    assert np.all(np.abs(v2 / ref2 - 1.0) < tol), (v2, ref2)
    assert abs(v1.sum() / v2[0] - 1.0) < TOL_VOL  # regions partition the grid


def test_noalloc_volume_rejects_sizes_beyond_its_limit(L):
    import torch
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    fake_g = torch.empty(16, dtype=torch.float32, device="cuda")
    with pytest.raises(L.LbmError) as e:   # 600000 columns > 4096 CTAs x 128 columns
        L.lbm_phase_volume_noalloc(fake_g.data_ptr(), "f32", 600000, 1, 600000, 0, 1,
                                   out.data_ptr(), 0)
    assert e.value.status == L.LBM_ERR_ARG and "static scratch" in str(e.value)
    with pytest.raises(L.LbmError):
        L.lbm_phase_volume_noalloc(fake_g.data_ptr(), "f32", 4, 4, 16, 0, 9, out.data_ptr(), 0)
