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


@pytest.mark.parametrize("prec,nx,ny,pad", [("f32", 200, 3000, 64), ("f64", 200, 3000, 64),
                                           ("f32", 300, 20000, 0), ("f64", 131, 5, 3)])
def test_noalloc_volume_ragged_strips_and_row_runs(L, prec, nx, ny, pad):
    """Several 128-column strips with a ragged last one, more rows than CTA
    slots (each CTA sums a run of rows), a padded plane stride, and labels
    in {-1, 0, 1, 2}: every region against a host FP64 sum of the planes as
    passed, on two calls in a row (labelled, then one region)."""
    import torch
    stride = nx * ny + pad
    dtype = torch.float32 if prec == "f32" else torch.float64
    g = W.uniform(4242 + nx, (9 * stride,), 0.0, 0.2)
    g_dev = torch.from_numpy(g).to(device="cuda", dtype=dtype).contiguous()
    lab = (W.splitmix64(77 + ny, nx * ny) % np.uint64(4)).astype(np.int8) - np.int8(1)
    lab_dev = torch.from_numpy(lab).to("cuda")
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    gp = g_dev.double().cpu().numpy().reshape(9, stride)[:, :nx * ny].sum(axis=0)
    exact = np.array([gp[lab == r].sum() for r in range(3)])
    for _ in range(2):
        out.fill_(float("nan"))
        L.lbm_phase_volume_noalloc(g_dev.data_ptr(), prec, nx, ny, stride, lab_dev.data_ptr(),
                                   3, out.data_ptr(), stream)
        torch.cuda.synchronize()
        v = out[:3].cpu().numpy()
        assert np.all(np.abs(v / exact - 1.0) < TOL_VOL), (v, exact)
        out.fill_(float("nan"))
        L.lbm_phase_volume_noalloc(g_dev.data_ptr(), prec, nx, ny, stride, 0, 1,
                                   out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert abs(out[0].item() / gp.sum() - 1.0) < TOL_VOL


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
