"""Parity at the benchmark's full size and launch configuration: all 512 batched
droplet cases (36.7 M nodes) advance together in the autotuned launch that
bench.py times; sampled cases are compared with the FP64 oracle run on that
case alone (cases are independent), and properties that hold at any size are
checked on every case."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_10899_gb300 import build
    build.build()
    from paper_2505_10899_gb300 import lbm
    return lbm


def test_batched_512_sampled_against_oracle(L):
    import torch
    cases = W.batched_droplets(512, seed=2026)
    phis, us = zip(*(W.case_fields(c) for c in cases))
    s = L.Sim(cases, list(phis), list(us), precision="f32")
    s.autotune(1)
    vol = s.track_volume(True)
    nsteps = 10
    s.step(nsteps)
    torch.cuda.synchronize()
    assert s.status() == L.LBM_OK
    # every case: tracked FP64 volume (state entering the last step) is finite
    # and within FP32 rounding of the initial sum of phi
    v = vol.cpu().numpy()
    v0 = np.array([p.sum() for p in phis])
    assert np.all(np.isfinite(v)) and np.abs(v / v0 - 1).max() < 1e-5
    # sampled cases: smallest and largest edges, extreme density ratios, ends
    edges = np.array([c["nx"] for c in cases])
    ratios = np.array([c["rho_l"] for c in cases])
    sample = sorted({0, 511, int(edges.argmin()), int(edges.argmax()),
                     int(ratios.argmin()), int(ratios.argmax())})
    for k in sample:
        o = oracle.Oracle(cases[k], phis[k], us[k]).step(nsteps)
        phi, ux, uy, p = s.fields(k)
        ophi, oux, ouy, op = o.fields()
        assert np.abs(phi - ophi).max() <= 1e-5, k
        assert np.abs(ux - oux).max() <= 1e-6 and np.abs(uy - ouy).max() <= 1e-6, k


def test_batched_512_fp32_volume_drift_1e4_steps(L):
    # The FP32 bar on the benchmark workload: every case's phase volume
    # (FP64 sum of the FP32 state, g_0 a float pair) stays within 1e-6
    # relative of its initial value over 10^4 steps.
    cases = W.batched_droplets(512, seed=2026)
    phis, us = zip(*(W.case_fields(c) for c in cases))
    s = L.Sim(cases, list(phis), list(us), precision="f32")
    s.autotune(1)
    v0 = s.volume().copy()
    s.step(10000)
    assert s.status() == L.LBM_OK
    v = s.volume()
    assert np.all(np.isfinite(v))
    assert np.abs(v / v0 - 1.0).max() <= 1e-6
