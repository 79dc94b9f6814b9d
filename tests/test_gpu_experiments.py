"""The Sec. 4.3 and 4.4 experiments on the GPU path: parity of their set-ups
with the FP64 oracle, and the paper's claims as measured outcomes of the
modified model (lambda = 0.5) against the classical Cahn-Hilliard model
(lambda = 0):

  * Sec. 4.4, a droplet of radius 8 in the 128 x 64 sheared cavity: the
    classical model dissolves it into the bulk, the modified model keeps the
    area enclosed by phi = 1/2;
  * Sec. 4.3, Eq. 45: on the 2-D Cartesian grid as printed the film does
    not break up (a flat film has no capillary instability), which is why
    the experiment runs as a 3-D thread; there the thread pinches off, and
    the classical model shrinks the satellite droplets and loses volume
    inside phi = 1/2 while the modified model keeps both."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_10899_gb300 import build
    build.build()
    from paper_2505_10899_gb300 import experiments
    return experiments


def md(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max())


@pytest.mark.parametrize("lam", [0.5, 0.0])
def test_coarse_sheared_droplet_fp64_parity(E, lam):
    from paper_2505_10899_gb300 import lbm
    case, phi0, u0 = W.coarse_sheared_droplet(lam=lam)
    s = lbm.Sim(case, phi0, u0, precision="f64").step(300)
    o = oracle.Oracle(case, phi0, u0).step(300)
    f, g, j, t = s.get_state(0)
    assert t == 300 and md(f, o.f) <= 1e-12 and md(g, o.g) <= 1e-12 and md(j, o.j) <= 1e-12
    assert md(s.fields(0)[0], o.fields()[0]) <= 1e-12


@pytest.mark.parametrize("lam", [0.5, 0.0])
def test_film_eq45_fp64_parity(E, lam):
    from paper_2505_10899_gb300 import lbm
    case, phi0 = W.film_eq45(lam=lam)
    s = lbm.Sim(case, phi0, None, precision="f64").step(50)
    o = oracle.Oracle(case, phi0).step(50)
    assert md(s.fields(0)[0], o.fields()[0]) <= 1e-12


def test_column_eq45_fp64_parity(E):
    # a 24-node-wide box keeps the oracle fast; the thread is 6 nodes thick.
    # Seeded noise of 1e-3 removes the symmetric zeros of grad psi on the
    # axis, where the unit normal of Eq. 17 would be set by rounding and the
    # two summation orders would pick different directions.
    from paper_2505_10899_gb300 import lbm3
    case, phi0 = W.column_eq45(lam=0.5, n_side=24)
    phi0 = phi0 + W.uniform(4545, phi0.shape, -1e-3, 1e-3)
    s = lbm3.Sim3(case, phi0, None, precision="f64")
    s.step(20)
    o = oracle.Oracle3(case, phi0).step(20)
    f, g, j, t = s.get_state()
    assert md(f, o.f) <= 1e-12 and md(g, o.g) <= 1e-12 and md(j, o.j) <= 1e-12
    assert md(s.fields()[0], o.fields()[0]) <= 1e-12


def test_coarse_sheared_droplet_classical_vanishes_modified_keeps(E):
    times = [0, 5000, 40000, 160000, 240000]
    area, drops = {}, {}
    for lam in (0.5, 0.0):
        case, phi0, u0 = W.coarse_sheared_droplet(lam=lam)
        rows = E.sheared_droplet(case, phi0, u0, times)
        area[lam] = np.array([r["area"] for r in rows])
        drops[lam] = [r["drops"] for r in rows]
    a0 = area[0.5][0]
    assert abs(a0 / (np.pi * 64) - 1) < 0.02
    # modified: after the initial profile settles (first 5000 steps) the
    # enclosed area moves by at most four refined samples
    assert np.abs(area[0.5][1:] - area[0.5][1]).max() <= 0.25
    assert abs(area[0.5][-1] / a0 - 1) < 0.01 and drops[0.5] == [1] * len(times)
    # classical: the area falls monotonically and the droplet is gone
    assert np.all(np.diff(area[0.0]) < 0)
    assert area[0.0][3] < 0.5 * a0 and drops[0.0][-1] == 0


def test_film_eq45_stays_whole_in_2d(E):
    for lam in (0.5, 0.0):
        case, phi0 = W.film_eq45(lam=lam)
        rows = E.film(case, phi0, [0, 50000])
        assert [r["drops"] for r in rows] == [1, 1]
        assert rows[1]["h_min"] > 0.95 * rows[0]["h_min"]
        assert rows[1]["h_max"] < rows[0]["h_max"]


@pytest.mark.slow
def test_column_eq45_satellites_kept_by_modified_model(E):
    # the 3-D thread of Eq. 45 in a 128-wide transverse box (FP32): both
    # models pinch off and leave satellites by step 50000; between then and
    # step 80000 the classical model shrinks the satellites and has lost
    # over 10% of the volume inside phi = 1/2, the modified model keeps
    # both.  Satellite sizes are compared as totals.
    res = {}
    for lam in (0.5, 0.0):
        case, phi0 = W.column_eq45(lam=lam, n_side=128)
        res[lam] = E.column(case, phi0, [0, 50000, 80000])
    for lam, rows in res.items():
        assert rows[0]["drops"] == 1 and rows[1]["drops"] >= 3 and rows[2]["drops"] >= 3
        assert rows[2]["phi_max"] < 1.1 and rows[2]["phi_min"] > -0.01
    sat = {lam: [sum(r["sizes"][1:]) for r in rows] for lam, rows in res.items()}
    vol = {lam: [r["inside"] / rows[0]["inside"] for r in rows] for lam, rows in res.items()}
    assert abs(vol[0.5][2] - 1) < 0.04 and abs(sat[0.5][2] / sat[0.5][1] - 1) < 0.02
    assert vol[0.0][2] < 0.9 and sat[0.0][2] < 0.98 * sat[0.0][1]
    assert sat[0.5][2] > 1.5 * sat[0.0][2]
