"""The N > 1 path of bench.py on CPU: two gloo ranks each own an independent,
differently seeded batch; the only communication is the barrier and the
max-over-ranks timing reduction."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

from conftest import ROOT  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench

    class A:
        ncases, seed = 6, 2026

    ws, r, local, pg = bench.dist_setup(A)
    cases = bench.rank_cases(A, r)
    sig = [(c["nx"], round(c["R"], 6), round(c["rho_l"], 6)) for c in cases]
    t_max = bench.max_over_ranks(pg, 10.0 + 5.0 * r, "cpu")
    pg.barrier()
    out[r] = (ws, sig, t_max, bench.whole_job_mlups(ws, 1000, 10, t_max))
    pg.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (ws0, sig0, t0, v0), (ws1, sig1, t1, v1) = out[0], out[1]
    assert ws0 == ws1 == 2
    assert sig0 != sig1                        # independent batches per rank
    assert t0 == t1 == 15.0                    # max over ranks
    assert v0 == v1 == pytest.approx(2 * 1000 * 10 / 15e-3 / 1e6)


def _partition_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    import workloads as W

    class A:
        ncases, seed = 512, 2026

    ws, r, local, pg = bench.dist_setup(A)
    cases = W.batched_droplets(512, seed=2026)
    mine = bench.partition_cases(cases, ws, r)
    vols = [1000.0 + i + 0.25 for i in mine]   # stand-in per-case volumes
    full = bench.gather_case_volumes(pg, mine, vols, len(cases), "cpu")
    pg.barrier()
    out[r] = (mine, sum(cases[i]["nx"] * cases[i]["ny"] for i in mine), full.tolist())
    pg.destroy_process_group()


def test_two_gloo_ranks_partition_one_batch():
    """--partition: the 512 cases of one batch are split over two ranks,
    balanced by node count to within one case; the per-case volumes are
    all-gathered back into case order on every rank."""
    import numpy as np
    import workloads as W
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_partition_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    (m0, n0, f0), (m1, n1, f1) = out[0], out[1]
    assert sorted(m0 + m1) == list(range(512)) and not set(m0) & set(m1)
    cases = W.batched_droplets(512, seed=2026)
    biggest = max(c["nx"] * c["ny"] for c in cases)
    assert abs(n0 - n1) <= biggest
    assert n0 + n1 == sum(c["nx"] * c["ny"] for c in cases)
    expect = 1000.0 + np.arange(512) + 0.25
    assert np.array_equal(np.asarray(f0), expect) and np.array_equal(np.asarray(f1), expect)
