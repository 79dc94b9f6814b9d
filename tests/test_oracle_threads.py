"""The oracles' OpenMP loops give the same bits with one thread as with all
host cores (each node is computed by one thread; nothing is reduced across
nodes), so the timed multi-core baseline is the same computation as the
single-core one."""
import numpy as np

import oracle
import workloads as W


def _run2(threads):
    oracle.set_num_threads(threads)
    case, phi0, u0, _, _ = W.two_droplets(noise=1e-3)
    o = oracle.Oracle(dict(case, rho_l=3.0, tau_f_l=0.7), phi0, u0).step(25)
    return o.f.copy(), o.g.copy(), o.j.copy()


def _run3(threads):
    oracle.set_num_threads(threads)
    case = W.base_case3(20, 12, 10, sigma=1e-2, rho_l=3.0, tau_f_l=0.7)
    f, g, j = W.random_state3(20, 12, 10, seed=5, phi_lo=0.1, phi_hi=0.9)
    o = oracle.Oracle3(case, state=(f, g, j, 0)).step(10)
    return o.f.copy(), o.g.copy(), o.j.copy()


def test_thread_count_does_not_change_the_bits():
    n = oracle.num_threads()
    try:
        for run in (_run2, _run3):
            one = run(1)
            many = run(max(n, 2))
            for a, b in zip(one, many):
                assert np.array_equal(a, b)
    finally:
        oracle.set_num_threads(n)
