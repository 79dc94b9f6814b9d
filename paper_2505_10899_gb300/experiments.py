"""The experiments of Secs. 4.3 and 4.4 run through the GPU path, with the
host-side measurements that compare the modified model (lambda > 0, the
sharpening flux of Eq. 17) with the classical Cahn-Hilliard model
(lambda = 0), which is what the paper's comparison model solves.

Sec. 4.4 (droplet in a sheared cavity, 128 x 64, radius 8): the classical
model loses the droplet to the bulk by the coarsening that removes droplets
below a critical radius; the modified model keeps it.  Measured here as the
area enclosed by the phi = 1/2 contour over time.

Sec. 4.3 (perturbed liquid thread of Eq. 45): the thread necks where the
perturbation makes it thinnest, pinches off and leaves satellite droplets,
which the classical model dissolves and the modified model keeps.  Measured
as the phi > 1/2 connected components (number and sizes), the volume inside
phi = 1/2 and the thinnest cross-section over time.

Every step runs in the CUDA library (Sim, Sim3); the measurements read the
fields back and use numpy and scipy on the host.

    python -m paper_2505_10899_gb300.experiments [--quick]

runs both set-ups for lambda = 0.5 and 0 and prints one JSON line."""
from __future__ import annotations

import time

import numpy as np


def contour_measure(phi, up=4, periodic=True):
    """Area (2-D) or volume (3-D) enclosed by the phi = 1/2 level set: the
    count of phi > 1/2 samples of the multilinear interpolant on a grid
    refined `up` times per axis, in lattice units.  periodic=False clamps the
    interpolant at the grid edges instead of wrapping it."""
    from scipy import ndimage

    z = ndimage.zoom(np.asarray(phi, dtype=np.float64), up, order=1,
                     mode="grid-wrap" if periodic else "nearest", grid_mode=True)
    return float(np.count_nonzero(z > 0.5)) / up ** np.ndim(phi)


def components(mask, periodic_axes=None):
    """Face-connected components of a boolean field, joined across the
    periodic faces of `periodic_axes` (all axes by default).  Returns the
    component sizes in nodes, largest first."""
    from scipy import ndimage

    mask = np.asarray(mask, dtype=bool)
    lab, n = ndimage.label(mask)
    parent = np.arange(n + 1)

    def root(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    axes = range(mask.ndim) if periodic_axes is None else periodic_axes
    for ax in axes:
        lo, hi = np.take(lab, 0, axis=ax), np.take(lab, -1, axis=ax)
        both = (lo > 0) & (hi > 0)
        for p, q in set(zip(lo[both].tolist(), hi[both].tolist())):
            rp, rq = root(p), root(q)
            if rp != rq:
                parent[rp] = rq
    counts = np.bincount(lab.ravel(), minlength=n + 1)
    sizes = {}
    for i in range(1, n + 1):
        r = root(i)
        sizes[r] = sizes.get(r, 0) + int(counts[i])
    return sorted(sizes.values(), reverse=True)


def sheared_droplet(case, phi0, u0, times, precision="f32"):
    """Advance the Sec. 4.4 cavity to each of the increasing step counts in
    `times` and record (t, enclosed area, phi max, phi min, droplet count,
    wall-clock seconds so far)."""
    from . import lbm

    s = lbm.Sim(case, phi0, u0, precision=precision)
    rows, t, busy = [], 0, 0.0
    try:
        for t_next in times:
            t0 = time.perf_counter()
            s.step(t_next - t)
            phi = s.fields(0)[0]
            busy += time.perf_counter() - t0
            t = t_next
            rows.append(dict(t=t, area=contour_measure(phi),
                             drops=len(components(phi > 0.5, periodic_axes=(1,))),
                             phi_max=float(phi.max()), phi_min=float(phi.min()), seconds=busy))
        if s.status() != lbm.LBM_OK:
            raise lbm.LbmError(s.status(), "sheared_droplet", "non-finite state")
    finally:
        s.close()
    return rows


def film(case, phi0, times, precision="f32"):
    """Advance the two-dimensional film of Eq. 45 and record (t, number of
    phi > 1/2 components, thinnest and thickest column of liquid, i.e. the
    minimum and maximum over x of the sum of phi along y)."""
    from . import lbm

    s = lbm.Sim(case, phi0, None, precision=precision)
    rows, t = [], 0
    try:
        for t_next in times:
            s.step(t_next - t)
            t = t_next
            phi = s.fields(0)[0]
            height = phi.sum(axis=0)
            rows.append(dict(t=t, drops=len(components(phi > 0.5, periodic_axes=(1,))),
                             h_min=float(height.min()), h_max=float(height.max())))
        if s.status() != lbm.LBM_OK:
            raise lbm.LbmError(s.status(), "film", "non-finite state")
    finally:
        s.close()
    return rows


def column(case, phi0, times, precision="f32", autotune=True):
    """Advance the three-dimensional thread of Eq. 45 (axis along z) and
    record, at each step count in `times`: the phi > 1/2 components (count
    and the largest sizes in nodes), the nodes with phi > 1/2, the thinnest
    and thickest cross-section (sum of phi over a z plane), phi max and min,
    and the wall-clock seconds spent stepping and reading the fields back."""
    from . import lbm3

    s = lbm3.Sim3(case, phi0, None, precision=precision)
    rows, t, busy = [], 0, 0.0
    try:
        if autotune:
            s.autotune(1)
        for t_next in times:
            t0 = time.perf_counter()
            s.step(t_next - t)
            phi = s.fields()[0]
            busy += time.perf_counter() - t0
            t = t_next
            inside = phi > 0.5
            sizes = components(inside)
            section = phi.sum(axis=(1, 2))
            rows.append(dict(t=t, drops=len(sizes), sizes=sizes[:16],
                             inside=int(np.count_nonzero(inside)),
                             section_min=float(section.min()), section_max=float(section.max()),
                             phi_max=float(phi.max()), phi_min=float(phi.min()), seconds=busy))
        if s.status() != 0:
            raise lbm3.LbmError(s.status(), "column", "non-finite state")
    finally:
        s.close()
    return rows


def main(argv=None):
    """Both set-ups for lambda = 0.5 (modified) and 0 (classical); one JSON
    line on stdout.  --quick shortens the runs (a 96-node-wide column box,
    fewer steps) for a smoke check."""
    import argparse
    import json
    import sys

    sys.path.insert(0, __import__("os").path.dirname(__import__("os").path.dirname(__file__)))
    import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    a = ap.parse_args(argv)
    t_drop = [0, 5000, 10000, 20000, 40000, 80000, 160000, 240000, 320000, 400000]
    t_film = [0, 50000, 100000, 200000]
    t_col = list(range(0, 200001, 10000))
    side = None
    if a.quick:
        t_drop, t_film, t_col, side = t_drop[:5], t_film[:2], t_col[:4], 96
    res = {}
    for lam in (0.5, 0.0):
        c, p, u = W.coarse_sheared_droplet(lam=lam)
        res[f"sheared_droplet_128x64_lambda{lam}"] = sheared_droplet(c, p, u, t_drop, a.precision)
        c, p = W.film_eq45(lam=lam)
        res[f"film_eq45_256x128_lambda{lam}"] = film(c, p, t_film, a.precision)
        c, p = W.column_eq45(lam=lam, n_side=side)
        res[f"column_eq45_{c['nx']}x{c['ny']}x{c['nz']}_lambda{lam}"] = column(c, p, t_col, a.precision)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
