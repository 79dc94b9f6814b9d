#!/usr/bin/env python3
"""Benchmark of the coupled volume-conserving LB step on GB300.

Default workload: 512 independent 2-D droplet cases advanced together, one
kernel launch per time step over all of them (static and translating droplets,
square edges drawn from {64, ..., 512}, density ratio 1:1 to 1:10, W = 4,
FP32 populations, FP64 phase-volume sums fused into the step).  A bench "step"
is one coupled LB time step of every case: pull-stream, phi/psi, isotropic
stencils, chemical potential and surface force, hydrodynamic and phase-field
MRT collisions, phi*u update and the per-case FP64 volume reduction.

metric: MLUPS (million lattice-node updates per second, whole job).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun) every rank advances its own independent batch (weak
scaling); the only communication is the barrier and the max-time reduction.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

BYTES_PER_NODE = {"f32": 160, "f64": 320}  # f, g read+write, phi*u read+write
# 3-D: 19 f + 7 g read+write, phi*u (3) read+write; FP16 storage keeps phi*u in FP32
BYTES_PER_NODE_3D = {"f32": 232, "f16": 128, "f64": 464}
WORKLOAD_NAME = ("batched droplets: 512 independent 2-D cases, square edges from "
                 "{64,96,128,192,256,384,512}, R in [0.05,0.3]*edge, translation "
                 "speed in [0,0.02] lu/step, density ratio 1:1..1:10, W=4, "
                 "coupled D2Q9 MRT phase-field + hydrodynamic LB")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["f32", "f64"], default="f32")
    ap.add_argument("--ncases", type=int, default=512)
    ap.add_argument("--partition", action="store_true",
                    help="N > 1: split one batch over the ranks instead of one batch per rank")
    ap.add_argument("--seed", type=int, default=2026)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--kernel", type=int, default=0, help="0 auto, 1 register, 2 bulk-copy")
    ap.add_argument("--tiling", type=str, default=None, help="BX,ROWS (default: autotuned)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--chains", type=int, default=0,
                    help="independent case groups as parallel graph branches (0: library default)")
    ap.add_argument("--only-3d", action="store_true",
                    help="only the 3-D Rayleigh-Plateau numbers (D3Q19 + D3Q7)")
    ap.add_argument("--grid3", type=str, default="256,256,1024", help="NX,NY,NZ of the 3-D box")
    ap.add_argument("--prec3", type=str, default="f32,f16,f64", help="3-D storage precisions")
    ap.add_argument("--steps3", type=int, default=50, help="timed 3-D steps (FP64: a fifth)")
    ap.add_argument("--tiling3", type=str, default=None,
                    help="VARIANT,BX,BY,ZC for the 3-D step (default: autotuned)")
    ap.add_argument("--only-shear", action="store_true",
                    help="only the sheared-droplet numbers (walls, FP32/FP64, D gradient)")
    ap.add_argument("--only-lattice", action="store_true",
                    help="only the droplet-lattice grid (one large case)")
    ap.add_argument("--lattice", type=str, default="16384,8192",
                    help="NX,NY of the droplet-lattice grid (multiples of 256)")
    ap.add_argument("--only-batching", action="store_true",
                    help="only the batched-vs-separate-handles comparison")
    ap.add_argument("--only-adjoint", action="store_true",
                    help="print the reverse-mode timings only (profiling aid)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return ws, rank, local, pg


def max_over_ranks(pg, value, device):
    """Max of a per-rank scalar over all ranks (timing plumbing only)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world_size, nodes_per_rank, steps, t_max_ms):
    """Weak scaling: every rank updates its own nodes each step."""
    return world_size * nodes_per_rank * steps / (t_max_ms * 1e-3) / 1e6


def rank_cases(args, rank):
    """Each rank owns an independent batch (seeded by rank)."""
    return W.batched_droplets(args.ncases, seed=args.seed + 7919 * rank)


def partition_cases(cases, world, rank):
    """Indices of the cases that rank `rank` advances when one batch is split
    over `world` ranks (--partition): cases taken largest first, each dealt
    to the rank with the fewest nodes so far (ties to the lowest rank), so
    the ranks' node counts differ by at most one case."""
    order = sorted(range(len(cases)), key=lambda i: (-cases[i]["nx"] * cases[i]["ny"], i))
    load = [0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += cases[i]["nx"] * cases[i]["ny"]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def gather_case_volumes(pg, idx, vols, ncases, device):
    """The per-case FP64 volumes of all ranks, in case order (all-gather of
    (index, volume) pairs, padded to the longest list)."""
    import torch
    n = torch.tensor([len(idx)], dtype=torch.int64, device=device)
    sizes = [torch.zeros_like(n) for _ in range(pg.get_world_size())]
    pg.all_gather(sizes, n)
    m = int(max(int(x.item()) for x in sizes))
    buf = torch.full((m, 2), -1.0, dtype=torch.float64, device=device)
    if len(idx):
        buf[:len(idx), 0] = torch.tensor(idx, dtype=torch.float64)
        buf[:len(idx), 1] = torch.as_tensor(np.asarray(vols, dtype=np.float64))
    out = [torch.empty_like(buf) for _ in range(pg.get_world_size())]
    pg.all_gather(out, buf)
    full = np.full(ncases, np.nan)
    for t in out:
        t = t.cpu().numpy()
        for k, v in t:
            if k >= 0:
                full[int(k)] = v
    return full


def host_inputs(cases):
    phis, us = [], []
    for c in cases:
        phi, u = W.case_fields(c)
        phis.append(phi)
        us.append(u)
    return phis, us


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "power_w_max": float(max(power)), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2505_10899_gb300", "csrc")
    for name in ("lbm_kernels_tma.cuh", "lbm_node.cuh", "lbm_tma.cuh", "lbm_layout.h"):
        h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag, nodes):
    """DRAM bytes per launch scaled from the committed ncu summary, or None if
    the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    if not os.path.exists(path):
        return None, None
    txt = open(path).read()
    m_h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"dram_bytes_per_node:\s*([0-9.]+)", txt)
    if not m_h or not m_b:
        return None, None
    if m_h.group(1) != kernel_source_hash():
        return None, "stale"
    return float(m_b.group(1)) * nodes, "scaled"


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    from paper_2505_10899_gb300 import lbm

    ws, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    if args.partition:
        # one batch split over the ranks (strong scaling)
        all_cases = rank_cases(args, 0)
        mine = partition_cases(all_cases, ws, rank)
        cases = [all_cases[i] for i in mine]
        total_nodes = sum(c["nx"] * c["ny"] for c in all_cases)
    else:
        cases = rank_cases(args, rank)
    nodes = sum(c["nx"] * c["ny"] for c in cases)
    phis, us = host_inputs(cases)

    with torch.cuda.stream(stream):
        sim = lbm.Sim(cases, phis, us, precision=args.precision, stream=stream)
        sim.set_kernel(args.kernel)
        if args.chains:
            sim.set_chains(args.chains)
        tuned = None
        if args.tiling:
            bx, rows = (int(v) for v in args.tiling.split(","))
            sim.set_tiling(bx, rows)
        elif not args.no_autotune and args.kernel == 0:
            tuned = sim.autotune(2)   # part of the warm-up; the state is unchanged
        vol = sim.track_volume(True)
        v0 = None
        sim.step(max(args.warmup, 3))
        K = args.steps
        # capture the step graphs of the timed call now (no step runs)
        sim.prepare(K)
        stream.synchronize()
        v0 = vol.clone()

        # ---------------- timed region ----------------
        # one lbm_step(K) call: graphs of up to 64 steps, one branch per chain
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        sampler = ClockSampler(local) if rank == 0 else None
        if pg:
            pg.barrier()
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.start()
            time.sleep(0.4)
        ev[0].record(stream)
        sim.step(K)
        ev[1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize(dev)
        if pg:
            pg.barrier()
        clocks = sampler.stop() if sampler else None
        total_ms = ev[0].elapsed_time(ev[1])
        status = sim.status()
        nchains = sim.chains()
        vend = vol.clone().cpu().numpy()
        drift = float(np.max(np.abs(vend / v0.cpu().numpy() - 1.0)))

    t_max = max_over_ranks(pg, total_ms, dev) if pg else total_ms
    if args.partition:
        value = total_nodes * K / (t_max * 1e-3) / 1e6
        vols_all = gather_case_volumes(pg, mine, vend, len(all_cases), dev) if pg else vend
    else:
        value = whole_job_mlups(ws, nodes, K, t_max)

    # time per step: the K steps run as graphs whose branches (one per chain)
    # each hold the step kernel and the volume finalisation of their cases,
    # plus one clock kernel per graph
    kms = total_ms / K
    bpn = BYTES_PER_NODE[args.precision]
    achieved = bpn * nodes / (kms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    tag = f"coupled_step_{args.precision}_batched512"
    traffic, traffic_kind = profiled_traffic(tag, nodes)

    result = {
        "metric": "coupled-step MLUPS",
        "value": round(value, 1),
        "unit": "MLUPS",
        "n_gpus": ws,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(t_max / K, 4),
        "higher_is_better": True,
        "scaling": "strong" if args.partition else "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.precision == "f32" else "f64",
        "data": "synthetic (seeded tanh droplets; no dataset in the paper)",
        "config": {"workload": WORKLOAD_NAME, "ncases": len(cases), "nodes_per_gpu": nodes,
                   "precision": args.precision, "volume_sums": "f64, fused, every step",
                   "l2": "inputs larger than L2 (%.1f GB of state)" % (
                       sim.ws_bytes / 1e9),
                   "parallelism": (f"one batch of {args.ncases} cases split over {ws} "
                                   "rank(s), balanced by nodes; per-case volumes all-gathered"
                                   if args.partition else
                                   f"independent batches, {ws} rank(s)"),
                   "chains": nchains,
                   "tiling": "strip/run work items; the cases in %d chains, each chain one "
                             "step-kernel launch per step, chains as parallel CUDA-graph "
                             "branches" % nchains},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "traffic_source": traffic_kind,
                     "kernel": ("step_kernel_tma" if sim.kernel() == 2 else "step_kernel")
                               + f"<{'float' if args.precision == 'f32' else 'double'},"
                               f"{sim_bx(sim)},coupled>",
                     "tiling": {"bx": sim.tiling()[0], "rows": sim.tiling()[1],
                                "ctas": sim.tiling()[2],
                                "chosen_by": "autotune" if tuned else "fixed"},
                     "algorithmic_bytes_per_node": bpn, "peak_kind": peak_kind,
                     "kernel_ms": round(kms, 4)},
        "clocks": clocks,
        "gpu_launches": 2 * nchains * K + (K + 63) // 64,
        "status": status,
        "volume_drift_rel": drift,
    }
    if args.partition:
        result["partition"] = {"cases_this_rank": len(cases), "nodes_this_rank": nodes,
                               "volumes_gathered": int(np.isfinite(vols_all).sum()),
                               "ncases": len(all_cases)}
    e2e_tiling = tuple(sim.tiling()[:2])
    sim.close()
    del sim
    torch.cuda.empty_cache()

    if rank == 0 and not args.no_e2e:
        result["e2e"] = run_e2e(args, cases, phis, us, dev, K, tiling=e2e_tiling)
    if rank == 0 and not args.no_extras:
        ex = run_extras(args, cases, dev)
        result["extras"] = ex
        # the secondary headline ratios, also at the top level of the line
        result.update(headline_ratios(ex))
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(cases, args.cpu_seconds)
    if pg:
        pg.barrier()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if pg:
        pg.destroy_process_group()


def fp64_peak(dev):
    """Measured FP64 FMA rate of this GPU (lbm_fp64_fma_rate: 8 independent
    FMA chains per thread, 4 CTAs of 256 threads per SM), timed for about
    0.4 s with the SM clock sampled meanwhile."""
    from paper_2505_10899_gb300 import lbm
    import torch
    _, ms = lbm.lbm_fp64_fma_rate(2000, 4)
    trips = max(2000, int(2000 * 400.0 / max(ms, 1e-3)))
    smp = ClockSampler(dev.index if dev.index is not None else 0)
    smp.start()
    time.sleep(0.3)
    rate, ms = lbm.lbm_fp64_fma_rate(trips, 4)
    clocks = smp.stop()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    per_clk = None
    if clocks.get("sm_mhz"):
        per_clk = rate / (clocks["sm_mhz"] * 1e6 * sms)
    # the pipe's rate: FP64 FMAs per cycle per SM from ncu's peak_sustained of
    # sm__sass_thread_inst_executed_op_dfma_pred_on (committed summary) x SMs
    # x the SM clock sampled during the probe
    derived = None
    path = os.path.join(ROOT, "profiles", "coupled_step_f64_batched16.md")
    if os.path.exists(path) and clocks.get("sm_mhz"):
        m = re.search(r"fp64_fma_per_cycle_per_sm:\s*([0-9.]+)", open(path).read())
        if m:
            derived = float(m.group(1)) * sms * clocks["sm_mhz"] * 1e6
    return {"fma_per_s": rate, "tflops": round(2 * rate / 1e12, 4), "timed_ms": round(ms, 2),
            "sms": sms, "fma_per_clock_per_sm": per_clk, "clocks": clocks,
            "derived_fma_per_s": derived,
            "probe_frac_of_derived": None if not derived else round(rate / derived, 4),
            "how": "lbm_fp64_fma_rate: 8 independent FMA chains per thread, "
                   "4 x 256 threads per SM, CUDA events"}


def fp64_roofline(tag, nodes, ms_per_launch, peak):
    """FP64 launches are bound by the FP64 pipe, not by HBM: achieved = FP64
    pipe instructions per node (warp instructions x 32 from the committed
    ncu summary, which also gives the pipe's busy fraction) x nodes / the
    launch time, against the measured FMA rate (one FP64 pipe instruction
    per FMA)."""
    path = os.path.join(ROOT, "profiles", f"{tag}.md")
    per_node = None
    pipe = None
    if os.path.exists(path):
        txt = open(path).read()
        m = re.search(r"fp64_pipe_inst_per_node:\s*([0-9.]+)", txt)
        per_node = float(m.group(1)) if m else None
        m = re.search(r"fp64_pipe_busy_pct:\s*([0-9.]+)", txt)
        pipe = float(m.group(1)) if m else None
    derived = peak.get("derived_fma_per_s")
    pk = (derived if derived else peak["fma_per_s"]) / 1e9
    kind = ("derived: FP64 FMAs per cycle per SM (ncu peak_sustained) x SMs x sampled SM "
            "clock" if derived else "measured (lbm_fp64_fma_rate)")
    if per_node is None:
        return {"bound": "fp64_alu", "achieved": None, "peak": round(pk, 2),
                "unit": "G FP64 inst/s", "frac": None, "note": "no committed instruction count"}
    ach = per_node * nodes / (ms_per_launch * 1e-3) / 1e9
    return {"bound": "fp64_alu", "achieved": round(ach, 2), "peak": round(pk, 2),
            "unit": "G FP64 inst/s", "frac": round(ach / pk, 4),
            "fp64_inst_per_node": per_node, "ncu_fp64_pipe_busy_pct": pipe,
            "peak_kind": kind, "probe_fma_per_s_g": round(peak["fma_per_s"] / 1e9, 2)}


def headline_ratios(ex):
    """Compact copies of the secondary ratios the metric names: batching
    against separate per-case launches, the adjoint step against the forward
    step, the whole reverse-mode gradient against the forward run (FP64 and
    FP32), and the FP64 step against the FP64 pipe's measured peak."""
    out = {}

    def get(*path):
        o = ex
        for k in path:
            if not isinstance(o, dict) or k not in o:
                return None
            o = o[k]
        return o

    out["batching_speedup_vs_launch_per_case"] = get(
        "batching", "speedup_vs_launch_per_case_per_step")
    out["batching_speedup_vs_graph_per_case"] = get("batching", "speedup_vs_graph_per_case")
    out["adjoint_step_over_forward"] = get("adjoint", "vjp_over_forward")
    out["adjoint_step_over_forward_f32"] = get("adjoint_sweep_shear", "f32",
                                               "adjoint_over_forward")
    out["adjoint_step_over_forward_f64"] = get("adjoint_sweep_shear", "f64",
                                               "adjoint_over_forward")
    out["adjoint_backward_over_forward_recorded"] = get(
        "adjoint", "backward_states_recorded", "backward_over_forward_step")
    out["gradient_over_forward_f64"] = get("shear_droplet", "gradient_f64",
                                           "backward_over_plain_forward")
    out["gradient_over_forward_f32"] = get("shear_droplet", "gradient_f32",
                                           "backward_over_plain_forward")
    out["fp64_step_fp64_pipe_frac"] = get("f64_first64cases", "roofline", "frac")
    out["fp64_peak_tflops"] = get("fp64_peak", "tflops")
    return out


def sim_bx(sim):
    return sim.tiling()[0]


def run_e2e(args, cases, phis, us, dev, K, tiling=None):
    """End to end through the public API: H2D of the initial fields from
    pinned host memory (one copy of the host arena into device memory, then
    lbm_init from the device copy), the tiling of the device-timed run set
    through lbm_set_tiling, K steps, and every step the per-case volumes
    (the step's result) delivered to host memory and read by the host.
    Beside it (init_reads_pinned_arena): lbm_init reading the pinned host
    arena in place, without the copy.

    Main number: the volumes go to a page-locked host history of K slots
    (lbm_track_volume_history), which the step's final reduction kernel
    writes directly every step; the K steps are one lbm_step call; the host
    reads all K slots after the stream has drained, inside the clock.
    Second number (host_loop): one lbm_step(h, 1) per step and a copy of
    the volumes into pinned memory after each, read by the host one step
    behind (double-buffered); each step then waits for all chains of the
    previous one."""
    import torch
    from paper_2505_10899_gb300 import lbm

    stream = torch.cuda.Stream(device=dev)
    # The initial fields sit in one page-locked arena, the way a caller keeps
    # its staging buffers: lbm_init reads one large pinned allocation faster
    # than 1,024 separately pinned arrays (7.2 against 8.2 ms for the batch).
    total = sum(p.size for p in phis) + sum(u.size for u in us)
    arena_t = torch.empty(total, dtype=torch.float64, pin_memory=True)
    arena = arena_t.numpy()
    # the same arena in device memory, allocated before the clock: the staged
    # form copies the host arena there with one copy-engine transfer inside
    # the clock and lets lbm_init read the device copy
    dev_arena = torch.empty(total, dtype=torch.float64, device=dev)
    pin_phi, pin_u, dev_phi, dev_u, off = [], [], [], [], 0
    for p, u in zip(phis, us):
        for src, dst, ddst in ((p, pin_phi, dev_phi), (u, pin_u, dev_u)):
            v = arena[off:off + src.size].reshape(src.shape)
            v[...] = src
            dst.append(v)
            ddst.append(dev_arena.data_ptr() + 8 * off)
            off += src.size
    params = [lbm.make_params(c, args.precision) for c in cases]
    nbytes = lbm.lbm_workspace_bytes(params)
    wsbuf = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    ptr = (wsbuf.data_ptr() + 255) // 256 * 256
    nc = len(cases)
    nodes = sum(c["nx"] * c["ny"] for c in cases)
    h2d = total * 8

    def init(staged=True):
        if staged:  # one H2D copy of the whole arena, then init from device memory
            with torch.cuda.stream(stream):
                dev_arena.copy_(arena_t, non_blocking=True)
            h = lbm.lbm_init(params, ptr, nbytes, dev_phi, dev_u, stream.cuda_stream)
        else:  # the init kernel reads the pinned arena in place over the CPU-GPU link
            h = lbm.lbm_init(params, ptr, nbytes, pin_phi, pin_u, stream.cuda_stream)
        if tiling:
            lbm.lbm_set_tiling(h, *tiling)
        return h

    # main: per-step volumes written to a pinned host history by the kernels
    hist = torch.zeros((K, nc), dtype=torch.float64).pin_memory()

    def run_hist(staged):
        hist.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h = init(staged)
        lbm.lbm_track_volume_history(h, hist.data_ptr(), K)
        lbm.lbm_step(h, K)
        stream.synchronize()
        vols = hist.numpy().copy()  # the host reads every step's volumes
        t1 = time.perf_counter()
        lbm.lbm_destroy(h)
        return t1 - t0, bool(np.isfinite(vols).all() and vols.min() > 0)

    t_direct, ok_direct = run_hist(False)
    t_main, ok_hist = run_hist(True)
    ok_hist = ok_hist and ok_direct

    # second: one call per step, volumes copied and read one step behind
    vol_d = torch.zeros(nc, dtype=torch.float64, device=dev)
    vol_h = [torch.zeros(nc, dtype=torch.float64).pin_memory() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    total = np.zeros(nc)
    torch.cuda.synchronize(dev)
    u0 = time.perf_counter()
    h = init()
    lbm.lbm_track_volume(h, vol_d.data_ptr())
    for k in range(K + 1):
        if k < K:
            lbm.lbm_step(h, 1)
            with torch.cuda.stream(stream):
                vol_h[k & 1].copy_(vol_d, non_blocking=True)
                done[k & 1].record(stream)
        if k > 0:  # the host reads the volumes of step k-1
            done[(k - 1) & 1].synchronize()
            total += vol_h[(k - 1) & 1].numpy()
    u1 = time.perf_counter()
    lbm.lbm_destroy(h)
    return {"value": round(nodes * K / t_main / 1e6, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": int(h2d / K), "d2h_bytes_per_step": nc * 8,
            "tiling": list(tiling) if tiling else "default",
            "volumes_read": ok_hist and bool(np.isfinite(total).all() and total.min() > 0),
            "includes": "one H2D copy of the pinned host arena of phi0, u0 into device "
                        "memory, lbm_init from that copy, lbm_set_tiling, "
                        "lbm_track_volume_history (pinned host history of K slots), one "
                        "lbm_step(K) call whose kernels write each step's per-case volumes to "
                        "the host history, stream sync, host read of all K slots",
            "init_reads_pinned_arena": {
                "value": round(nodes * K / t_direct / 1e6, 1),
                "includes": "as above, but lbm_init reads phi0, u0 from the pinned host "
                            "arena in place over the CPU-GPU link (no copy)"},
            "host_loop": {"value": round(nodes * K / (u1 - u0) / 1e6, 1),
                          "includes": "as the main figure, but K x (lbm_step(h, 1) + D2H copy of the "
                                      "per-case volumes into pinned memory, read by the host "
                                      "one step behind)"}}


def run_extras(args, cases, dev):
    """Secondary numbers: FP64 on a slice of the batch; FP32 vs FP64 on the
    two-droplet case; the single-vortex period (256^2, T = 16384 steps) in
    FP32 and FP64 with its shape error and volume drift."""
    import torch
    from paper_2505_10899_gb300 import lbm

    def timed(sim, n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(sim.stream)
        sim.step(n)
        b.record(sim.stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b)

    out = {}
    out["fp64_peak"] = fp64_peak(dev)
    sub = cases[:64]
    nodes = sum(c["nx"] * c["ny"] for c in sub)
    phis, us = host_inputs(sub)
    for prec in ("f64", "f32"):
        s = lbm.Sim(sub, phis, us, precision=prec)
        s.autotune(1)
        s.step(3)
        s.prepare(20)
        torch.cuda.synchronize(dev)
        ms = timed(s, 20)
        out[f"{prec}_mlups_first64cases"] = round(nodes * 20 / (ms * 1e-3) / 1e6, 1)
        if prec == "f64":
            out["f64_first64cases"] = {
                "mlups": out["f64_mlups_first64cases"], "ms_per_step": round(ms / 20, 4),
                "tiling": list(s.tiling()[:2]), "kernel": s.kernel(),
                "roofline": fp64_roofline("coupled_step_f64_batched16", nodes, ms / 20,
                                          out["fp64_peak"])}
        s.close()
    # FP32 vs FP64 on the two-droplet case (128x64, 100 steps)
    case, phi0, u0, _, _ = W.two_droplets(noise=1e-3)
    res = {}
    for prec in ("f32", "f64"):
        s = lbm.Sim(case, phi0, u0, precision=prec)
        s.step(100)
        res[prec] = s.fields(0)[0]
        s.close()
    out["two_droplets_phi_maxdiff_f32_vs_f64_100steps"] = float(
        np.abs(res["f32"] - res["f64"]).max())
    # single vortex, one full period
    vcase, vphi0, _ = W.single_vortex(n=256, W=3.0, U=0.02, T=16384)
    vort = {"grid": "256x256", "period_steps": 16384}
    fin = {}
    for prec in ("f32", "f64"):
        s = lbm.Sim(vcase, vphi0, None, precision=prec)
        s.autotune(1)
        v0 = s.volume()[0]
        ms = timed(s, 16384)
        phi = s.fields(0)[0]
        fin[prec] = phi
        vort[f"{prec}_kernel"] = {"variant": s.kernel(), "bx": s.tiling()[0], "rows": s.tiling()[1]}
        vort[f"{prec}_mlups"] = round(256 * 256 * 16384 / (ms * 1e-3) / 1e6, 1)
        vort[f"{prec}_shape_error"] = float(np.abs(phi - vphi0).sum() / vphi0.sum())
        vort[f"{prec}_volume_drift"] = float(s.volume()[0] / v0 - 1.0)
        s.close()
    vort["phi_maxdiff_f32_vs_f64"] = float(np.abs(fin["f32"] - fin["f64"]).max())
    out["single_vortex"] = vort
    out["batching"] = batching_timing(cases, dev)
    out["droplet_lattice_16384x8192"] = lattice_timing(dev)
    out["adjoint"] = adjoint_timing(dev)
    out["adjoint_sweep_shear"] = adjoint_sweep_timing(dev)
    out["rayleigh_plateau_3d"] = rp3d_timing(dev, steps=args.steps3, peak64=out["fp64_peak"])
    out["shear_droplet"] = shear_timing(dev)
    return out


def batching_timing(cases, dev, steps_launch=10, steps_graph=64):
    """The headline batch advanced by one launch per step for all cases,
    against the same cases as separate single-case handles on one stream:
    (a) one lbm_step(h, 1) per case per step, i.e. one launch per case per
    step, against the batch stepped the same way (one launch per chain per
    step); (b) each case advanced steps_graph steps in turn, which the
    library replays as a CUDA graph per case, against the batch's own
    steps_graph-step graph.  FP32; the batch is autotuned as in the headline,
    the separate handles keep the library's default tiling."""
    import torch
    from paper_2505_10899_gb300 import lbm

    nodes = sum(c["nx"] * c["ny"] for c in cases)
    phis, us = host_inputs(cases)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b)

    sim = lbm.Sim(cases, phis, us, precision="f32")
    sim.autotune(1)
    sim.step(3)
    ms_b = timed(lambda: [sim.step(1) for _ in range(steps_launch)]) / steps_launch
    sim.prepare(steps_graph)
    ms_bg = timed(lambda: sim.step(steps_graph)) / steps_graph
    sim.close()
    del sim
    torch.cuda.empty_cache()
    sims = [lbm.Sim(c, p, u, precision="f32") for c, p, u in zip(cases, phis, us)]
    for s in sims:
        s.step(2)

    def per_launch():
        for _ in range(steps_launch):
            for s in sims:
                s.step(1)

    ms_l = timed(per_launch) / steps_launch
    ms_g = timed(lambda: [s.step(steps_graph) for s in sims]) / steps_graph
    ok = all(s.status() == lbm.LBM_OK for s in sims)
    for s in sims:
        s.close()
    del sims
    torch.cuda.empty_cache()
    mlups = lambda ms: round(nodes / (ms * 1e-3) / 1e6, 1)
    return {"ncases": len(cases), "nodes": nodes,
            "batched_one_step_per_call_mlups": mlups(ms_b),
            "batched_graph_mlups": mlups(ms_bg),
            "per_case_launch_each_step_mlups": mlups(ms_l),
            "per_case_graph_replay_mlups": mlups(ms_g),
            "speedup_vs_launch_per_case_per_step": round(ms_l / ms_b, 2),
            "speedup_vs_graph_per_case": round(ms_g / ms_bg, 2),
            "how": "one lbm_step(1) per call: the batch (one launch per chain) against one "
                   "launch per case; 64-step runs: the batch's graph against each case's own "
                   "64-step graph replayed in turn",
            "status_ok": ok}


def lattice_timing(dev, steps=50, grid=(16384, 8192), tiling=None):
    """The coupled FP32 step on one large periodic grid: 16384 x 8192 nodes
    (134 M) holding a 64 x 32 lattice of R = 24 droplets with the physics of
    the two-droplet set-up; about 22 GB of state.  Autotuned, 3 warm-up steps,
    `steps` timed steps with CUDA events; MLUPS and the fraction of the
    measured HBM peak at 160 algorithmic bytes per node."""
    import torch
    from paper_2505_10899_gb300 import lbm

    torch.cuda.empty_cache()
    nx, ny = grid
    case, phi0, _ = W.droplet_lattice(nx, ny, nx // 256, ny // 256)
    nodes = case["nx"] * case["ny"]
    s = lbm.Sim(case, phi0, None, precision="f32")
    if tiling:
        s.set_tiling(*tiling)
    else:
        s.autotune(1)
    s.step(3)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s.stream)
    s.step(steps)
    b.record(s.stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    peak, kind = measured_peaks()
    gbs = 160 * nodes / (ms * 1e-3) / 1e9
    out = {"grid": f"{case['nx']}x{case['ny']}", "nodes": nodes,
           "droplets": f"{nx // 256}x{ny // 256}, R = 24",
           "mlups": round(nodes / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms, 4),
           "kernel": "step_kernel_tma" if s.kernel() == 2 else "step_kernel",
           "tiling": {"bx": s.tiling()[0], "rows": s.tiling()[1],
                      "chosen_by": "fixed" if tiling else "autotune"},
           "roofline": {"achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(gbs / peak, 4), "peak_kind": kind},
           "status": s.status()}
    s.close()
    del s
    torch.cuda.empty_cache()
    return out


def rp3d_timing(dev, grid=(256, 256, 1024), precisions=("f32", "f16", "f64"), steps=50,
                tiling=None, peak64=None):
    """3-D Rayleigh-Plateau column (D3Q19 flow + D3Q7 phase field, SRT limit of
    the model): MLUPS per storage precision in the autotuned launch with its
    HBM roofline, the phase-volume drift over the timed steps, and the largest
    |phi| difference of each precision from the FP64 GPU path over the whole
    box after 20 steps (the FP64 path itself matches the FP64 oracle to 1e-12
    in the GPU tests, at this size on sampled blocks)."""
    import torch
    from paper_2505_10899_gb300 import lbm3

    nx, ny, nz = grid
    R = 32.0 * min(nx, ny) / 256.0
    case, phi0 = W.rayleigh_plateau(nx, ny, nz, R=R)
    n = nx * ny * nz
    peak, peak_kind = measured_peaks()
    out = {"grid": f"{nx}x{ny}x{nz}", "nodes": n, "R": R, "eps": 0.05, "W": case["W"],
           "rho_ratio": case["rho_l"] / case["rho_g"], "sigma": case["sigma"],
           "tau_g": case["tau_g"], "tau_f": case["tau_f_l"], "l2": "state far larger than L2"}
    ref = None
    order = sorted(precisions, key=lambda p: p != "f64")  # FP64 first: the reference
    for prec in order:
        s = lbm3.Sim3(case, phi0, None, precision=prec)
        s.step(20)
        phi20 = s.fields()[0]
        if prec == "f64":
            ref = phi20
        err = None if ref is None else float(np.abs(phi20 - ref).max())
        del phi20
        s.close()
        s = lbm3.Sim3(case, phi0, None, precision=prec)
        if tiling:
            v, bx, by, zc = tiling
            s.set_kernel(0)
            s.set_tiling(bx, by, zc)
            s.set_kernel(v)
        else:
            s.autotune(2 if prec != "f64" else 1)
        s.step(3)
        v0 = s.volume()[0]
        K = steps if prec != "f64" else max(2, steps // 5)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(s.stream)
        s.step(K)
        b.record(s.stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / K
        v1 = s.volume()[0]
        bpn = BYTES_PER_NODE_3D[prec]
        achieved = bpn * n / (ms * 1e-3) / 1e9
        var = {1: "step3_kernel", 2: "step3_async_kernel<2 stages>",
               3: "step3_async_kernel<3 stages>", 4: "step3_bulk_kernel",
               5: "step3_strip_kernel", 6: "step3_strip_kernel (two stages, 3-5 CTAs per SM)"}[s.kernel()]
        out[prec] = {
            "mlups": round(n / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms, 4),
            "steps": K, "kernel": var, "tiling": dict(zip(("bx", "by", "zc", "ctas"), s.tiling())),
            "chosen_by": "fixed" if tiling else "autotune",
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "algorithmic_bytes_per_node": bpn, "peak_kind": peak_kind},
            "volume_drift_rel": float(v1 / v0 - 1.0),
            "phi_maxdiff_vs_f64_20steps": err,
            "status": s.status(),
        }
        if prec == "f64":
            # FP64 is bound by the FP64 pipe: that is the roofline; the HBM
            # fraction stays beside it for reference
            if peak64 is None:
                peak64 = fp64_peak(dev)
            hbm = out[prec]["roofline"]
            out[prec]["roofline"] = fp64_roofline("rp3d_step_f64_128x128x256", n, ms, peak64)
            out[prec]["roofline"]["hbm_frac"] = hbm["frac"]
        s.close()
        del s
        torch.cuda.empty_cache()
    return out


def adjoint_timing(dev, nx=512, ny=256, nsteps=32, ckpt=8):
    """Reverse mode (FP64) against the FP64 forward step on a 512x256 droplet:
    the bare vector-Jacobian step, and the full checkpointed backward of
    torch.autograd (recompute + adjoint) per step."""
    import torch
    from paper_2505_10899_gb300 import adjoint as A

    torch.cuda.empty_cache()
    case = W.base_case(nx, ny)
    phi0 = W.tanh_disc(nx, ny, nx / 2, ny / 2, 40.0, 4.0, periodic=True)
    s = A.AdjointSim(case, phi0)
    s.sim.autotune(1)  # the forward step of the comparison: the fastest kernel
    stream = s.sim.stream

    def timed(fn, n):
        fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / n

    fwd_ms = timed(lambda: s.step(1), 50)
    s.restore(s.snapshot(), s.t)
    adj = torch.as_tensor(W.uniform(5, (20, ny, nx), -1, 1), device=s.dev)
    out = torch.empty_like(adj)

    def one_vjp():
        s.vjp_step(adj, None, out)

    vjp_ms = timed(one_vjp, 20)
    s.close()

    # full backward through torch.autograd: forward states recorded in device
    # memory (the default), and checkpoints every `ckpt` steps with
    # recomputation (store_bytes=0).  The second run of each is timed: the
    # first one loads the kernels.
    def fwd_bwd(store):
        phi0_t = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
        theta = torch.tensor([case["sigma"], case["tau_g"], case["lambda"], case["tau_f_l"]],
                             dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        phiT = A.coupled_run(phi0_t, theta, case, nsteps, ckpt, store_bytes=store)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        phiT.sum().backward()
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        return (t1 - t0) * 1e3 / nsteps, (t2 - t1) * 1e3 / nsteps

    res = {}
    for name, store in (("recorded", None), ("recomputed", 0)):
        fwd_bwd(store)
        f_ms, b_ms = fwd_bwd(store)
        res[name] = {"forward_ms_per_step": round(f_ms, 4), "backward_ms_per_step": round(b_ms, 4),
                     "backward_over_forward_step": round(b_ms / fwd_ms, 3)}
    res["recomputed"]["checkpoint_every"] = ckpt
    return {"grid": f"{nx}x{ny}", "precision": "f64", "steps": nsteps,
            "forward_ms_per_step": round(fwd_ms, 4),
            "vjp_ms_per_step": round(vjp_ms, 4),
            "vjp_over_forward": round(vjp_ms / fwd_ms, 3),
            "backward_states_recorded": res["recorded"],
            "backward_states_recomputed": res["recomputed"]}


def adjoint_sweep_timing(dev, precisions=("f32", "f64"), nrec=256):
    """Reverse-mode step against the forward step on the sheared droplet in
    a 512 x 256 channel (walls at -U and +U = 0.01, R = 40, Ca = 0.1,
    Re = 0.1), per precision: the forward step autotuned and replayed from
    graphs, then lbm_record_steps of nrec states and one lbm_adjoint_sweep
    over them (two launches per step), both timed with CUDA events."""
    import torch
    from paper_2505_10899_gb300 import adjoint as A
    from paper_2505_10899_gb300 import lbm

    case, phi0, u0 = W.shear_droplet(512, 256, R=40.0, U=0.01, Ca=0.1, Re=0.1)
    out = {"grid": "512x256", "walls_u": 0.01, "steps": nrec}
    for prec in precisions:
        a = A.AdjointSim(case, phi0, u0, prec)
        a.sim.autotune(1)
        a.step(300)
        st = a.sim.stream
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        torch.cuda.synchronize(dev)
        e0.record(st)
        a.step(nrec)
        e1.record(st)
        torch.cuda.synchronize(dev)
        fwd = e0.elapsed_time(e1) / nrec
        rec = torch.empty((nrec, a.planes) + a.shape, dtype=a.dtype, device=a.dev)
        stride = rec[0].numel() * rec.element_size()
        lbm.lbm_record_steps(a.h, nrec, rec.data_ptr(), stride)
        adj = a.seed_phi(torch.ones(a.shape, dtype=torch.float64))
        spare = torch.empty_like(adj)
        t0 = a.t - nrec
        for _ in range(2):  # the first sweep loads the kernels; the second is timed
            torch.cuda.synchronize(dev)
            e0.record(st)
            lbm.lbm_adjoint_sweep(a.h, rec.data_ptr(), stride, t0, nrec, adj.data_ptr(),
                                  spare.data_ptr())
            e1.record(st)
            torch.cuda.synchronize(dev)
        adj_ms = e0.elapsed_time(e1) / nrec
        out[prec] = {"forward_us_per_step": round(fwd * 1e3, 2),
                     "adjoint_us_per_step": round(adj_ms * 1e3, 2),
                     "adjoint_over_forward": round(adj_ms / fwd, 3),
                     "forward_kernel": a.sim.kernel(), "forward_tiling": list(a.sim.tiling()),
                     "status": a.sim.status()}
        a.close()
        del rec, adj, spare
        torch.cuda.empty_cache()
    return out


def shear_timing(dev, nsteps=20000, ckpt=256, grad_steps=20000):
    """The sheared droplet in a 512 x 256 channel (walls at -U and
    +U = 0.01, R = 40, W = 4, Ca = 0.1, Re = 0.1): FP32 forward MLUPS over
    nsteps (register-pipelined kernel with walls), the Taylor deformation D
    after nsteps in FP32 and FP64, and the checkpointed reverse mode of
    D(phi_T) with respect to (sigma, tau_g, U_w) in FP64 and in FP32, each
    with its cost relative to the plain forward run of its own precision
    (U_w moves both walls: dD/dU_w = dD/du_top - dD/du_bot)."""
    import torch
    from paper_2505_10899_gb300 import adjoint as A
    from paper_2505_10899_gb300 import lbm

    case, phi0, u0 = W.shear_droplet(512, 256, R=40.0, U=0.01, Ca=0.1, Re=0.1)
    out = {"grid": "512x256", "walls_u": 0.01, "R": 40.0, "Ca": 0.1, "Re": 0.1, "W": 4.0,
           "steps": nsteps}
    for prec in ("f32", "f64"):
        s = lbm.Sim(case, phi0, u0, precision=prec)
        s.autotune(1)
        s.step(3)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s.stream)
        s.step(nsteps - 3)
        b.record(s.stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / (nsteps - 3)
        phi = torch.as_tensor(s.fields(0)[0])
        out[prec] = {"mlups": round(512 * 256 / (ms * 1e-3) / 1e6, 1),
                     "tiling": {"bx": s.tiling()[0], "rows": s.tiling()[1]},
                     "kernel": {1: "step_kernel", 3: "step_kernel_persistent"}.get(s.kernel(),
                                                                                    "?"),
                     "taylor_D": float(A.taylor_deformation(phi)),
                     "status": s.status()}
        s.close()
    # the parameter range of the set-up: D after nsteps for Ca in {0.1, 0.2,
    # 0.4} and Re in {0.1, 1} (FP32), beside Taylor's small-deformation
    # value D = Ca (19 m + 16) / (16 m + 16) = 35/32 Ca at viscosity ratio m = 1
    sweep = []
    for Ca in (0.1, 0.2, 0.4):
        for Re in (0.1, 1.0):
            c, p0, v0 = W.shear_droplet(512, 256, R=40.0, U=0.01, Ca=Ca, Re=Re)
            s = lbm.Sim(c, p0, v0, precision="f32")
            s.step(nsteps)
            phi = torch.as_tensor(s.fields(0)[0])
            sweep.append({"Ca": Ca, "Re": Re, "taylor_D": round(float(A.taylor_deformation(phi)), 5),
                          "small_deformation_theory": round(35.0 / 32.0 * Ca, 5),
                          "status": s.status()})
            s.close()
    out["ca_re_sweep_f32"] = sweep
    # reverse mode of D(phi_T); cached blocks of the earlier legs are returned
    # first so that the 64 GiB of recorded states is one fresh allocation
    torch.cuda.empty_cache()
    # untimed: the first CUDA call of the objective and of its derivative loads
    # torch's own kernels
    A.taylor_deformation(torch.tensor(phi0, device=dev, requires_grad=True)).backward()
    torch.cuda.synchronize(dev)
    for prec in ("f64", "f32"):
        torch.cuda.empty_cache()
        th = torch.tensor([case["sigma"], case["tau_g"], case["lambda"], case["tau_f_l"],
                           case["u_top"], case["u_bot"]], dtype=torch.float64, requires_grad=True)
        phi0_t = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        # device memory for recorded states (the rest is recomputed): every
        # state if they fit, leaving 24 GiB free for the rest of the run; the
        # FP32 states of 2x10^4 steps (220 GB) fit in the GPU's 288 GB, the
        # FP64 ones (420 GB) do not
        state_bytes = (20 if prec == "f64" else 21) * (8 if prec == "f64" else 4) * 512 * 256
        free = torch.cuda.mem_get_info(dev)[0]
        store = max(0, min(grad_steps * state_bytes, free - (24 << 30)))
        phiT = A.coupled_run(phi0_t, th, case, grad_steps, ckpt, u0=u0, store_bytes=store,
                             precision=prec)
        D = A.taylor_deformation(phiT)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        D.backward()
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        g = th.grad.numpy()
        plain_s = grad_steps * 512 * 256 / (out[prec]["mlups"] * 1e6)
        res = {"steps": grad_steps, "checkpoint_every": ckpt,
               "recorded_steps": min(grad_steps, store // state_bytes),
               "D": float(D.detach()),
               "dD_dsigma": float(g[0]), "dD_dtau_g": float(g[1]),
               "dD_dU_w": float(g[4] - g[5]),
               "forward_s": round(t1 - t0, 3), "backward_s": round(t2 - t1, 3),
               "backward_over_forward": round((t2 - t1) / (t1 - t0), 3),
               "backward_over_plain_forward": round((t2 - t1) / plain_s, 3),
               f"plain_{prec}_forward_s": round(plain_s, 3),
               "adjoint_arithmetic": "fp64" if prec == "f64" else
                                     ("fp32 (parameter terms summed per warp in fp32, "
                                      "then accumulated in fp64)")}
        if prec == "f32":
            ref = out["gradient_f64"]
            res["rel_diff_vs_f64_gradient"] = {
                k: round(abs(res[k] - ref[k]) / abs(ref[k]), 6)
                for k in ("dD_dsigma", "dD_dtau_g", "dD_dU_w")}
        out[f"gradient_{prec}"] = res
        del phiT, D
    return out


def cpu_baseline(cases, seconds):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the same workload: the first cases of the batch, 2 steps each."""
    import oracle

    oracle.build()
    steps = 2
    done_nodes, t_used, used = 0, 0.0, 0
    for c in cases:
        phi, u = W.case_fields(c)
        o = oracle.Oracle(c, phi, u)
        t0 = time.perf_counter()
        o.step(steps)
        t_used += time.perf_counter() - t0
        done_nodes += c["nx"] * c["ny"]
        used += 1
        if t_used > seconds:
            break
    out = {"value": round(done_nodes * steps / t_used / 1e6, 3), "unit": "MLUPS",
           "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"first {used} of {len(cases)} cases x {steps} steps "
                     f"({done_nodes} nodes, {t_used:.1f} s of oracle time)"}
    # the same loops on one core (the results are the same bits), first case
    n = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        phi, u = W.case_fields(cases[0])
        o = oracle.Oracle(cases[0], phi, u)
        t0 = time.perf_counter()
        o.step(1)
        t1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(n)
    out["single_core_value"] = round(cases[0]["nx"] * cases[0]["ny"] / t1 / 1e6, 3)
    return out


def run_reference(args):
    ws, rank, local, pg = dist_setup(args)
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    cases = rank_cases(args, 0)
    import oracle
    oracle.build()
    # each "step" is a bounded sample: the oracle advances a fixed subset of
    # the batch by one time step
    budget_nodes = 300_000
    sub, n = [], 0
    for c in cases:
        if n + c["nx"] * c["ny"] > budget_nodes and sub:
            break
        sub.append(c)
        n += c["nx"] * c["ny"]
    ors = []
    for c in sub:
        phi, u = W.case_fields(c)
        ors.append(oracle.Oracle(c, phi, u))
    for _ in range(args.warmup):
        for o in ors:
            o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for o in ors:
            o.step(1)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt / 1e6
    res = {"impl": "reference", "metric": "coupled-step MLUPS", "value": round(value, 3),
           "unit": "MLUPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded tanh droplets)",
           "config": {"workload": WORKLOAD_NAME, "ncases": len(cases)},
           "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS",
                            "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"first {len(sub)} cases ({n} nodes) per step"},
           "e2e": {"value": round(value, 3), "unit": "MLUPS",
                   "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)
    if pg:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.only_adjoint:
        import torch
        dev = torch.device("cuda", 0)
        print(json.dumps({"adjoint": adjoint_timing(dev),
                          "adjoint_sweep_shear": adjoint_sweep_timing(dev)}), flush=True)
        return
    if args.only_lattice:
        import torch
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        grid = tuple(int(v) for v in args.lattice.split(","))
        til = tuple(int(v) for v in args.tiling.split(",")) if args.tiling else None
        print(json.dumps({"droplet_lattice": lattice_timing(dev, grid=grid, tiling=til)}),
              flush=True)
        return
    if args.only_batching:
        import torch
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        print(json.dumps({"batching": batching_timing(rank_cases(args, 0), dev)}), flush=True)
        return
    if args.only_shear:
        import torch
        print(json.dumps({"shear_droplet": shear_timing(torch.device("cuda", 0))}), flush=True)
        return
    if args.only_3d:
        import torch
        grid = tuple(int(v) for v in args.grid3.split(","))
        til = tuple(int(v) for v in args.tiling3.split(",")) if args.tiling3 else None
        print(json.dumps({"rayleigh_plateau_3d": rp3d_timing(
            torch.device("cuda", 0), grid, tuple(args.prec3.split(",")), args.steps3, til)}),
            flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
