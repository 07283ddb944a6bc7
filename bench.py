#!/usr/bin/env python
"""Benchmark of the SDD mesh generator's hot path on GB300.

Workload (default): the 257x257 grid split 4x4 (1521 interface nodes), moving-front monitor
u = tanh(50 (r - 0.25 - 0.1 t)), omega = sqrt(1 + 50 |grad u|^2), tau = 1e-2, dt = 1e-3,
K = 100 substeps, paths stepped in FP32 with Kahan-compensated sums, every interface node
estimated to SE <= 1e-4 (adaptive: first chunk 1e5 paths), then the 16 backward-Euler
subdomain solves.  One benchmark step = one alternating time step (sdd_step): monitor on
the mesh, interface Monte Carlo, subdomain solves, new mesh.  Synthetic inputs only.

Prints one JSON line.  value = interface-node estimates/s at SE <= 1e-4 over all ranks;
path-steps/s, the roofline of the path kernel (CUDA events inside the library, on its
stream), the end-to-end rate through the C ABI with host buffers, sampled clocks and the
oracle timed on the host cores are reported beside it.  Multi-GPU (torchrun): every rank
runs its own independent problem (seed + rank), no collective on the data path: weak
scaling, max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "interface-node estimates/s & path-steps/s at SE≤1e-4; % FP32 peak; p99 latency"
UNIT = "interface-node estimates/s"
# Algorithmic 32-bit operations of one path-step (Sec. 3.4, Eq. 7), each special function
# counted once: Philox4x32-10 (10 rounds of two 32x32->64 products as hi/lo pairs and two
# three-way xors) 60, three uniforms 9, Box-Muller (one log, one sqrt, one sin, one cos and
# their products) 8, bilinear gather of three fields (cell location, weights, 12 FMA) 30,
# drift and diffusion (one sqrt) 5, Euler-Maruyama update 4, endpoint test 6, Brownian-bridge
# test (distances, four exponentials, survival product, compare) 28, loop and path bookkeeping 8.
OPS_PER_PATH_STEP = 158

# Issued warp instructions per path-step of the current FP32 path kernel on the benchmarked
# configuration (ncu, smsp__inst_executed.sum / path-steps on a full 2^19-path round); the
# issue fraction below divides by 4 warp instructions per clock per SM.
WARP_INST_PER_PATH_STEP = 8.61
LANES_PER_SM_CLK, ISSUE_PER_SM_CLK, SM_MAX_MHZ = 128, 4, 2070.0
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of one path-kernel launch on this grid, from an ncu
# capture of the current kernel on a full round (2^19 paths per node): the cold fill of the packed
# monitor cell records (64 B per node) and mesh displacements (8 B per node), ~4.8 MB of FP32 data
# per 257x257 grid, which does not grow with the number of paths.
MC_TRAFFIC_BYTES_PER_LAUNCH = 4.80e6


def ops_per_path_step(prob):
    """Algorithmic operations of a path-step for this problem's switches: a periodic path takes no
    endpoint test (6) and no bridge test (28), and neither it nor a Dirichlet path without the
    bridge test draws the bridge's uniform (3)."""
    ops = OPS_PER_PATH_STEP
    if prob.periodic:
        ops -= 6 + 28 + 3
    elif not prob.bb_test:
        ops -= 28 + 3
    return ops


def counters_apply(prob, args):
    """The ncu-derived constants (instructions per path-step, DRAM bytes per launch) were taken on
    the Dirichlet front with the bridge test in the default form and Kahan sums; other switches
    compile another kernel, for which they would be a guess."""
    return (args.precision == "kahan" and not prob.periodic and prob.bb_test and prob.form == 0
            and prob.bicubic and args.iface_stride <= 1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="kahan", choices=["fp32", "fp64", "kahan"])
    ap.add_argument("--se-target", type=float, default=1e-4)
    ap.add_argument("--paths", type=int, default=100000)
    ap.add_argument("--max-paths", type=int, default=1 << 25)
    ap.add_argument("--periodic", type=int, default=0)
    ap.add_argument("--form", type=int, default=0, choices=[0, 1],
                    help="0: tau x_t = div(omega grad x) (the benchmark plan's generator); 1: the paper's")
    ap.add_argument("--tau", type=float, default=1e-2)
    ap.add_argument("--iface-stride", type=int, default=0,
                    help="Monte Carlo at every k-th interface node, the rest interpolated (0: all)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default path-kernel launch configuration instead of running the autotuner "
                         "(sdd_tune / sdd_batch_tune_mc) before the warm-up steps")
    ap.add_argument("--mc-config", default="",
                    help="fixed path-kernel launch configuration 'threads_per_block,blocks_per_sm,paths_per_task' "
                         "(0 keeps a field's default) in place of the autotuner")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="front", choices=["front", "mix", "serve", "sweep"],
                    help="front: the 257x257 / 4x4 moving-front problem (the benchmark line); "
                         "mix: the batch of 64 uneven problems, batched vs one at a time; "
                         "serve: one-step requests of the mix's shapes with Poisson arrivals through "
                         "the continuous-batching server; sweep: precision sweep on the 257x257 sine "
                         "mode against its closed form")
    ap.add_argument("--serve-n", type=int, default=64, help="serve: requests")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="serve: mean arrivals per second")
    ap.add_argument("--serve-first-chunk", type=int, default=10000, help="serve: first paths per node")
    ap.add_argument("--serve-budget-gb", type=float, default=150.0, help="serve: device-memory budget")
    ap.add_argument("--serve-fp64-baseline", type=int, default=0,
                    help="serve: also step the first K requests one at a time in plain FP64 (same SE target)")
    ap.add_argument("--serve-round-paths", type=int, default=1 << 27,
                    help="serve: paths per round, oldest requests first (0: all pending chunks)")
    ap.add_argument("--split", default="problems", choices=["problems", "nodes"],
                    help="under torchrun: one problem per rank (weak scaling, the default), or one "
                         "problem's interface nodes split over the ranks (strong scaling)")
    ap.add_argument("--mix-n", type=int, default=64)
    ap.add_argument("--mix-batched-only", action="store_true",
                    help="mix: skip the one-at-a-time comparisons (profiling case)")
    ap.add_argument("--mc-only", type=int, default=0,
                    help="profiling case: run `steps` interface-MC calls at this fixed N per node and "
                         "print the library's counters (not a benchmark line)")
    return ap.parse_args()


def workload(args, rank=0):
    import workloads as W
    prec = {"fp32": W.PREC_FP32_ACC64, "fp64": W.PREC_FP64, "kahan": W.PREC_FP32_KAHAN}[args.precision]
    p = W.c1_front(prec, periodic=args.periodic)
    return p.replace(se_target=args.se_target, paths_per_node=args.paths,
                     max_paths_per_node=max(args.max_paths, args.paths), seed=p.seed + rank,
                     iface_stride=args.iface_stride, form=args.form, tau=args.tau)


def config_of(p, M):
    return {"workload": f"{p.name}: {p.nx}x{p.ny} grid, {p.px}x{p.py} subdomains, moving-front monitor, "
                        f"SE<=1e-4 per interface node",
            "grid": [p.nx, p.ny], "subdomains": [p.px, p.py], "interface_nodes": M,
            "periodic": p.periodic, "se_target": p.se_target, "paths_first_chunk": p.paths_per_node,
            "max_paths_per_node": p.max_paths_per_node, "substeps": p.substeps, "tau": p.tau, "dt": p.dt,
            "path_precision": {0: "fp64", 1: "fp32 (fp64 sums)", 2: "fp32 (kahan fp32 sums)"}[p.precision],
            "l2": "256 MiB buffer written between timed steps (inputs are ~1 MB)",
            **({"iface_stride": p.iface_stride} if p.iface_stride > 1 else {}),
            **({"generator_form": "paper (x_t = grad w / w . grad x + lap x, scaled by tau)"} if p.form == 1 else {})}


def reduce_over_ranks(dist, T, path_steps, estimates, device):
    """Whole-job numbers of a weak-scaling run: the slowest rank's time, the work of all ranks."""
    if dist is None:
        return float(T), float(path_steps), float(estimates)
    import torch
    t = torch.tensor([float(T)], dtype=torch.float64, device=device)
    w = torch.tensor([float(path_steps), float(estimates)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t[0]), float(w[0]), float(w[1])


def node_ranges(M, world):
    """Contiguous interface-node ranges [lo, hi) of a partition of [0, M) into `world` parts
    whose sizes differ by at most one."""
    return [(M * r // world, M * (r + 1) // world) for r in range(world)]


def allgather_node_estimates(dist, est, ranges, rank, device):
    """Assemble the M x 2 estimates on every rank from each rank's own range: one all-gather of
    the full arrays, then each range taken from its owner's copy."""
    import torch
    if dist is None:
        return est
    mine = torch.as_tensor(est, dtype=torch.float64).to(device)
    parts = [torch.empty_like(mine) for _ in ranges]
    dist.all_gather(parts, mine)
    out = mine.clone()
    for r, (lo, hi) in enumerate(ranges):
        if r != rank:
            out[lo:hi] = parts[r][lo:hi]
    return out.cpu().numpy()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    @staticmethod
    def warm():
        """One query before anything is timed: a fresh machine pages nvidia-smi and its driver
        library in on first use, which must not fall inside a timed region."""
        try:
            subprocess.run(["nvidia-smi", "-L"], capture_output=True, timeout=60)
        except (OSError, subprocess.SubprocessError):
            pass

    def stop(self, window=None):
        """Median SM clock and throttle reasons of the samples taken inside window = (t0, t1)
        (time.time() seconds; all samples when None)."""
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        import datetime
        rows = []
        for line in self.f.read().splitlines():
            c = [v.strip() for v in line.split(",")]
            if len(c) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(c[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            rows.append((ts, c[1:]))
        inside = [r for r in rows if window is None or (r[0] is not None and window[0] <= r[0] <= window[1])]
        for _, c in inside or rows:
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return None
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(prob, seconds):
    """The oracle (C core, OpenMP over nodes, all host cores) on a bounded sample of the same
    workload: a spread of interface nodes, first time step, FP32 paths.  Converted to
    interface-node estimates/s with the path-steps one estimate at SE <= target needs, taken
    from the sample itself (the same basis in the repository's line and the reference arm)."""
    import numpy as np

    import oracle
    from oracle import _clib, mc
    from oracle.layout import interface_nodes
    from oracle.step import monitor_on_mesh
    import workloads as W

    oracle.build()
    x, y = W.identity_mesh(prob)
    om = monitor_on_mesh(prob, x, y, prob.t0)
    real = np.float64 if prob.precision == W.PREC_FP64 else np.float32
    inp = mc.prepare(prob, x, y, om, 0, real)
    nodes = interface_nodes(prob.nx, prob.ny, prob.px, prob.py, prob.periodic)
    M = len(nodes)
    pick = np.linspace(0, M - 1, 32).astype(int)
    shift = np.stack([x[nodes[pick, 1], nodes[pick, 0]], y[nodes[pick, 1], nodes[pick, 0]]], 1)

    def run(n):
        t = time.perf_counter()
        sums, steps = mc.interface_sums(inp, pick, nodes[pick], np.zeros(len(pick), np.int64),
                                        np.full(len(pick), n, np.int64), shift)
        return time.perf_counter() - t, sums, steps

    cores = int(_clib.lib().oracle_max_threads())
    dt0, _, st0 = run(512)
    rate0 = st0.sum() / max(dt0, 1e-9)
    # the same C core on one thread, on a sample an eighth of the time
    n1 = int(max(64, min(1 << 20, seconds / 8 * rate0 / cores / max(st0.sum() / 512, 1.0))))
    _clib.lib().oracle_set_threads(1)
    try:
        dt1, _, st1 = run(n1)
    finally:
        _clib.lib().oracle_set_threads(cores)
    rate1 = float(st1.sum() / max(dt1, 1e-9))
    n = int(max(512, min(1 << 20, seconds * rate0 / max(st0.sum() / 512, 1.0))))
    dt, sums, steps = run(n)
    rate = float(steps.sum() / dt)
    _, _, se = mc.estimate(sums, np.full(len(pick), n), shift)
    need = np.maximum((se.max(axis=1) / prob.se_target) ** 2, 1.0) * n  # paths for SE <= target
    sigma = se.max(axis=1) * np.sqrt(n)  # per-path standard deviation of the node values
    ps_per_est = float(np.mean(need * steps / n))
    return {"value": rate / ps_per_est, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{len(pick)} of {M} interface nodes x {n} paths, first time step, "
                      f"{'fp64' if real is np.float64 else 'fp32'} paths, {dt:.1f} s; path-steps/s "
                      f"{rate:.4g} divided by {ps_per_est:.4g} path-steps per node estimate at SE<=1e-4",
            "path_steps_per_s": rate,
            "single_core": {"path_steps_per_s": rate1, "value": rate1 / ps_per_est,
                            "sample": f"{len(pick)} nodes x {n1} paths on one thread, {dt1:.1f} s"},
            "sigma_v": {"mean": float(sigma.mean()), "max": float(sigma.max()),
                        "basis": "per-path standard deviation of a node's value (larger component), "
                                 "se * sqrt(paths) over the sampled nodes"}}


def mix_cpu_baseline(mix, seconds):
    """The oracle (all host cores) on a bounded sample of the batched mix: up to 256 nodes of every
    8th problem, first time step, FP32 paths, 10^3 paths per node; converted to interface-node
    estimates/s at the mix's paths per node with the sample's path-steps per path."""
    import numpy as np

    import oracle
    from oracle import _clib, mc
    from oracle.layout import interface_nodes
    from oracle.step import monitor_on_mesh
    import workloads as W

    oracle.build()
    n = 1000
    steps_tot, paths_tot, t_tot = 0, 0, 0.0
    t_start = time.perf_counter()
    for q in mix[::8]:
        q = q.replace(precision=W.PREC_FP32_KAHAN)
        x, y = W.identity_mesh(q)
        om = monitor_on_mesh(q, x, y, q.t0)
        inp = mc.prepare(q, x, y, om, 0, np.float32)
        nodes = interface_nodes(q.nx, q.ny, q.px, q.py, q.periodic)
        pick = np.unique(np.linspace(0, len(nodes) - 1, 256).astype(int))
        shift = np.stack([x[nodes[pick, 1], nodes[pick, 0]], y[nodes[pick, 1], nodes[pick, 0]]], 1)
        t = time.perf_counter()
        _, st = mc.interface_sums(inp, pick, nodes[pick], np.zeros(len(pick), np.int64),
                                  np.full(len(pick), n, np.int64), shift)
        t_tot += time.perf_counter() - t
        steps_tot += int(st.sum())
        paths_tot += n * len(pick)
        if time.perf_counter() - t_start > seconds:
            break
    rate = steps_tot / max(t_tot, 1e-9)
    ps_per_est = steps_tot / paths_tot * mix[0].paths_per_node
    return {"value": rate / ps_per_est, "unit": "interface-node estimates/s",
            "cores": int(_clib.lib().oracle_max_threads()), "kind": "oracle",
            "sample": f"{paths_tot // n} nodes of every 8th problem x {n} paths, first time step, fp32 paths, "
                      f"{t_tot:.1f} s; path-steps/s {rate:.4g} divided by {ps_per_est:.4g} path-steps "
                      f"per node estimate at {mix[0].paths_per_node} paths",
            "path_steps_per_s": rate}


def accuracy_vs_fp64_oracle(prob, stream, n=4096, nodes=8):
    """The bench problem's first step at a fixed n paths per node on the GPU (the bench's own
    precision), against the oracle with FP64 paths and sums on the same Philox streams, at a
    spread of nodes: the largest difference of the estimates, absolute and in units of the GPU's
    standard error.  Near the front, paths are chaotic (a rounding difference can grow by orders
    of magnitude), so the two are draws of the same estimator rather than equal numbers."""
    import numpy as np

    import oracle
    import paper_1504_00084_gb300 as S
    from oracle import mc
    from oracle.layout import interface_nodes
    from oracle.step import monitor_on_mesh
    import workloads as W

    oracle.build()
    q = prob.replace(se_target=0.0, paths_per_node=n, max_paths_per_node=n)
    x, y = W.identity_mesh(q)
    with S.SddProblem(S.params_from(q), x, y, stream=stream) as h:
        h.set_monitor_analytic(q.monitor_kind, q.monitor_params)
        est, se, _, _ = h.interface_mc()
    q64 = q.replace(precision=W.PREC_FP64)
    om = monitor_on_mesh(q64, x, y, q64.t0)
    inp = mc.prepare(q64, x, y, om, 0, np.float64)
    ij = interface_nodes(q.nx, q.ny, q.px, q.py, q.periodic)
    pick = np.linspace(0, len(ij) - 1, nodes).astype(int)
    shift = np.stack([x[ij[pick, 1], ij[pick, 0]], y[ij[pick, 1], ij[pick, 0]]], 1)
    sums, _ = mc.interface_sums(inp, pick, ij[pick], np.zeros(len(pick), np.int64),
                                np.full(len(pick), n, np.int64), shift)
    oest, _, _ = mc.estimate(sums, np.full(len(pick), n), shift)
    d = np.abs(est[pick] - oest)
    return {"nodes": int(len(pick)), "paths_per_node": n, "max_abs": float(d.max()),
            "max_in_se": float((d / np.maximum(se[pick], 1e-300)).max()),
            "basis": "first step at fixed paths; GPU at the bench precision vs the FP64 oracle"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prob = workload(args)
    K, Wm = args.steps, args.warmup
    per = max(2.0, min(args.cpu_seconds, 60.0 / max(K + Wm, 1)))
    vals = []
    for i in range(Wm + K):
        r = cpu_baseline(prob, per)
        if i >= Wm:
            vals.append(r)
    value = statistics.median(v["value"] for v in vals)
    from oracle.layout import interface_nodes
    M = len(interface_nodes(prob.nx, prob.ny, prob.px, prob.py, prob.periodic))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": K, "warmup": Wm, "ms_per_step": M / value * 1e3,
           "ms_per_step_basis": "extrapolated: the step's interface nodes at the sampled rate",
           "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64", "data": "synthetic",
           "config": config_of(prob, M),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                            "sample": vals[0]["sample"], "sigma_v": vals[0]["sigma_v"],
                            "single_core": vals[0]["single_core"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_1504_00084_gb300 as S
    import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    ClockSampler.warm()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    prob = workload(args, rank)
    x0, y0 = W.identity_mesh(prob)
    stream = torch.cuda.current_stream()

    tuned = {}

    def fresh_problem():
        h = S.SddProblem(S.params_from(prob), x0, y0, stream=stream)
        h.set_monitor_analytic(prob.monitor_kind, prob.monitor_params)
        # launch configuration: tuned once on the first problem's first round (outside any timed
        # region), then given to every later problem so both timed runs do the same work
        if args.mc_config and not tuned:
            _, bps, tp = (int(v) for v in args.mc_config.split(","))
            h.set_mc_config(blocks_per_sm=bps, paths_per_task=tp)
            tuned.update(h.mc_config())
        elif not args.no_tune and not tuned:
            tuned.update(h.tune_mc(True))
        elif tuned:
            h.set_mc_config(blocks_per_sm=tuned["blocks_per_sm"], paths_per_task=tuned["paths_per_task"])
        for _ in range(args.warmup):
            S.sdd_step(h.h)
        torch.cuda.synchronize()
        return h

    # End to end through the C ABI with host buffers: every step uploads its mesh from pinned
    # host memory and reads the new mesh back.  Run on its own problem over the same trajectory
    # steps as the device-timed run below (results are deterministic, so the work is identical).
    e2e = None
    if not args.no_e2e:
        h = fresh_problem()
        hx = torch.from_numpy(np.ascontiguousarray(h.mesh()[0])).pin_memory()
        hy = torch.from_numpy(np.ascontiguousarray(h.mesh()[1])).pin_memory()
        ox, oy = torch.empty_like(hx).pin_memory(), torch.empty_like(hy).pin_memory()
        barrier()
        torch.cuda.synchronize()
        te = time.perf_counter()
        for _ in range(args.steps):
            S.sdd_set_mesh(h.h, hx, hy)
            S.sdd_step(h.h, ox, oy)
            hx, ox = ox, hx
            hy, oy = oy, hy
        torch.cuda.synchronize()
        barrier()
        Te, _, _ = reduce_over_ranks(dist, time.perf_counter() - te, 0, 0, "cuda")
        nb = 2 * prob.nx * prob.ny * 8
        e2e = {"value": h.M * args.steps * world / Te, "unit": UNIT, "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb}
        h.close()

    # clocks sampled from before the timed problem's warm-up steps; only the samples inside the
    # timed window are reported
    sampler = ClockSampler(local)
    h = fresh_problem()
    M = h.M
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    flush.zero_()  # the first fill loads its kernel (lazily, from the torch library): not in the timed region
    launches0 = h.stats()["kernel_launches"]
    path_steps, mc_ms, mc_launches, paths = 0, 0.0, 0, 0
    max_se, not_reached = 0.0, 0
    barrier()
    torch.cuda.synchronize()
    w0 = time.time()
    t0 = time.perf_counter()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        flush.zero_()
        S.sdd_step(h.h)
        st = h.stats()
        path_steps += st["path_steps"]
        paths += st["paths"]
        mc_ms += st["mc_kernel_ms"]
        mc_launches += st["mc_kernel_launches"]
        max_se = max(max_se, st["max_se"])
        not_reached += st["nodes_not_reached"]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    clocks = sampler.stop((w0, time.time()))
    dev_s = ev0.elapsed_time(ev1) / 1e3
    T = max(dev_s, 1e-9)
    launches = h.stats()["kernel_launches"] - launches0
    T_all, ps_all, est_all = reduce_over_ranks(dist, T, path_steps, M * args.steps, "cuda")
    h.close()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clocks["sm_mhz"] if clocks and clocks.get("sm_mhz") else SM_MAX_MHZ
    alu_peak = sms * LANES_PER_SM_CLK * mhz * 1e6  # lane-ops/s
    ps_rate = path_steps / (mc_ms / 1e3) if mc_ms > 0 else 0.0
    ops = ops_per_path_step(prob)
    achieved = ops * ps_rate
    measured = counters_apply(prob, args)
    out = {"metric": METRIC, "value": est_all / T_all, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * T_all / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp32": "f32", "fp64": "f64", "kahan": "f32"}[args.precision], "data": "synthetic",
           "config": config_of(prob, M),
           "path_steps_per_s": ps_all / T_all,
           "paths_per_node_mean": paths / max(M * args.steps, 1),
           "max_se": max_se, "nodes_not_reached": not_reached,
           "wall_s": wall,
           "gpu_launches": int(launches),
           "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": alu_peak / 1e12,
                        "unit": "Tops/s (32-bit lane ops)", "frac": achieved / alu_peak,
                        "traffic": MC_TRAFFIC_BYTES_PER_LAUNCH if measured else None,
                        "traffic_unit": "bytes per launch", "kernel": "mc_kernel<float>",
                        "ops_per_path_step": ops,
                        "ops_basis": "algorithmic operations of a path-step, each special function once",
                        "path_steps_per_s_in_kernel": ps_rate,
                        "kernel_ms": mc_ms, "kernel_launches": mc_launches,
                        "kernel_share_of_step": (mc_ms / 1e3) / T if T > 0 else None,
                        "peak_basis": f"{sms} SMs (queried) x {LANES_PER_SM_CLK} lanes x {mhz:.0f} MHz "
                                      f"(median sampled SM clock under load)",
                        "issue": {"warp_inst_per_path_step": WARP_INST_PER_PATH_STEP if measured else None,
                                  "frac": (WARP_INST_PER_PATH_STEP * ps_rate / (sms * ISSUE_PER_SM_CLK * mhz * 1e6)
                                           if measured else None),
                                  "basis": "issued warp instructions (ncu count of this kernel) over "
                                           "4 per clock per SM: the instruction-level fraction"}},
           "clocks": clocks, "e2e": e2e,
           "launch_config": tuned or {"threads_per_block": 256, "paths_per_task": 2048,
                                      "blocks_per_sm": "register limit", "tuned": False}}
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(prob, args.cpu_seconds)
        # part of the oracle leg: the GPU's first-step estimates against the FP64 oracle's
        out["cpu_baseline"]["accuracy_vs_fp64_oracle"] = accuracy_vs_fp64_oracle(prob, stream)
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_mc_only(args):
    import torch

    import paper_1504_00084_gb300 as S
    import workloads as W

    torch.cuda.set_device(0)
    prob = workload(args).replace(se_target=0.0, paths_per_node=args.mc_only, max_paths_per_node=args.mc_only)
    x0, y0 = W.identity_mesh(prob)
    with S.SddProblem(S.params_from(prob), x0, y0, stream=torch.cuda.current_stream()) as h:
        h.set_monitor_analytic(prob.monitor_kind, prob.monitor_params)
        for _ in range(args.warmup + args.steps):
            h.interface_mc()
            st = h.stats()
            print(json.dumps({"mc_only": args.mc_only, "path_steps": st["path_steps"], "paths": st["paths"],
                              "mc_kernel_ms": st["mc_kernel_ms"],
                              "path_steps_per_s": st["path_steps"] / (st["mc_kernel_ms"] / 1e3)}))
    return 0


def hbm_peak_gbs():
    """Measured copy bandwidth of this GPU pool (generated file), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def subdomain_unknowns(p):
    """Interior nodes of all subdomains of a problem (subdomain I spans floor(I (n-1)/P) ..)."""
    def widths(n, P):
        return [((I + 1) * (n - 1)) // P - (I * (n - 1)) // P for I in range(P)]
    return sum((wx - 1) * (wy - 1) for wx in widths(p.nx, p.px) for wy in widths(p.ny, p.py))


def run_mix(args):
    """The batched mix: 64 independent problems (grids 65..513, splits 2x2..8x8, bump monitors,
    1e4 paths per node) stepped as one batch in a CUDA graph, against the same problems stepped
    one at a time with sdd_step -- in FP32 and in plain FP64 at the same path count (the same
    standard error)."""
    import torch

    import paper_1504_00084_gb300 as S
    import workloads as W

    torch.cuda.set_device(0)
    mix = W.c3_mix(args.mix_n, paths=args.paths if args.paths != 100000 else 10000)
    prec = W.PREC_FP32_KAHAN
    stream = torch.cuda.Stream()

    def make(precision):
        hs = []
        for p in mix:
            q = p.replace(precision=precision)
            x0, y0 = W.identity_mesh(q)
            h = S.SddProblem(S.params_from(q), x0, y0)
            h.set_monitor_analytic(q.monitor_kind, q.monitor_params)
            hs.append(h)
        return hs

    hs = make(prec)
    M = sum(h.M for h in hs)
    b = S.SddBatch(hs, stream=stream, use_graph=True)
    # launch configuration timed on the first round: block size and blocks per SM change no
    # result; the task size changes the grouping of the sums (and is set on every problem)
    if args.mc_config:
        tpb, bps, tp = (int(v) for v in args.mc_config.split(","))
        b.set_mc_config(threads_per_block=tpb, blocks_per_sm=bps, paths_per_task=tp)
        cfg = b.mc_config()
    else:
        cfg = b.mc_config() if args.no_tune else b.tune_mc(True)
    for _ in range(args.warmup):
        b.step()
    stream.synchronize()
    l0 = b.stats()["kernel_launches"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ps = 0
    e0.record(stream)
    for _ in range(args.steps):
        b.step()
    e1.record(stream)
    stream.synchronize()
    st = b.stats()
    T = e0.elapsed_time(e1) / 1e3
    # the batched solve's own device time, from one more step outside the graph (events
    # captured inside a graph carry no timing)
    b.close()
    b = S.SddBatch(hs, stream=stream, use_graph=False)
    b.step()
    solve_ms = b.stats()["solve_kernel_ms"]
    U = sum(subdomain_unknowns(p) for p in mix)
    peak, basis = hbm_peak_gbs()
    solve_bytes = 40.0 * U  # FP64 x^n, y^n, omega read and x, y written once per unknown
    solve_gbs = solve_bytes / (solve_ms / 1e3) / 1e9 if solve_ms > 0 else None
    batch = {"s_per_step": T / args.steps, "interface_node_estimates_per_s": M * args.steps / T,
             "path_steps_last_step": st["path_steps"], "launches_per_step": (st["kernel_launches"] - l0) / args.steps,
             "launch_config": cfg,
             "solve_iters_max": st["solve_iters_max"], "solve_outer_max": st["solve_outer_max"],
             "solve_rel_residual": st["solve_rel_residual"],
             "solve_roofline": {"bound": "hbm", "kernel": "solve_batch_items_kernel (512-thread CTAs; clusters of 4 for subdomains of >= 32768 unknowns) or solve_batch_kernel", "ms": solve_ms,
                                "unknowns": U, "algorithmic_bytes": solve_bytes, "achieved": solve_gbs,
                                "peak": peak, "unit": "GB/s", "peak_basis": basis,
                                "frac": solve_gbs / peak if solve_gbs else None}}
    b.close()
    if args.mix_batched_only:
        for h in hs:
            h.close()
        print(json.dumps({"workload": "mix", "interface_nodes": M, "batched_fp32_graph": batch}))
        return 0

    def one_at_a_time(handles, steps):
        for h in handles:
            S.sdd_step(h.h)  # warm
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(steps):
            for h in handles:
                S.sdd_step(h.h)
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / steps

    t32 = one_at_a_time(hs, 1)
    for h in hs:
        h.close()
    h64 = make(W.PREC_FP64)
    t64 = one_at_a_time(h64, 1)
    for h in h64:
        h.close()
    out = {"metric": "interface-node estimates/s, batched mix vs one problem at a time",
           "workload": f"{args.mix_n} problems, grids 65..513, splits 2x2..8x8, bump monitors, "
                       f"{mix[0].paths_per_node} paths per node, K = 100",
           "interface_nodes": M, "batched_fp32_graph": batch,
           "one_at_a_time_fp32_s_per_step": t32, "one_at_a_time_fp64_s_per_step": t64,
           "speedup_vs_one_at_a_time_fp32": t32 / batch["s_per_step"],
           "speedup_vs_one_at_a_time_fp64": t64 / batch["s_per_step"]}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = mix_cpu_baseline(mix, args.cpu_seconds)
    print(json.dumps(out))
    return 0


def run_serve(args):
    """Serving with continuous batching: requests drawn like the batched mix (grids 65..513, splits
    2x2..8x8, 1-4 bump monitors), each one alternating step with every interface node at
    SE <= --se-target, arriving as a Poisson process at --serve-rate per second and served by one
    sdd_server (device-memory budget --serve-budget-gb).  Reports completed requests/s, interface-node
    estimates/s and the latency from arrival to result collected (p50, p99)."""
    import numpy as np
    import torch

    import paper_1504_00084_gb300 as S
    import workloads as W

    torch.cuda.set_device(0)
    n = args.serve_n
    reqs = [p.replace(precision=W.PREC_FP32_KAHAN, se_target=args.se_target, paths_per_node=args.serve_first_chunk,
                      max_paths_per_node=args.max_paths)
            for p in W.c3_mix(n + 2, seed=777, paths=args.serve_first_chunk)]
    meshes = [W.identity_mesh(p) for p in reqs]
    params = [S.params_from(p) for p in reqs]
    mparams = [np.asarray(p.monitor_params, dtype=np.float64) for p in reqs]
    arrivals = W.poisson_arrivals(n, args.serve_rate)
    q = S.SddServerParams()
    q.precision = W.PREC_FP32_KAHAN
    q.max_resident = 1024
    q.max_nodes = 1 << 19
    q.mem_budget_bytes = int(args.serve_budget_gb * (1 << 30))
    q.se_target = args.se_target
    q.paths_per_node = args.serve_first_chunk
    q.max_paths_per_node = args.max_paths
    q.round_paths = args.serve_round_paths
    stream = torch.cuda.Stream()
    srv = S.SddServer(q, stream)

    def submit(k):
        return srv.submit(params[k], meshes[k][0], meshes[k][1], reqs[k].monitor_kind, mparams[k])

    # warm-up: the last two requests of the draw, not timed
    warm = [submit(n), submit(n + 1)]
    got = []
    while len(got) < len(warm):
        srv.progress()
        got += srv.poll()
    for rid in got:
        srv.result(rid)
    s0 = srv.stats()
    lat, done_at, nodes, ps = [], [], 0, 0
    id_to_k = {}
    t0 = time.perf_counter()
    k = 0
    while len(lat) < n:
        now = time.perf_counter() - t0
        while k < n and arrivals[k] <= now:
            id_to_k[submit(k)] = k
            k += 1
        running, queued = srv.progress()
        for rid in srv.poll():
            _, st = S.sdd_server_result(srv.h, rid, None, None, None, None)
            t = time.perf_counter() - t0
            lat.append(t - arrivals[id_to_k[rid]])
            done_at.append(t)
            nodes += st["M"]
            ps += st["path_steps"]
        if running == 0 and queued == 0 and k < n:
            wait = arrivals[k] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
    s1 = srv.stats()
    srv.close()
    T = max(done_at) - arrivals[0]
    lat_ms = np.sort(np.asarray(lat)) * 1e3
    out = {"metric": "serving: completed requests/s, interface-node estimates/s, latency p50/p99",
           "workload": f"{n} one-step requests, grids 65..513, splits 2x2..8x8, bump monitors, "
                       f"SE <= {args.se_target:g} per node (first chunk {args.serve_first_chunk}), "
                       f"Poisson arrivals at {args.serve_rate:g}/s, {args.serve_round_paths} paths per round",
           "requests_per_s": n / T, "interface_node_estimates_per_s": nodes / T,
           "path_steps_per_s": ps / T, "latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                                                      "p99": float(np.percentile(lat_ms, 99)),
                                                      "max": float(lat_ms[-1])},
           "offered_span_s": float(arrivals[-1] - arrivals[0]), "makespan_s": T,
           "rounds": s1["rounds"] - s0["rounds"],
           "path_kernel_s": (s1["mc_kernel_ms"] - s0["mc_kernel_ms"]) / 1e3,
           "kernel_launches": s1["kernel_launches"] - s0["kernel_launches"],
           "allocations": s1["allocations"], "resident_gb": s1["resident_bytes"] / 2 ** 30,
           "pool_gb": s1["pool_bytes"] / 2 ** 30, "pool_high_water": s1["pool_high_water"]}
    kb = min(args.serve_fp64_baseline, n)
    if kb > 0:
        # the plain per-problem path: the same requests stepped one at a time with FP64 paths and
        # FP64 sums at the same standard-error target
        torch.cuda.synchronize()
        t = time.perf_counter()
        ps64, nodes64 = 0, 0
        for k in range(kb):
            q = reqs[k].replace(precision=W.PREC_FP64)
            x, y = meshes[k]
            with S.SddProblem(S.params_from(q), x, y) as h:
                h.set_monitor_analytic(q.monitor_kind, q.monitor_params)
                h.step()
                st = h.stats()
                ps64 += st["path_steps"]
                nodes64 += st["M"]
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t
        ts = t64 / kb
        out["sequential_fp64"] = {"requests": kb, "s_per_request": ts, "requests_per_s": 1.0 / ts,
                                  "interface_node_estimates_per_s": nodes64 / t64,
                                  "path_steps_per_s": ps64 / t64,
                                  "served_speedup": (n / T) * ts,
                                  "served_speedup_estimates": (nodes / T) / (nodes64 / t64),
                                  "basis": "the first requests of the draw stepped one at a time with FP64 paths and "
                                           "sums at the same SE target; served_speedup compares requests/s, "
                                           "served_speedup_estimates interface-node estimates/s (size-independent)"}
    print(json.dumps(out))
    return 0


def run_sweep(args):
    """Precision sweep on the 257x257 / 4x4 sine mode (omega = 1, mesh xi + 0.05 sin(pi xi)
    sin(pi eta), closed form xi + 0.05 e^{-2 pi^2 t / tau} sin sin at t = dt): for N = 1e3..1e6
    paths per node, FP32 paths with FP64 or Kahan-FP32 sums (and FP64 paths up to 1e5), the
    interface estimates' error against the closed form (absolute and in standard errors), the
    FP32-vs-FP64 difference on the same paths, and the path-kernel time; then the subdomain
    solves in FP32 with FP64 refinement against all-FP64 on the same interface data."""
    import math

    import numpy as np
    import torch

    import paper_1504_00084_gb300 as S
    import workloads as W

    torch.cuda.set_device(0)
    base = W.c2_sine()
    x0, y0 = W.sine_mode_mesh(base, amp=0.05)
    decay = math.exp(-2 * math.pi ** 2 * base.dt / base.tau)
    rows = []
    est64 = {}
    for prec, name, Ns in ((W.PREC_FP64, "fp64", (1000, 10000, 100000)),
                           (W.PREC_FP32_ACC64, "fp32_acc64", (1000, 10000, 100000, 1000000)),
                           (W.PREC_FP32_KAHAN, "fp32_kahan", (1000, 10000, 100000, 1000000))):
        for N in Ns:
            p = base.replace(precision=prec, paths_per_node=N)
            with S.SddProblem(S.params_from(p), x0, y0) as h:
                h.set_monitor_analytic(p.monitor_kind, p.monitor_params)
                est, se, _, _ = h.interface_mc()
                st = h.stats()
                nodes = h.nodes()
            xi = nodes[:, 0] / (p.nx - 1)
            eta = nodes[:, 1] / (p.ny - 1)
            mode = 0.05 * decay * np.sin(np.pi * xi) * np.sin(np.pi * eta)
            exact = np.stack([p.Lx * xi + mode, p.Ly * eta + mode], 1)
            err = np.abs(est - exact)
            row = {"precision": name, "paths_per_node": N, "max_abs_error": float(err.max()),
                   "max_error_in_se": float((err / np.maximum(se, 1e-300)).max()),
                   "mean_se": float(se.mean()), "path_kernel_ms": st["mc_kernel_ms"],
                   "path_steps_per_s": st["path_steps"] / (st["mc_kernel_ms"] / 1e3)}
            if name == "fp64":
                est64[N] = est
            elif N in est64:
                row["max_diff_vs_fp64_same_paths"] = float(np.abs(est - est64[N]).max())
            rows.append(row)
    # solves: FP32 CG + FP64 refinement vs FP64, same interface data
    iface = est64[max(est64)]
    meshes = {}
    for prec, name in ((W.PREC_FP64, "fp64"), (W.PREC_FP32_KAHAN, "fp32_refined")):
        p = base.replace(precision=prec)
        with S.SddProblem(S.params_from(p), x0, y0) as h:
            h.set_monitor_analytic(p.monitor_kind, p.monitor_params)
            gx, gy, _ = h.subdomain_solve(iface)
            meshes[name] = (gx, gy, h.stats())
    dx = max(float(np.abs(meshes["fp64"][0] - meshes["fp32_refined"][0]).max()),
             float(np.abs(meshes["fp64"][1] - meshes["fp32_refined"][1]).max()))
    out = {"metric": "precision sweep: interface error vs closed form, FP32 vs FP64",
           "workload": "sine257_4x4: 257x257 grid, 4x4 subdomains, omega = 1, sine-mode mesh, one step",
           "closed_form_decay": decay, "interface": rows,
           "solve": {"max_mesh_diff_fp32_refined_vs_fp64": dx,
                     "fp32_refined_rel_residual": meshes["fp32_refined"][2]["solve_rel_residual"],
                     "fp64_rel_residual": meshes["fp64"][2]["solve_rel_residual"],
                     "fp32_refined_solve_ms": meshes["fp32_refined"][2]["solve_kernel_ms"],
                     "fp64_solve_ms": meshes["fp64"][2]["solve_kernel_ms"]}}
    print(json.dumps(out))
    return 0


def run_split_nodes(args):
    """One problem shared by all ranks (strong scaling): each rank estimates its range of the
    interface nodes (sdd_interface_mc_range), one all-gather assembles the M x 2 estimates, and
    every rank takes the rest of the step (sdd_step_from_interface), so every rank holds the same
    new mesh.  Rank 0 prints the job's estimates/s of the one problem."""
    import numpy as np
    import torch

    import paper_1504_00084_gb300 as S
    import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    ClockSampler.warm()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prob = workload(args, 0)  # the same problem (same seed) on every rank
    x0, y0 = W.identity_mesh(prob)
    h = S.SddProblem(S.params_from(prob), x0, y0, stream=torch.cuda.current_stream())
    h.set_monitor_analytic(prob.monitor_kind, prob.monitor_params)
    M = h.M
    lo, hi = node_ranges(M, world)[rank]
    ranges = node_ranges(M, world)

    def split_step():
        est = np.zeros((M, 2))
        h.interface_mc_range(lo, hi, est)
        est = allgather_node_estimates(dist, est, ranges, rank, f"cuda:{local}")
        h.step_from_interface(est)

    for _ in range(args.warmup):
        split_step()
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.time()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        split_step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    T = time.perf_counter() - t0
    clocks = sampler.stop((w0, time.time()))
    T_all, _, _ = reduce_over_ranks(dist, T, 0, 0, f"cuda:{local}")
    h.close()
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    cfg = config_of(prob, M)
    cfg["split"] = f"interface nodes over {world} ranks, one all-gather of M x 2 estimates per step"
    print(json.dumps({"metric": METRIC, "value": M * args.steps / T_all, "unit": UNIT, "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T_all / args.steps,
                      "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype":
                      {"fp32": "f32", "fp64": "f64", "kahan": "f32"}[args.precision], "data": "synthetic",
                      "config": cfg, "clocks": clocks, "timing": "host wall clock around the whole split step"}))
    return 0


def main():
    args = parse()
    if args.mc_only > 0:
        return run_mc_only(args)
    if args.workload == "mix":
        return run_mix(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.split == "nodes":
        return run_split_nodes(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
