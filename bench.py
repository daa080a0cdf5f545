#!/usr/bin/env python3
"""Benchmark of the GB300 transport sweep (cell x direction x group updates/s, % of HBM roofline).

One step = one solve of the headline workload with the inputs resident in HBM:
classification + levelisation of all directions, then the periodic-boundary iteration
(batched FP32 sweep + FP64 tallies + periodic exchange) until max |E_i| < 1e-6.
Prints ONE JSON line (rank 0). Under torchrun every rank solves its own box (seed + rank):
weak scaling, no data-path collective.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload periodic|batched]
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell·dir·group sweep updates/s and % HBM roofline, batched FP32 vs plain FP64 sweep"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_sweep_periodic_2p22.txt")
WORKLOADS = {
    "periodic": "periodic Voronoi box, 2^22 cells sampled ~rho (lognormal, P(k)~k^-2.5, sigma_ln=1.5), 10^4 "
                "log-uniform sources, absorption only, 128 directions, 1 group, periodic iteration to E<1e-6",
    "batched": "64 Poisson-Voronoi meshes of log-uniform size (2^12..2^17, 2^22 cells), lognormal kappa, "
               "8 sources/mesh, 128 directions, 2 groups, one persistent launch",
    "scatter": "Voronoi mesh of 2^20 cells sampled ~rho (lognormal, P(k)~k^-3), albedo 0.5, 64 sources, "
               "96 directions, 4 groups, source iteration to relative change of J < 1e-6",
    "periodic_scatter": "periodic Voronoi box, 2^20 cells sampled ~rho as in the periodic workload, 10^4 "
                        "log-uniform sources, isotropic scattering with albedo 0.5, 128 directions, 1 group; "
                        "scattering and periodic iterations to 1e-6, nested or fused (Sec. 2.7)",
    "adjoint": "Poisson-Voronoi mesh of 2^18 cells, lognormal kappa, 32 sources, 64 directions, 2 groups; "
               "gradient of sum (Gamma - T)^2 in kappa and emissivity by the transposed sweep, forward "
               "intensities recomputed",
}


# ---------------------------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class Dist:
    """Barrier and max-reduction across ranks (no-op for one rank)."""

    def __init__(self, backend: str | None = None):
        self.rank, self.world, self.local = dist_env()
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
            self.dist = dist
            self.backend = backend
            self.pg = True

    def barrier(self):
        if self.pg:
            if self.backend == "nccl":
                import torch
                self.dist.barrier(device_ids=[self.local])
            else:
                self.dist.barrier()

    def reduce(self, vals: list[float], op: str) -> list[float]:
        if not self.pg:
            return list(vals)
        import torch
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor(vals, dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX if op == "max" else self.dist.ReduceOp.SUM)
        return [float(x) for x in t.cpu()]

    def close(self):
        if self.pg:
            self.dist.destroy_process_group()


def aggregate(dist: Dist, elapsed_s: float, updates: float) -> tuple[float, float]:
    """Whole-job throughput: updates summed over ranks / slowest rank's time."""
    t = dist.reduce([elapsed_s], "max")[0]
    u = dist.reduce([updates], "sum")[0]
    return u / t, t


# ---------------------------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in ("sweep.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2207_12848_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per launch of the batched sweep from the committed ncu summary, if still current."""
    if workload != "periodic" or not os.path.exists(PROFILE_SUMMARY):
        return None
    vals = {}
    with open(PROFILE_SUMMARY) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_sha") != kernel_sha():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def make_problem(workload: str, rank: int, threads: int | None, cells: int | None = None):
    from synth import configs
    if workload == "periodic":
        return configs.periodic(n_cells=cells or 1 << 22, seed=4 + 100 * rank, threads=threads)
    if workload == "batched":
        return configs.batched(total=cells or 1 << 22, seed=1 + 100 * rank, threads=threads)
    if workload == "scatter":
        return configs.scatter(n_cells=cells or 1 << 20, seed=3 + 100 * rank, threads=threads)
    if workload == "periodic_scatter":
        p = configs.periodic(n_cells=cells or 1 << 20, seed=6 + 100 * rank, threads=threads)
        return dataclasses.replace(p, name="periodic_scatter", kappa_scat=p.kappa_abs.copy())
    if workload == "adjoint":
        return configs.adjoint(n_cells=cells or 1 << 18, seed=5 + 100 * rank, threads=threads)
    raise ValueError(workload)


def step_text(p, fused: int) -> str:
    from synth.mesh import FACE_PERIODIC
    pbc = bool((p.mesh.flags & FACE_PERIODIC).any())
    scat = p.kappa_scat is not None and bool((p.kappa_scat != 0).any())
    loops = []
    if scat:
        loops.append("source iteration to max|dJ|/J<=1e-6")
    if pbc:
        loops.append("periodic iteration to max|E|<1e-6")
    it = " inside ".join(loops) if not (fused and pbc and scat) else \
        "fused iteration (one sweep per periodic iteration) to both tolerances"
    return "classify + levelise + " + (it or "one sweep")


def bytes_per_update(p, law: str = "balance") -> float:
    """Algorithmic DRAM bytes per (cell, direction, group) update.

    Per task (cell, direction): the row bounds (8 B) and every face-side record of the cell
    (16 B each: neighbour + A n_out in FP32), F_bar = face sides / cells. Per group: the
    source/denominator pair (8 B, FP32) and the intensity write (4 B), and under the EXP law the
    cell-mean write (4 B); the upwind re-reads hit L2 (the wavefront is on chip) and are not counted.
    """
    m = p.mesh
    S = 2 * m.n_faces - int((m.face_cells[:, 1] < 0).sum())
    fbar = S / m.n_cells
    G = p.n_groups
    return (8.0 + 16.0 * fbar) / G + 12.0 + (4.0 if law == "exp" else 0.0), fbar


# ---------------------------------------------------------------------------------------------
def cpu_baseline(p, seconds_target: float = 15.0, law: str = "balance") -> dict:
    """The FP64 oracle as it stands, on a bounded sample: one sweep of a subset of directions."""
    import numpy as np

    import oracle
    cores = os.cpu_count() or 1
    N, G = p.mesh.n_cells, p.n_groups
    # calibrate on one direction, then size the sample to ~seconds_target of CPU work
    t0 = time.perf_counter()
    oracle.solve(p.mesh, p.omega[:1], np.full(1, 4 * math.pi), p.kappa_abs, p.emissivity, max_it_pbc=1, threads=1,
                 law=law)
    t1 = time.perf_counter() - t0
    nd = int(max(cores, min(p.n_dir, round(seconds_target / max(t1, 1e-3)))))
    nd = min(nd, p.n_dir)
    nd = max(cores * max(1, nd // cores), 1) if nd >= cores else nd
    nd = min(nd, p.n_dir)
    om = p.omega[:nd]
    w = np.full(nd, 4 * math.pi / nd)
    t0 = time.perf_counter()
    oracle.solve(p.mesh, om, w, p.kappa_abs, p.emissivity, max_it_pbc=1, threads=min(cores, nd), law=law)
    dt = time.perf_counter() - t0
    ups = N * nd * G / dt
    return {"value": ups, "unit": "updates/s", "cores": min(cores, nd), "kind": "oracle",
            "sample": "one FP64 sweep of %d of %d directions over all %d cells (Alg. 2 task queue, threads over "
                      "directions), %.1f s wall" % (nd, p.n_dir, N, dt)}


def run_reference(args, dist: Dist):
    """The reference arm: the FP64 CPU oracle on the host cores, each step a bounded sample."""
    if dist.rank != 0:
        return
    import numpy as np

    import oracle
    p = make_problem(args.workload, 0, None, args.cells)
    cores = os.cpu_count() or 1
    nd = min(p.n_dir, cores)
    om, w = p.omega[:nd], np.full(nd, 4 * math.pi / nd)
    N, G = p.mesh.n_cells, p.n_groups
    for _ in range(args.warmup):
        oracle.solve(p.mesh, om, w, p.kappa_abs, p.emissivity, max_it_pbc=1, threads=nd, law=args.law)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve(p.mesh, om, w, p.kappa_abs, p.emissivity, max_it_pbc=1, threads=nd, law=args.law)
    dt = time.perf_counter() - t0
    v = N * nd * G * args.steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "updates/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "n_cells": N, "n_dir": p.n_dir, "n_groups": G,
                      "sample_dirs": nd},
           "cpu_baseline": {"value": v, "unit": "updates/s", "cores": nd, "kind": "oracle",
                            "sample": "one FP64 sweep of %d of %d directions per step" % (nd, p.n_dir)},
           "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_ours(args, dist: Dist):
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2207_12848_gb300 import Context, default_opts

    torch.cuda.set_device(dist.local)
    if dist.rank == 0 or dist.world == 1:
        __graft_entry__.build()
    dist.barrier()
    __graft_entry__.build()
    p = make_problem(args.workload, dist.rank, args.threads, args.cells)
    stream = torch.cuda.current_stream()
    N, D, G = p.mesh.n_cells, p.n_dir, p.n_groups
    ctx = Context(dist.local, stream.cuda_stream)
    ctx.set_mesh(p.mesh)
    ctx.set_directions(p.omega, p.weight)
    ka = torch.from_numpy(p.kappa_abs).cuda()
    em = torch.from_numpy(p.emissivity).cuda()
    ks = None if p.kappa_scat is None else torch.from_numpy(p.kappa_scat).cuda()
    ctx.set_material(ka, em, kappa_scat=ks)
    J = torch.empty((N, G), dtype=torch.float64, device="cuda")
    Gm = torch.empty_like(J)
    opts = default_opts(precision=32, relevel=1, tol_pbc=1e-6, max_it_pbc=200, tol_scat=1e-6, max_it_scat=200,
                        fused_loops=args.fused_loops, law=args.law, transport=args.transport)
    for _ in range(args.warmup):
        ctx.solve_dev(J, Gm, opts)
    torch.cuda.synchronize()
    dist.barrier()
    clocks = Clocks(dist.local)
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    dist.barrier()
    ev0.record(stream)
    agg = {"updates": 0.0, "sweep_ms": 0.0, "sweeps": 0, "launches": 0, "classify_ms": 0.0, "levelise_ms": 0.0,
           "assemble_ms": 0.0,
           "it_pbc": [], "it_scat": [], "defect": [], "res_pbc": []}
    for _ in range(args.steps):
        st, s = ctx.solve_dev(J, Gm, opts)
        agg["updates"] += st["updates"]
        agg["sweep_ms"] += st["t_sweep_ms"]
        agg["sweeps"] += st["sweep_launches"]
        agg["launches"] += st["kernel_launches"]
        agg["classify_ms"] += st["t_classify_ms"]
        agg["levelise_ms"] += st["t_levelise_ms"]
        agg["assemble_ms"] += st["t_assemble_ms"]
        agg["it_pbc"].append(st["it_pbc"])
        agg["it_scat"].append(st["it_scat"])
        agg["defect"].append(st["defect"])
        agg["res_pbc"].append(st["res_pbc"])
        last = st
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    clk = clocks.stop()
    value, tmax = aggregate(dist, elapsed, agg["updates"])

    # roofline of the dominant kernel (the batched sweep), CUDA events around each launch
    bpu, fbar = bytes_per_update(p, args.law)
    avg_launch_s = agg["sweep_ms"] / max(1, agg["sweeps"]) / 1e3
    alg_bytes = bpu * N * D * G
    peaks = measured_peaks()
    achieved = alg_bytes / avg_launch_s / 1e9
    from paper_2207_12848_gb300._lib import KERNELS
    roof = {"bound": "hbm", "kernel": "%s (%s schedule, %d lanes per task)" % (
                KERNELS.get(last.get("kernel_used", 0), "?"), {1: "level", 2: "dataflow"}.get(last["schedule_used"], "?"),
                last["lanes_used"]),
            "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
            "peak_source": peaks["source"],
            # the recorded DRAM traffic is that of the BALANCE law's kernel on the periodic box
            "traffic": profiled_traffic(args.workload) if args.law == "balance" else None,
            "bytes_per_update": bpu, "face_sides_per_cell": fbar, "updates_per_launch": N * D * G,
            "avg_launch_ms": avg_launch_s * 1e3}

    extra = {}
    if dist.rank == 0 and not args.quick:
        # plain FP64 per-(direction, level) sweep, same mesh, one sweep; and FP32/FP64 batched single sweeps
        one = dict(max_it_pbc=1, tol_pbc=0.0, max_it_scat=1, tol_scat=0.0)
        o1 = default_opts(precision=32, **one)
        st32, _ = ctx.solve_dev(J, Gm, o1)
        o64 = default_opts(precision=64, **one)
        st64, _ = ctx.solve_dev(J, Gm, o64)
        op = default_opts(schedule="plain", **one)
        stp, _ = ctx.solve_dev(J, Gm, op)
        u1 = N * D * G
        extra["plain_fp64"] = {
            "sweep_ms": stp["t_sweep_ms"], "updates_per_s": u1 / (stp["t_sweep_ms"] / 1e3),
            "batched_fp32_sweep_ms": st32["t_sweep_ms"], "batched_fp64_sweep_ms": st64["t_sweep_ms"],
            "speedup_fp32_vs_plain": stp["t_sweep_ms"] / st32["t_sweep_ms"],
            "speedup_fp64_batched_vs_plain": stp["t_sweep_ms"] / st64["t_sweep_ms"],
            "plain_launches": stp["kernel_launches"]}

    if dist.rank == 0 and not args.quick and args.law == "balance" and args.transport == 0:
        # the same box under the EXP law and under scheme (b) (direction-conserving to 3 neighbours): one
        # step each as timed above (classify, levelise, assemble, periodic iteration to 1e-6)
        for key, kw, law in (("exp_law", dict(law="exp"), "exp"), ("scheme_b", dict(transport=3), "balance")):
            ok = default_opts(precision=32, relevel=1, tol_pbc=1e-6, max_it_pbc=200, tol_scat=1e-6, max_it_scat=200,
                              **kw)
            ctx.solve_dev(J, Gm, ok)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sx, _ = ctx.solve_dev(J, Gm, ok)
            torch.cuda.synchronize()
            tx = time.perf_counter() - t0
            swm = sx["t_sweep_ms"] / max(1, sx["sweep_launches"])
            extra[key] = {"value": sx["updates"] / tx, "unit": "updates/s", "ms_per_step": 1e3 * tx,
                          "roofline": _roof(p, swm, peaks, KERNELS.get(sx["kernel_used"], "?"), law),
                          "solve": {"it_pbc": sx["it_pbc"], "n_sweeps": sx["n_sweeps"], "defect": sx["defect"],
                                    "depth_max": sx["depth_max"], "depth_mean": sx["depth_mean"],
                                    "depth_max_scheme_a": last["depth_max"], "classify_ms": sx["t_classify_ms"],
                                    "levelise_ms": sx["t_levelise_ms"], "assemble_ms": sx["t_assemble_ms"],
                                    "sweep_ms_per_launch": swm}}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        m = p.mesh
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hv, hfc, har, hnr, hfl = pin(m.volume), pin(m.face_cells), pin(m.area), pin(m.normal), pin(m.flags)
        hom, hw, hka, hem = pin(p.omega), pin(p.weight), pin(p.kappa_abs), pin(p.emissivity)
        hks = None if p.kappa_scat is None else pin(p.kappa_scat)
        h2d = sum(a.nbytes for a in (hv, hfc, har, hnr, hfl, hom, hw, hka, hem) + (() if hks is None else (hks,)))
        d2h = 2 * N * G * 8
        ctx2 = Context(dist.local, stream.cuda_stream)
        o = default_opts(precision=32, tol_pbc=1e-6, max_it_pbc=200, tol_scat=1e-6, max_it_scat=200,
                         fused_loops=args.fused_loops, law=args.law, transport=args.transport)

        def e2e_step():
            ctx2.set_mesh(volume=hv, face_cells=hfc, area=har, normal=hnr, flags=hfl)
            ctx2.set_directions(hom, hw)
            ctx2.set_material(hka, hem, kappa_scat=hks)
            return ctx2.solve(o)

        e2e_step()
        torch.cuda.synchronize()
        dist.barrier()
        n_e2e = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        upd = 0.0
        for _ in range(n_e2e):
            _, _, st, _ = e2e_step()
            upd += st["updates"]
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        dist.barrier()
        ev, _ = aggregate(dist, te, upd)
        e2e = {"value": ev, "unit": "updates/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": 1e3 * te / n_e2e}
        ctx2.close()

    cpu = None
    if dist.rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(p, law=args.law)
    ctx.close()
    others = None
    if dist.rank == 0 and not args.no_others and args.workload == "periodic" and args.cells is None:
        others = other_configs(args, stream)
    if dist.rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": dist.world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOADS[args.workload], "n_cells": N, "n_dir": D, "n_groups": G,
                          "face_sides_per_cell": round(fbar, 3), "precision": "FP32 intensities, FP64 tallies",
                          "l2": "no flush: >10 GB resident working set, 78x the 129 MB L2",
                          "step": step_text(p, args.fused_loops), "fused_loops": args.fused_loops,
                          "law": args.law, "transport": "scheme (a)" if args.transport == 0 else
                          "scheme (b), direction-conserving to %d neighbours" % args.transport,
                          "parallelism": "one independent box per GPU" if dist.world > 1 else "1 GPU"},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": agg["launches"],
               "clocks": clk,
               "solve": {"it_pbc": agg["it_pbc"], "it_scat": agg["it_scat"], "defect_max": max(abs(x) for x in agg["defect"]),
                         "res_pbc": max(agg["res_pbc"]), "depth_max": last["depth_max"],
                         "depth_mean": last["depth_mean"], "classify_ms": agg["classify_ms"] / args.steps,
                         "levelise_ms": agg["levelise_ms"] / args.steps,
                         "assemble_ms": agg["assemble_ms"] / args.steps,
                         "sweep_ms_per_launch": avg_launch_s * 1e3,
                         "schedule": {1: "level", 2: "dataflow"}.get(last["schedule_used"], last["schedule_used"]),
                         "lanes_per_task": last["lanes_used"], "threads_per_block": last["threads_used"],
                         "blocks_per_sm": last["blocks_per_sm_used"],
                         "iterations_as_cuda_graphs": bool(last["graph_used"])}}
        out.update(extra)
        if others is not None:
            out["other_configs"] = others
        print(json.dumps(out))


def run_adjoint(args, dist: Dist):
    """The differentiation workload: each step is one adjoint call (forward intensities recomputed, then
    the transposed sweep), timed with CUDA events; inputs resident on the device."""
    import torch

    import __graft_entry__
    torch.cuda.set_device(dist.local)
    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    clocks = Clocks(dist.local)
    clocks.start()
    time.sleep(0.3)
    dist.barrier()
    e = adjoint_entry(args, stream, measured_peaks(), steps=args.steps, warmup=args.warmup,
                      cpu=dist.rank == 0 and not args.no_cpu, e2e=not args.no_e2e, rank=dist.rank)
    dist.barrier()
    clk = clocks.stop()
    elapsed = e["ms_per_step"] * args.steps / 1e3
    value, tmax = aggregate(dist, elapsed, e["value"] * elapsed)
    if dist.rank != 0:
        return
    print(json.dumps({"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": dist.world, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": WORKLOADS["adjoint"], "n_cells": e["n_cells"], "n_dir": e["n_dir"],
                                 "n_groups": e["n_groups"],
                                 "step": "one adjoint call: forward recompute + transposed sweep + FP64 gradients"},
                      "roofline": e["roofline"], "cpu_baseline": e.get("cpu_baseline"), "e2e": e.get("e2e"),
                      "gpu_launches": e["gpu_launches"], "clocks": clk, "solve": e["solve"]}))


# ---------------------------------------------------------------------------------------------
# The other configurations of the benchmark set, measured after the headline (outside its timed
# region): a few solves each, CUDA events on the context's stream, inputs resident in HBM.
def _timed(stream, fn, steps: int, warmup: int):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    outs = [fn() for _ in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3, outs


def _roof(p, sweep_ms: float, peaks: dict, kernel: str, law: str = "balance") -> dict:
    bpu, fbar = bytes_per_update(p, law)
    upd = p.mesh.n_cells * p.n_dir * p.n_groups
    ach = bpu * upd / (sweep_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "peak_source": peaks["source"], "bytes_per_update": bpu,
            "avg_launch_ms": sweep_ms}


def _roof_sweeps(p, sweep_ms_total: float, n_sweeps: int, updates: float, peaks: dict, kernel: str) -> dict:
    """Roofline over sweeps of different group counts (the adjoint: forward sweeps over G groups, transposed
    sweeps over 2G split groups): per sweep every task reads its row (8 B + 16 B per face side), per
    update the source pair and the write (12 B)."""
    m = p.mesh
    fbar = (2 * m.n_faces - int((m.face_cells[:, 1] < 0).sum())) / m.n_cells
    alg = m.n_cells * p.n_dir * (8.0 + 16.0 * fbar) * n_sweeps + 12.0 * updates
    ach = alg / (sweep_ms_total / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "peak_source": peaks["source"], "bytes_per_update": alg / updates,
            "avg_launch_ms": sweep_ms_total / max(1, n_sweeps)}


def _solve_entry(name: str, workload: str, p, ctx, stream, opts, steps: int, warmup: int, peaks: dict) -> dict:
    import torch
    from paper_2207_12848_gb300._lib import KERNELS
    N, D, G = p.mesh.n_cells, p.n_dir, p.n_groups
    J = torch.empty((N, G), dtype=torch.float64, device="cuda")
    Gm = torch.empty_like(J)
    dt, outs = _timed(stream, lambda: ctx.solve_dev(J, Gm, opts)[0], steps, warmup)
    st = outs[-1]
    upd = sum(o["updates"] for o in outs)
    sweep_ms = sum(o["t_sweep_ms"] for o in outs) / max(1, sum(o["sweep_launches"] for o in outs))
    return {"config": name, "workload": workload, "n_cells": N, "n_dir": D, "n_groups": G, "steps": steps,
            "value": upd / dt, "unit": "updates/s", "ms_per_step": 1e3 * dt / steps,
            "dtype": "f64" if opts.precision == 64 else "f32",
            "roofline": _roof(p, sweep_ms, peaks, KERNELS.get(st["kernel_used"], "?")) if st["sweep_launches"] else None,
            "solve": {"depth_max": st["depth_max"], "depth_mean": st["depth_mean"], "it_scat": st["it_scat"],
                      "it_pbc": st["it_pbc"], "n_sweeps": st["n_sweeps"], "defect": st["defect"],
                      "classify_ms": st["t_classify_ms"], "levelise_ms": st["t_levelise_ms"],
                      "assemble_ms": st["t_assemble_ms"], "sweep_ms_per_launch": sweep_ms}}


def other_configs(args, stream) -> list:
    """Configurations 1, 2, 3 and 5 of the benchmark set (the headline is configuration 4)."""
    import numpy as np
    import torch

    import oracle
    from paper_2207_12848_gb300 import Context, default_opts
    from synth import configs
    peaks = measured_peaks()
    out = []
    th = args.threads
    # 1: 32^3 lattice, FP64: the batched sweep, the plain per-(direction, level) sweep, the oracle on one core
    p = configs.plain32()
    with Context(0, stream.cuda_stream) as ctx:
        ctx.set_mesh(p.mesh)
        ctx.set_directions(p.omega, p.weight)
        ctx.set_material(torch.from_numpy(p.kappa_abs).cuda(), torch.from_numpy(p.emissivity).cuda())
        e = _solve_entry("1 (plain method, FP64)", "32^3 lattice Voronoi mesh, vacuum, tau=0.1 per cell, unit "
                         "source at the centre, 16 directions, 1 group", p, ctx, stream,
                         default_opts(precision=64, relevel=1), 5, 3, peaks)
        ep = _solve_entry("1", "", p, ctx, stream, default_opts(schedule="plain", relevel=1), 2, 1, peaks)
        e["plain_fp64"] = {"value": ep["value"], "unit": "updates/s", "ms_per_step": ep["ms_per_step"],
                           "sweep_launches_per_step": 0, "speedup_batched_vs_plain": e["value"] / ep["value"]}
        t0 = time.perf_counter()
        oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, threads=1)
        dt = time.perf_counter() - t0
        e["cpu_baseline"] = {"value": p.mesh.n_cells * p.n_dir / dt, "unit": "updates/s", "cores": 1,
                             "kind": "oracle", "sample": "the whole configuration, one FP64 solve (%.2f s)" % dt}
        out.append(e)
    # 2: 64 uneven meshes in one launch, 2 groups, one sweep per solve
    p = configs.batched(threads=th)
    with Context(0, stream.cuda_stream) as ctx:
        ctx.set_mesh(p.mesh)
        ctx.set_directions(p.omega, p.weight)
        ctx.set_material(torch.from_numpy(p.kappa_abs).cuda(), torch.from_numpy(p.emissivity).cuda())
        out.append(_solve_entry("2 (batched)", WORKLOADS["batched"], p, ctx, stream,
                                default_opts(precision=32, relevel=1), 3, 2, peaks))
    del p
    # 3: scattering, source iteration to 1e-6 as CUDA graphs
    p = configs.scatter(threads=th)
    with Context(0, stream.cuda_stream) as ctx:
        ctx.set_mesh(p.mesh)
        ctx.set_directions(p.omega, p.weight)
        ks = torch.from_numpy(p.kappa_scat).cuda()
        ctx.set_material(torch.from_numpy(p.kappa_abs).cuda(), torch.from_numpy(p.emissivity).cuda(), kappa_scat=ks)
        out.append(_solve_entry("3 (scattering)", WORKLOADS["scatter"], p, ctx, stream,
                                default_opts(precision=32, relevel=1, tol_scat=1e-6, max_it_scat=200), 2, 1, peaks))
    del p
    # 5: the adjoint
    out.append(adjoint_entry(args, stream, peaks, steps=3, warmup=2))
    return out


def adjoint_entry(args, stream, peaks: dict, steps: int, warmup: int, cpu: bool = True, e2e: bool = True,
                  rank: int = 0) -> dict:
    """One adjoint call per step (forward intensities recomputed, transposed sweep, FP64 gradients) on the
    differentiation configuration, with the oracle's adjoint on a bounded sample and the host-pointer call."""
    import numpy as np
    import torch

    import oracle
    from paper_2207_12848_gb300 import Context, default_opts
    from paper_2207_12848_gb300._lib import KERNELS
    p = make_problem("adjoint", rank, args.threads, args.cells)
    N, D, G = p.mesh.n_cells, p.n_dir, p.n_groups
    rng = np.random.default_rng(5)
    ka_t = p.kappa_abs * (1.0 + 0.1 * rng.standard_normal(p.kappa_abs.shape)).clip(0.5, 1.5)
    with Context(0, stream.cuda_stream) as ctx:
        ctx.set_mesh(p.mesh)
        ctx.set_directions(p.omega, p.weight)
        ctx.set_material(ka_t, p.emissivity)
        _, T, _, _ = ctx.solve(precision=32)  # target: absorbed rate of the perturbed kappa
        ctx.set_material(torch.from_numpy(p.kappa_abs).cuda(), torch.from_numpy(p.emissivity).cuda())
        J = torch.empty((N, G), dtype=torch.float64, device="cuda")
        Gm = torch.empty_like(J)
        ctx.solve_dev(J, Gm, default_opts(precision=32))
        sf, _ = ctx.solve_dev(J, Gm, default_opts(precision=32))  # the forward sweep alone, for comparison
        dg = 2.0 * (Gm - torch.from_numpy(T).cuda())
        gk, ge = torch.empty_like(J), torch.empty_like(J)
        opts = default_opts(precision=32)
        dt, outs = _timed(stream, lambda: ctx.adjoint_dev(gk, ge, None, dg, opts), steps, warmup)
        upd = sum(o["updates"] for o in outs)
        sweeps = sum(o["n_sweeps"] for o in outs)
        t_sw = sum(o["t_sweep_ms"] for o in outs)
        st = outs[-1]
        e = {"config": "5 (differentiation)", "workload": WORKLOADS["adjoint"], "n_cells": N, "n_dir": D,
             "n_groups": G, "steps": steps, "value": upd / dt, "unit": "updates/s", "ms_per_step": 1e3 * dt / steps,
             "dtype": "f32", "roofline": _roof_sweeps(p, t_sw, sweeps, upd, peaks, KERNELS.get(st["kernel_used"], "?")),
             "gpu_launches": sum(o["kernel_launches"] for o in outs),
             "solve": {"depth_max": st["depth_max"], "forward_sweeps": st["it_scat"], "transposed_passes": st["it_pbc"],
                       "sweeps": st["n_sweeps"], "sweep_ms_per_launch": t_sw / max(1, sweeps),
                       "assemble_ms": st["t_assemble_ms"]}}
        e["forward_roofline"] = _roof(p, sf["t_sweep_ms"] / max(1, sf["sweep_launches"]), peaks,
                                      KERNELS.get(sf["kernel_used"], "?"))
        n_tr = sum(o["it_pbc"] for o in outs)  # transposed passes
        e["transposed_roofline"] = _roof_sweeps(p, sum(o["t_transposed_ms"] for o in outs), n_tr,
                                                float(N * D * 2 * G * n_tr), peaks, KERNELS.get(st["kernel_used"], "?"))
        # accuracy of the FP32 gradients against the FP64 adjoint of the same inputs
        gk64, ge64 = torch.empty_like(J), torch.empty_like(J)
        ctx.adjoint_dev(gk64, ge64, None, dg, default_opts(precision=64))
        acc = {}
        for name, a, b in (("grad_kappa_abs", gk, gk64), ("grad_emissivity", ge, ge64)):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            big = np.abs(b) >= 1e-3 * np.abs(b).max()
            rel = np.abs(a[big] - b[big]) / np.abs(b[big])
            acc[name] = {"max_abs_err_over_max": float(np.abs(a - b).max() / np.abs(b).max()),
                         "rel_err_p50": float(np.percentile(rel, 50)), "rel_err_p99": float(np.percentile(rel, 99)),
                         "rel_err_max": float(rel.max()), "outputs_compared": int(big.sum())}
        e["fp32_vs_fp64"] = acc
        dgh = dg.cpu().numpy()
        if e2e:
            # through the host-pointer call: the loss gradient in, both gradients out, copies included
            gkh = torch.empty((N, G), dtype=torch.float64).pin_memory().numpy()
            dgp = torch.from_numpy(dgh).pin_memory().numpy()
            t0 = time.perf_counter()
            u2 = 0.0
            for _ in range(steps):
                a, b, s2 = ctx.adjoint(dl_dGamma=dgp, opts=opts)
                u2 += s2["updates"]
            torch.cuda.synchronize()
            te = time.perf_counter() - t0
            e["e2e"] = {"value": u2 / te, "unit": "updates/s", "h2d_bytes_per_step": dgp.nbytes,
                        "d2h_bytes_per_step": 2 * N * G * 8, "ms_per_step": 1e3 * te / steps}
        # the forward sweep at the transposed sweep's width (2G groups, same mesh): the like-for-like comparison
        ka2, em2 = np.tile(p.kappa_abs, (1, 2)), np.tile(p.emissivity, (1, 2))
        ctx.set_material(ka2, em2)
        J2 = torch.empty((N, 2 * G), dtype=torch.float64, device="cuda")
        G2m = torch.empty_like(J2)
        ctx.solve_dev(J2, G2m, default_opts(precision=32))
        s2, _ = ctx.solve_dev(J2, G2m, default_opts(precision=32))
        p2 = dataclasses.replace(p, kappa_abs=ka2, emissivity=em2)
        e["forward_roofline_2G"] = _roof(p2, s2["t_sweep_ms"] / max(1, s2["sweep_launches"]), peaks,
                                         KERNELS.get(s2["kernel_used"], "?"))
    if cpu:
        # the oracle's adjoint (forward solve + transposed sweep) on the host cores, on a sample of directions
        cores = os.cpu_count() or 1
        nd = min(D, max(1, cores))
        om, w = p.omega[:nd], np.full(nd, 4 * math.pi / nd)
        t0 = time.perf_counter()
        oracle.adjoint(p.mesh, om, w, p.kappa_abs, p.emissivity, dl_dGamma=dgh, threads=nd)
        dt = time.perf_counter() - t0
        e["cpu_baseline"] = {"value": N * nd * G * 3.0 / dt, "unit": "updates/s", "cores": nd, "kind": "oracle",
                             "sample": "one FP64 adjoint (forward sweep + transposed sweep over 2G split groups) of %d "
                                       "of %d directions over all %d cells, %.1f s" % (nd, D, N, dt)}
    return e


def run_profile_case(args):
    """Small fixed case for ncu captures: one solve with two sweeps, no autotuning, no extras."""
    import torch

    import __graft_entry__
    from paper_2207_12848_gb300 import Context, default_opts
    __graft_entry__.build()
    p = make_problem(args.workload, 0, args.threads, args.cells or 1 << 20)
    ctx = Context(0, torch.cuda.current_stream().cuda_stream)
    ctx.set_mesh(p.mesh)
    ctx.set_directions(p.omega, p.weight)
    ctx.set_material(p.kappa_abs, p.emissivity)
    o = default_opts(precision=32, schedule=args.schedule, lanes_per_task=args.lanes,
                     block_threads=128 if args.lanes == 1 else 256, blocks_per_sm=args.bpsm, max_it_pbc=2, tol_pbc=0.0,
                     op_format=args.op_format, packets_per_step=args.pps)
    ctx.solve(o)  # warm-up: module loading, first-touch of buffers
    J, G, st, s = ctx.solve(o)
    ctx.close()
    print(json.dumps({"profile_case": args.workload, "n_cells": p.mesh.n_cells, "sweeps": st["n_sweeps"],
                      "sweep_ms_per_launch": st["t_sweep_ms"] / max(1, st["n_sweeps"]),
                      "levelise_ms": st["t_levelise_ms"], "assemble_ms": st["t_assemble_ms"],
                      "depth_max": st["depth_max"], "kernel": st["kernel_used"], "lanes": st["lanes_used"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="periodic", choices=sorted(WORKLOADS))
    ap.add_argument("--threads", type=int, default=None)
    ap.add_argument("--cells", type=int, default=None, help="smaller problem (testing only; not a bench line)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the plain-FP64 comparison sweep")
    ap.add_argument("--no-others", action="store_true", help="skip the other configurations after the headline")
    ap.add_argument("--law", default="balance", choices=["balance", "exp"],
                    help="absorption law of the cell update (exp: transmission exp(-tau) across the mean chord)")
    ap.add_argument("--transport", type=int, default=0, choices=range(0, 9),
                    help="transport scheme of Sec. 2.6: 0 = (a); n = (b), direction-conserving to n neighbours")
    ap.add_argument("--fused-loops", type=int, default=0, choices=[0, 1],
                    help="with scattering and periodic faces: one sweep per periodic iteration (Sec. 2.7)")
    ap.add_argument("--profile-case", action="store_true", help="small fixed solve for ncu captures")
    ap.add_argument("--schedule", default="dataflow", choices=["level", "dataflow"])
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 1, 2, 4, 8, 16],
                    help="profiling case: lanes per task over 128-byte lines (0 = the packed operator)")
    ap.add_argument("--op-format", default="auto", choices=["auto", "lines", "packets"])
    ap.add_argument("--pps", type=int, default=0, choices=[0, 1, 2], help="packets per warp step (0 = autotuned)")
    ap.add_argument("--bpsm", type=int, default=0, help="resident blocks per SM (profiling case)")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    dist = Dist("gloo" if args.impl == "reference" else None)
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        elif args.workload == "adjoint":
            run_adjoint(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
