#!/usr/bin/env python
"""Benchmark of the localized model-order-reduction hot path on one GB300.

A step = step 2 + step 3 of the method on one batch: mor_build_bases (assembly,
sketch, the four batched local solves, weighted randomized SVD, stitching and the
diagonal-block update) + mor_project (interface-only Q^T A Q) + mor_solve_reduced,
MOR_MIXED precision, on device-resident inputs (the mesh and the step-1 subdomain
plan are built once before timing; step 1 is timed separately and inside `e2e`).

value  = basis columns produced per second (all ranks' columns / the slowest rank's
         time); the FP64 GPU path and its energy distance to the mixed result are
         reported beside it (time-to-reduced-solution).
e2e    = the same metric through the public Python API from host buffers: pinned
         host -> device copy of the mesh, step 1 on the host, steps 2-3, and the
         device -> host read of the reduced solution, every step.
--impl reference runs the CPU oracle (test infrastructure, plain FP64 NumPy/SciPy) on
a bounded sample of the same workload: one subdomain's local basis per step.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "basis cols/s; time-to-reduced-solution at ≤1e-6 rel energy err vs FP64 GPU"
UNIT = "basis cols/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cube64_p4")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison step")
    ap.add_argument("--wave", type=int, default=0,
                    help="build a streamed plan and run the bases in waves of this many "
                         "subdomains (the 440^3 workload)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one mixed-precision build of the workload and exit (the "
                         "command profiled by ncu)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_opts(p):
    """Sketch widths of a workload: one rank for all subdomains, or seeded
    per-subdomain ranks (uneven batches)."""
    kw = dict(rank=p["rank"], oversample=p["oversample"], seed=p["seed"])
    if "ranks" in p:
        kw["ranks"] = p["ranks"]
    return kw


def mixed_rtol(p):
    """Local-solve tolerance of the mixed path: 1e-9, or tighter where the coefficient
    contrast makes the energy error of a solve larger (about rtol sqrt(cond A_II))."""
    return p.get("mixed_rtol", 1e-9)


def first_rank(p):
    return int(p["ranks"][0]) if "ranks" in p else p["rank"]


def reduce_over_ranks(t_ms, cols, world, device):
    """Whole-job figures of the replicas: the slowest rank's time and the basis columns
    of all ranks (value = columns / that time).  One process per GPU; `device` is the
    tensor device of the process group's backend."""
    if world == 1:
        return float(t_ms), float(cols)
    import torch
    import torch.distributed as dist
    tmax = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    tot = torch.tensor([float(cols)], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tot[0])


class Clocks:
    """nvidia-smi samples during the timed region (every 200 ms)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def ncu_traffic(kernel_key):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, if its source
    fingerprint still matches the current sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        data = json.load(fh)
    entry = data.get(kernel_key)
    if not entry:
        return None
    from paper_2404_06260_gb300 import _build
    if entry.get("source_fingerprint") != _build.source_fingerprint():
        return None
    return entry.get("dram_bytes_per_launch_scaled")


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    import synth
    from oracle import basis, subdomains
    mesh, kappa, owner, p = synth.workload(args.workload)
    adj = subdomains.node_adjacency(mesh.tets, mesh.n_nodes)
    sub = 0   # the smallest (corner) subdomain: an upper bound on the oracle's rate
    s = subdomains.subdomain_sets(mesh, owner, sub, p["r_hops"], adj)

    def step():
        b = basis.local_basis(mesh, kappa, s, first_rank(p), p["oversample"], p["seed"])
        return b["n_kept"]

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    cols = 0
    for _ in range(args.steps):
        cols += step()
    dt = time.perf_counter() - t0
    val = cols / dt
    cores = os.cpu_count()
    sample = ("oracle local basis of subdomain %d of %s (|I|=%d, |B|=%d), %d steps; the "
              "corner subdomain is the cheapest, so this is an upper bound on the oracle's "
              "rate over the whole batch" % (sub, args.workload, len(s["I"]), len(s["B"]),
                                             args.steps))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "subdomains": 1, "rank": first_rank(p),
                   "oversample": p["oversample"]},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def cpu_baseline(args):
    import synth
    from oracle import basis, subdomains
    mesh, kappa, owner, p = synth.workload(args.workload)
    adj = subdomains.node_adjacency(mesh.tets, mesh.n_nodes)
    s = subdomains.subdomain_sets(mesh, owner, 0, p["r_hops"], adj)
    t0 = time.perf_counter()
    b = basis.local_basis(mesh, kappa, s, first_rank(p), p["oversample"], p["seed"])
    dt = time.perf_counter() - t0
    return {"value": b["n_kept"] / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle local basis (field sketch, FP64, sparse LU + dense LAPACK) of "
                      "subdomain 0 of %s, the smallest (corner) subdomain: %.1f s for %d "
                      "columns; an upper bound on the oracle's rate over the batch"
                      % (args.workload, dt, b["n_kept"])}


def ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    from paper_2404_06260_gb300 import _build
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    from paper_2404_06260_gb300 import mor

    mesh, kappa, owner, p = synth.workload(args.workload)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"], wave=args.wave)
    a1_ms = 1e3 * (time.perf_counter() - t0)
    mixed = mor.basis_opts(precision="mixed", cg_rtol=mixed_rtol(p), **rank_opts(p))
    fp64 = mor.basis_opts(precision="fp64", cg_rtol=min(1e-10, mixed_rtol(p)),
                          **rank_opts(p))

    def step(opts):
        b = mor.Bases(sd, opts)
        r = mor.Reduced(sd, b)
        x, info = r.solve(rtol=1e-10)
        return b, r, x, info

    for _ in range(args.warmup):
        step(mixed)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    mor.profile_reset()
    mor.profile(True)
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = mor.kernel_launches()
    cols = 0
    for i in range(args.steps):
        flush.zero_()                        # L2 flush between steps (untimed)
        ev[i][0].record(stream)
        b, r, x, info = step(mixed)
        ev[i][1].record(stream)
        cols += b.total_kept
    torch.cuda.synchronize()
    launches = mor.kernel_launches() - launches0
    clk = clocks.stop()
    mor.profile(False)
    if world > 1:
        dist.barrier()
    t_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    t_max, tot_cols = reduce_over_ranks(t_ms, cols, world, "cuda")
    value = tot_cols / (t_max / 1e3)

    # dominant kernel of the timed region and its roofline
    fams = {f: mor.profile_query(f) for f in mor.KERNEL_FAMILIES}
    dom = max(fams, key=lambda f: fams[f]["ms"])
    fd = fams[dom]
    peaks, src = measured_peaks()
    per_launch_bytes = fd["bytes"] / max(fd["launches"], 1)
    per_launch_s = fd["ms"] / max(fd["launches"], 1) / 1e3
    achieved = per_launch_bytes / per_launch_s / 1e9
    roof = {"bound": "hbm", "kernel": mor.KERNEL_FAMILIES[dom], "achieved": achieved,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
            "peak_source": src, "launches": int(fd["launches"]),
            "algorithmic_bytes_per_launch": per_launch_bytes,
            "traffic": ncu_traffic(mor.KERNEL_FAMILIES[dom]),
            "time_share_of_step": fd["ms"] / t_ms,
            "families": {mor.KERNEL_FAMILIES[f]: {"ms": fams[f]["ms"],
                                                 "launches": int(fams[f]["launches"]),
                                                 "GBps": (fams[f]["bytes"] / fams[f]["ms"] / 1e6
                                                          if fams[f]["ms"] > 0 else None)}
                         for f in fams}}

    extra = {}
    if not args.no_fp64:
        u_m = mor.lift(sd, b, x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        bd, rd, xd, infod = step(fp64)
        e1.record(stream)
        torch.cuda.synchronize()
        u_d = mor.lift(sd, bd, xd)
        err = mor.energy_norm(sd, u_m, u_d) / mor.energy_norm(sd, u_d)
        extra = {"time_to_reduced_solution_ms": {"mixed": t_ms / args.steps,
                                                 "fp64": e0.elapsed_time(e1)},
                 "energy_err_mixed_vs_fp64": err,
                 "fp64_converged": bool(bd.converged and infod["converged"])}

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(args, mor, mesh, kappa, owner, p, mixed, stream, world)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": args.workload, "mesh": "%d^3 cells x 6 Kuhn tets" % p["n"],
                   "subdomains": sd.n_sub,
                   "rank": ("per subdomain, %d..%d" % p["rank_range"]) if "ranks" in p
                   else p["rank"], "oversample": p["oversample"],
                   "r_hops": p["r_hops"], "precision": "mixed (f32 CG sweeps, f64 refinement "
                   "and small dense work)", "parallelism": "replicas x%d" % world,
                   "l2": "working set > L2 and a 256 MB L2 flush between steps",
                   "basis_cols_per_step": int(b.total_kept),
                   "cg_rtol": {"mixed": mixed_rtol(p), "fp64": min(1e-10, mixed_rtol(p))}},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "a1_host_ms": a1_ms,
        "local_solve_iterations": b.stats()[:5].tolist(),
        **extra,
    }
    if args.wave:
        out["config"]["plan"] = "streamed, waves of %d subdomains" % args.wave
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


def end_to_end(args, mor, mesh, kappa, owner, p, mixed, stream, world):
    """The same metric through the public API with the mesh in pinned host memory: every
    step copies it to the device, runs steps 1-3 and reads x back."""
    import torch
    xyz_h = torch.from_numpy(mesh.xyz).pin_memory()
    tets_h = torch.from_numpy(mesh.tets).pin_memory()
    kap_h = torch.from_numpy(kappa).pin_memory()
    h2d = (xyz_h.numel() * 8 + tets_h.numel() * 4 * 2 + kap_h.numel() * 8 +
           mesh.dirichlet.nbytes + owner.nbytes)
    e2e_ms, d2h, cols = [], 0, 0
    for i in range(args.steps):
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        gm2 = mor.Mesh.from_device(xyz_h.to("cuda", non_blocking=True),
                                   tets_h.to("cuda", non_blocking=True),
                                   kap_h.to("cuda", non_blocking=True),
                                   tets_h.numpy(), mesh.dirichlet)
        sd2 = mor.Subdomains(gm2, owner, p["r_hops"], wave=args.wave)
        b2 = mor.Bases(sd2, mixed)
        r2 = mor.Reduced(sd2, b2)
        x2, _ = r2.solve(rtol=1e-10)
        xh = x2.to("cpu", non_blocking=False)
        s1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(s0.elapsed_time(s1))
        d2h = xh.numel() * 8
        cols += b2.total_kept
        del sd2, b2, r2
    t_max, tot_cols = reduce_over_ranks(sum(e2e_ms), cols, world, "cuda")
    return {"value": tot_cols / (t_max / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": t_max / args.steps}


def profile_case(args):
    import torch

    import synth
    from paper_2404_06260_gb300 import _build
    _build.build()
    from paper_2404_06260_gb300 import mor
    mesh, kappa, owner, p = synth.workload(args.workload)
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    opts = mor.basis_opts(precision="mixed", cg_rtol=mixed_rtol(p), **rank_opts(p))
    b = mor.Bases(sd, opts)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.workload, "basis_cols": int(b.total_kept),
                      "iterations": b.stats()[:5].tolist()}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile_case:
        return profile_case(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
