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
the host cores, one single-threaded process per core, on a bounded sample of the same
workload: the local bases of the `cores` smallest subdomains per step.
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
    ap.add_argument("--explicit-vs-randomized", action="store_true",
                    help="time the explicit weighted SVD (Eq. (14), dense factors) against "
                         "the randomized one on the 16^3 workload and exit (Sec. 7.2)")
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


def ncu_traffic(kernel_key, workload):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, if it was taken
    on this workload and its source fingerprint still matches the current sources (else
    None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        data = json.load(fh)
    entry = data.get(kernel_key)
    if not entry or not entry.get("workload", "").startswith(workload + " "):
        return None
    from paper_2404_06260_gb300 import _build
    if entry.get("source_fingerprint") != _build.source_fingerprint():
        return None
    return entry.get("dram_bytes_per_launch_scaled")


_ORACLE_CACHE = {}


def _oracle_subdomain(task):
    """One subdomain's local basis by the oracle (a process-pool task): returns
    (subdomain, basis columns, seconds)."""
    workload, sub = task
    import synth
    from oracle import basis, subdomains
    if workload not in _ORACLE_CACHE:
        mesh, kappa, owner, p = synth.workload(workload)
        adj = subdomains.node_adjacency(mesh.tets, mesh.n_nodes)
        _ORACLE_CACHE.clear()
        _ORACLE_CACHE[workload] = (mesh, kappa, owner, p, adj)
    mesh, kappa, owner, p, adj = _ORACLE_CACHE[workload]
    t0 = time.perf_counter()
    s = subdomains.subdomain_sets(mesh, owner, sub, p["r_hops"], adj)
    m = int(p["ranks"][sub]) if "ranks" in p else p["rank"]
    b = basis.local_basis(mesh, kappa, s, m, p["oversample"], p["seed"])
    return sub, int(b["n_kept"]), time.perf_counter() - t0


def oracle_pool(cores):
    """A pool of `cores` single-threaded oracle processes.  Started with spawn, so that no
    worker is forked from a process holding a CUDA context; each worker runs one BLAS
    thread, so the pool uses exactly `cores` threads."""
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    return mp.get_context("spawn").Pool(processes=cores)


def oracle_extension_sizes(workload):
    """|I| + |B| of every subdomain of a workload (the oracle's own sets)."""
    import numpy as np
    import synth
    from oracle import subdomains
    mesh, kappa, owner, p = synth.workload(workload)
    adj = subdomains.node_adjacency(mesh.tets, mesh.n_nodes)
    n_sub = int(owner.max()) + 1
    out = np.zeros(n_sub, dtype=np.int64)
    for i in range(n_sub):
        s = subdomains.subdomain_sets(mesh, owner, i, p["r_hops"], adj)
        out[i] = len(s["I"]) + len(s["B"])
    return out


def reference_arm(args):
    """The oracle on the host cores: every step runs the local bases of the `cores`
    subdomains with the smallest extensions, one per single-threaded process, and the
    metric is their basis columns over the step's wall time.  The smallest subdomains
    keep a step near one subdomain's oracle time (the run must end within minutes), so
    the rate over-states the oracle's rate on the whole batch, whose larger subdomains
    take up to about 3x longer."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import synth
    p = synth.workload(args.workload)[3]
    cores = os.cpu_count() or 1
    sizes = oracle_extension_sizes(args.workload)
    sample = [int(i) for i in np.argsort(sizes, kind="stable")[:cores]]
    pool = oracle_pool(len(sample))
    try:
        tasks = [(args.workload, i) for i in sample]
        pool.map(_oracle_subdomain, tasks[:1])   # worker start-up (untimed)
        for _ in range(args.warmup):
            pool.map(_oracle_subdomain, tasks)
        t0 = time.perf_counter()
        cols = 0
        for _ in range(args.steps):
            cols += sum(c for _, c, _ in pool.map(_oracle_subdomain, tasks))
        dt = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    val = cols / dt
    desc = ("oracle local bases (field sketch, FP64, SuperLU + LAPACK) of the %d subdomains "
            "of %s with the smallest extensions (|I|+|B| %d..%d of %d..%d over the batch), "
            "one per single-threaded process on %d host cores, %d steps; an upper bound "
            "on the oracle's rate over the whole batch"
            % (len(sample), args.workload, sizes[sample].min(), sizes[sample].max(),
               sizes.min(), sizes.max(), len(sample), args.steps))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "subdomains": len(sample),
                   "rank": first_rank(p), "oversample": p["oversample"]},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": len(sample), "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def cpu_baseline(args):
    """The oracle over the host cores on a seeded random sample of the batch: one
    subdomain per single-threaded process, `cores` subdomains, one round."""
    import numpy as np
    import synth
    cores = os.cpu_count() or 1
    mesh, kappa, owner, p = synth.workload(args.workload)
    n_sub = int(owner.max()) + 1
    rng = np.random.default_rng(12345)
    sample = sorted(int(i) for i in rng.choice(n_sub, size=min(cores, n_sub), replace=False))
    pool = oracle_pool(len(sample))
    try:
        pool.map(_oracle_subdomain, [(args.workload, sample[0])])   # start-up (untimed)
        t0 = time.perf_counter()
        res = pool.map(_oracle_subdomain, [(args.workload, i) for i in sample])
        dt = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    cols = sum(c for _, c, _ in res)
    per = [t for _, _, t in res]
    return {"value": cols / dt, "unit": UNIT, "cores": len(sample), "kind": "oracle",
            "sample": "oracle local bases (field sketch, FP64, SuperLU + LAPACK) of %d "
                      "subdomains of %s drawn at random (seed 12345) from all %d, one per "
                      "single-threaded process on %d host cores: %.1f s wall for %d "
                      "columns; per subdomain %.1f..%.1f s (mean %.1f), so the whole "
                      "batch would take about %.0f s on these cores (extrapolated)"
                      % (len(sample), args.workload, n_sub, len(sample), dt, cols,
                         min(per), max(per), float(np.mean(per)),
                         float(np.mean(per)) * n_sub / len(sample))}


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
            "traffic": ncu_traffic(mor.KERNEL_FAMILIES[dom], args.workload),
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
        "autotune": mor.autotune_report(),
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
    step hands the host arrays to step 1 (mor_build_subdomains_host copies them to the
    device inside the call while it builds the plan on the host), runs steps 2-3 and
    reads x back."""
    import torch
    xyz_h = torch.from_numpy(mesh.xyz).pin_memory()
    tets_h = torch.from_numpy(mesh.tets).pin_memory()
    kap_h = torch.from_numpy(kappa).pin_memory()
    dir_h = torch.from_numpy(mesh.dirichlet).pin_memory()
    h2d = xyz_h.numel() * 8 + tets_h.numel() * 4 + kap_h.numel() * 8
    e2e_ms, d2h, cols = [], 0, 0
    for i in range(args.steps):
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        sd2 = mor.Subdomains.from_host(xyz_h, tets_h, kap_h, dir_h, owner, p["r_hops"],
                                       wave=args.wave)
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
            "d2h_bytes_per_step": int(d2h), "ms_per_step": t_max / args.steps,
            "inputs": "coordinates, connectivity and coefficient copied by the library "
                      "(mor_build_subdomains_host); step 1 reads the host arrays"}


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


def explicit_vs_randomized(args):
    """Step 2 (mor_build_bases, binary64) on the 16^3 workload three ways: the field
    sketch with k = m + p columns, the paper's sketch W = R_BB^{-1} S (dense Cholesky
    of H^+), and the explicit weighted SVD of R_i Z_i R_BB^{-1} (dense factors of
    A_II, H_i, H^+).  CUDA-event times, median of 5 after 2 warm-up builds."""
    import torch

    import synth
    from paper_2404_06260_gb300 import _build
    _build.build()
    from paper_2404_06260_gb300 import mor
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    stream = torch.cuda.current_stream()
    variants = {
        "randomized_field": mor.basis_opts(rank=p["rank"], oversample=p["oversample"],
                                           seed=p["seed"], precision="fp64", cg_rtol=1e-13),
        "randomized_paper_sketch": mor.basis_opts(rank=p["rank"], oversample=p["oversample"],
                                                  seed=p["seed"], precision="fp64",
                                                  cg_rtol=1e-13, sketch="paper"),
        "explicit": mor.basis_opts(rank=p["rank"], oversample=0, seed=p["seed"],
                                   precision="fp64", explicit_svd=1),
    }
    out = {}
    for name, o in variants.items():
        for _ in range(2):
            mor.Bases(sd, o)
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            b = mor.Bases(sd, o)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[name] = {"ms": statistics.median(ts), "basis_cols": int(b.total_kept),
                     "sigma_1": float(b.sigma()[:, 0].max())}
    print(json.dumps({"workload": "cube16_p2", "n_sub": sd.n_sub, "rank": p["rank"],
                      "B_sizes": [int(sd.counts[:, 1].min()), int(sd.counts[:, 1].max())],
                      "builds": out,
                      "explicit_over_randomized": out["explicit"]["ms"] /
                      out["randomized_field"]["ms"]}))
    return 0


def main():
    args = parse()
    if args.explicit_vs_randomized:
        return explicit_vs_randomized(args)
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile_case:
        return profile_case(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
