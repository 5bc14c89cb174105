"""The multi-process path of bench.py (replicas only: one process per GPU, each running
the whole workload), on the CPU with gloo at world size 2.

- The whole-job figures are the slowest rank's time and the basis columns of all ranks,
  so value = all columns / the slowest time (weak scaling).
- Under torchrun the reference arm runs on rank 0 alone; the other ranks return 0 at
  once, without work and without output.
"""
import argparse
import multiprocessing
import os
import socket
import sys

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    # rank r took 100 + 50 r ms for 2112 + r columns
    q.put((rank, bench.reduce_over_ranks(100.0 + 50.0 * rank, 2112 + rank, world, "cpu")))
    dist.destroy_process_group()


def test_replicas_report_slowest_time_and_all_columns():
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank holds the same whole-job figures
    assert out[0] == out[1] == (150.0, 2112.0 + 2113.0)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(12.5, 2112, 1, "cpu") == (12.5, 2112.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(workload="cube64_p4", steps=3, warmup=3, gpus=2)
    assert bench.reference_arm(args) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_times_the_oracle_over_a_process_pool(capsys):
    # one single-threaded spawn worker per core over the smallest subdomains, one JSON
    # line with the cores the pool used
    import json
    sys.path.insert(0, ROOT)
    import bench
    os.environ.pop("RANK", None)
    os.environ.pop("WORLD_SIZE", None)
    args = argparse.Namespace(workload="cube16_p2", steps=1, warmup=0, gpus=1)
    assert bench.reference_arm(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == min(os.cpu_count(), 8)
    assert line["config"]["subdomains"] == line["cpu_baseline"]["cores"]
