"""Host logic of the multi-GPU job, as two gloo ranks on the CPU.

Every rank runs its own replica (nothing crosses ranks on the data path); the
host coordinates the timed region: a barrier on both sides, the slowest rank's
time, and the whole-job rate from the units all ranks processed.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import time

    import torch
    import torch.distributed as dist

    import bench

    R = bench.Ranks(rank, world, backend="gloo")
    # a stand-in timed region whose length differs per rank
    R.barrier()
    t0 = time.perf_counter()
    time.sleep(0.05 * (rank + 1))
    R.barrier()
    local_ms = (time.perf_counter() - t0) * 1e3
    slowest = R.max(local_ms)
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(rank))
    units = 1000 * (rank + 1)
    got = torch.tensor([units], dtype=torch.int64)
    dist.all_reduce(got)
    value = bench.job_throughput(1000, world, slowest)

    class Args:
        steps, warmup = 1, 0
    # rank 0 would time the oracle on the 512^3 lattice; only the others' no-op is checked here
    ref = bench.reference_arm(Args, rank, world) if rank != 0 else "rank0-skipped"
    R.close()
    with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
        json.dump({"local_ms": local_ms, "slowest": slowest, "seeds": seeds, "value": value,
                   "units_sum": int(got.item()), "ref": ref}, f)


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / ("r%d.json" % k))) for k in range(2)]
    # both ranks hold the same maximum, and it is the slower rank's time
    assert r[0]["slowest"] == r[1]["slowest"]
    assert r[0]["slowest"] == pytest.approx(max(r[0]["local_ms"], r[1]["local_ms"]))
    assert r[0]["slowest"] >= 100.0
    # replicas differ by seed
    assert r[0]["seeds"] == [1, 2]
    # whole-job rate: units of both ranks over the slowest rank's time
    assert r[0]["value"] == pytest.approx(2000 / (r[0]["slowest"] * 1e-3))
    assert r[0]["units_sum"] == 3000
    # the reference arm runs on rank 0 only; the other ranks do no work
    assert r[1]["ref"] is None


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    R = bench.Ranks(0, 1, backend="gloo")
    R.barrier()
    assert R.max(3.5) == 3.5
    R.close()
    assert bench.job_throughput(100, 1, 1000.0) == pytest.approx(100.0)
