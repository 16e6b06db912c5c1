"""The N > 1 benchmark path on CPU: two gloo ranks, each generating its own
replica graph (the generator does not shard; ranks share nothing but the
final timing reduction)."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle as O  # noqa: E402
from paper_1501_03545_gb300 import workloads as W  # noqa: E402

SMALL = W.scaled(W.LARGE, 3000)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica_entries(rank):
    w = SMALL
    R = O.solve_radius(w.n, w.alpha, w.kbar)
    r, phi = O.sample(w.n, w.alpha, R, bench.replica_seed(w, rank))
    off, _ = O.brute_csr(r, phi, R)
    return int(off[-1])


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        entries = _replica_entries(rank)
        ms = 10.0 * (rank + 1)
        dist.barrier()
        ms_max, total = bench.reduce_over_ranks(ms, entries, dist, torch.device("cpu"))
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"entries": entries, "ms_max": ms_max, "total": total}, f)
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_reduce(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % k))) for k in range(world)]
    serial = [_replica_entries(k) for k in range(world)]
    # each rank built its own, different graph of the same workload
    assert [r["entries"] for r in res] == serial
    assert serial[0] != serial[1]
    # every rank sees the slowest rank's time and the job's total output
    for r in res:
        assert r["ms_max"] == 20.0
        assert r["total"] == float(sum(serial))


def test_replica_seeds_distinct():
    seeds = [bench.replica_seed(W.LARGE, k) for k in range(8)]
    assert len(set(seeds)) == 8 and seeds[0] == W.LARGE.seed


def test_reference_arm_only_rank0_prints(capsys):
    class A:
        warmup = 0
        steps = 1
        gpus = 2
        oracle_n = 2000

    assert bench.run_reference(A, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""
    assert bench.run_reference(A, rank=0, world=2) == 0
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
