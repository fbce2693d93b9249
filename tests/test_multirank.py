"""The bench's multi-rank host logic on CPU (gloo, world size 2): each rank
decomposes its own replica with its own seed, the job's time is the slowest
rank's, and the value counts every rank's nonzeros against it."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as td
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    td.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist()
    ms = 10.0 + 5.0 * r                     # rank 1 is slower
    t = bench.max_over_ranks(ms, w)
    seeds = [None] * w
    td.all_gather_object(seeds, bench.rank_seed(r))
    out.put((r, w, local, t, bench.whole_job_value(1_000_000, w, t), seeds))
    td.barrier()
    td.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, t, value, seeds) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert t == 15.0                      # max over ranks
        assert value == pytest.approx(2_000_000 / 15e-3)
        assert len(set(seeds)) == 2           # independent replicas


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.whole_job_value(10, 1, 1.0) == 10_000.0


def test_reference_arm_rank0_only(monkeypatch, capsys):
    """Under torchrun the oracle's reference arm runs on rank 0 alone; the
    line carries the oracle's own throughput as value, cpu_baseline and e2e
    (no host-device bytes)."""
    import argparse
    import json
    sys.path.insert(0, ROOT)
    import bench
    calls = []

    def fake_sample():
        calls.append(1)
        return {"nnz": 1000, "seconds": 0.5, "err": 0.1, "dims": [30, 30, 3]}

    monkeypatch.setattr(bench, "run_oracle_sample", fake_sample)
    args = argparse.Namespace(gpus=2, steps=3, warmup=2, impl="reference")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.reference_arm(args)
    assert not calls and capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    bench.reference_arm(args)
    assert len(calls) == 5                    # warm-up + timed samples
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["value"] == pytest.approx(2000.0)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["steps"] == 3 and line["warmup"] == 2 and line["higher_is_better"] is True
