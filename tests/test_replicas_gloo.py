"""The N > 1 host path of bench.py on CPU: two gloo ranks (replicas, no data-
path collective; the only collective is the max over ranks of the step time)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    # rank r took 100 * (r + 1) ms for 3e12 flops of its own work
    ms, value = bench.whole_job(100.0 * (rank + 1), 3e12, world)
    bench.barrier(world)
    out.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(out.get() for _ in range(world))
    for rank, ms, value in got:
        assert ms == 200.0                       # the slowest rank's time, on every rank
        assert value == pytest.approx(2 * 3e12 / 0.2 / 1e12)   # all ranks' work / that time


def test_reference_arm_rank1_exits_without_work(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "time_oracle", lambda *a, **k: called.append(a) or (1.0, 1))
    import argparse
    bench.run_reference(argparse.Namespace(workload="f64_8192", steps=1, warmup=0))
    assert called == [] and capsys.readouterr().out == ""
