"""CPU, world_size 2 over gloo: the bench's multi-rank host logic — the job
time is the maximum over ranks, the value counts every rank's units, and the
reference arm prints only on rank 0 (the path shards into independent
replicas, so there is no data-path collective to test)."""
import contextlib
import io
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, e2e = bench.max_over_ranks([10.0 + 5 * rank, 30.0 - rank], world)
        value = bench.job_throughput(1000, 4, world, ms)
        out.put((rank, ms, e2e, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, e2e, value in got:
        assert ms == 15.0 and e2e == 30.0              # every rank sees the slowest rank's times
        assert value == pytest.approx(1000 * 4 * 2 / 15e-3)


def test_single_process_is_identity():
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.job_throughput(10, 3, 1, 2.0) == pytest.approx(15000.0)


def test_reference_arm_prints_on_rank0_only(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = bench.argparse.Namespace(steps=1, warmup=0, gpus=2)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""
