"""Multi-rank logic of bench.py on CPU with the gloo backend (world size 2):
replicas report the whole-job throughput over the slowest rank's time, and
the reference arm prints only on rank 0."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    out[rank] = (t, bench.job_value(10, t, world))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.5, 8.0)


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.job_value(5, 2.0, 1) == 2.5


def test_reference_arm_silent_off_rank0(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 3, 2
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
