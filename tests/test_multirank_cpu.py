"""Host logic of the multi-process (replicas) benchmark path on CPU ranks (gloo)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.job_throughput(10.0 + 5.0 * rank, units_per_rank=1000, steps=4, world=world)
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_job_throughput_takes_the_slowest_rank(world):
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    slow = 10.0 + 5.0 * (world - 1)
    for r in range(world):
        ms, value = out[r]
        assert ms == slow
        assert value == pytest.approx(world * 1000 * 4 / (slow / 1e3))


def test_reference_arm_only_rank0_works(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        taps, warmup, steps = 5, 0, 1
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
