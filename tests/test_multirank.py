"""Multi-GPU path of the benchmark on CPU with gloo (world size 2): replicas
of the search report the whole job's throughput over the slowest rank's time,
and the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    value, t = bench.job_throughput(100, 3, 10.0 * (rank + 1), world, dist)
    out.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_report_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t in res:
        assert t == 20.0                                  # the slower rank's time
        assert value == pytest.approx(100 * 2 * 3 / 0.020)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), dict(L=None, cpu_sample=10, warmup=0, steps=1, bloom_log2=16, gpus=2,
                               n=None, nq=None, ncomp=None))()
    assert bench.run_reference(args) == 0                 # returns before loading anything
