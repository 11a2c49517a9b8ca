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


def test_reference_arm_json_line(tmp_path):
    # the reference arm (the oracle on the host cores) prints one JSON line
    # with the contract's keys, on a small instance of the bench's workload
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, BANG_WORKLOAD_CACHE=str(tmp_path), RANK="0", WORLD_SIZE="1")
    # configuration 2's small instance: its index comes from the host
    # generator, so the arm runs without a GPU (the large configurations build
    # theirs on the GPU)
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--config", "2", "--n", "20000", "--nq", "200", "--ncomp", "8", "--L", "64",
                          "--cpu-sample", "100", "--steps", "1", "--warmup", "3"],
                         cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "queries/s"
    assert line["metric"].startswith("queries/s at recall@10") and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["L"] == 64
