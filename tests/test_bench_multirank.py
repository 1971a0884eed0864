"""The multi-rank path of bench.py on CPU (gloo, world size 2): replicas only, the job time is
the slowest rank's, the job throughput counts every rank's cells, and only rank 0 reports."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = 10.0 + 5.0 * rank
    ms_max = bench.reduce_max(local_ms, ws)
    value = bench.job_throughput(1_000_000, 100, ws, ms_max / 1e3)
    q.put((rank, ms_max, value, bench._dist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value, dist_env in out:
        assert ms_max == 15.0                       # the slowest rank sets the job time
        assert value == pytest.approx(2 * 1_000_000 * 100 / 0.015 / 1e6)
        assert dist_env == (2, rank, rank)


def test_reference_arm_is_rank0_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 10, 3, 2
    bench.bench_reference(A())
    assert capsys.readouterr().out == ""
