"""The multi-rank bench path on CPU: two gloo ranks on 127.0.0.1. The
whole-job rate divides the units of all ranks by the slowest rank's time;
the reference arm does its work on rank 0 only."""
import argparse
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    rate = bench.whole_job_rate(1000.0, 1.0 + rank, ws)     # rank r took 1 + r seconds
    slowest = bench.max_over_ranks(3.0 - rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, rate, slowest))


def test_whole_job_rate_uses_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # 2 ranks x 1000 units over the slowest rank's 2 s
    assert [o[1] for o in out] == [1000.0, 1000.0]
    assert [o[2] for o in out] == [3.0, 3.0]


def test_single_process_rate_needs_no_process_group():
    import bench
    assert bench.whole_job_rate(500.0, 2.0, 1) == 250.0
    assert bench.max_over_ranks(1.5) == 1.5


def test_reference_arm_does_no_work_off_rank_0(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    called = []
    monkeypatch.setattr(bench, "oracle_rate", lambda *a, **k: called.append(a))
    args = argparse.Namespace(gpus=2, steps=5, warmup=3, precision="f32_kahan")
    assert bench.run_reference(args) == 0
    assert called == [] and capsys.readouterr().out == ""


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
