"""The benchmark's multi-GPU path is independent replicas (one per rank, no
data-path collective): whole-job throughput = units summed over ranks /
slowest rank's time.  Checked with world_size 2 gloo ranks on CPU; and the
reference arm prints only on rank 0."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = [2.0, 3.0][rank]
    units = [100.0, 140.0][rank]
    value, t_max, total = bench.whole_job_rate(t_local, units)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, value, t_max, total))


def test_whole_job_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t_max, total in out:
        assert t_max == 3.0 and total == 240.0
        assert value == pytest.approx(80.0)


def test_whole_job_rate_single_process():
    import bench
    assert bench.whole_job_rate(2.0, 10.0) == (5.0, 2.0, 10.0)


def test_reference_arm_only_rank0_runs(capsys):
    import argparse
    import bench
    args = argparse.Namespace(steps=1, warmup=0)
    assert bench.run_reference(args, 2, 1) == 0
    assert capsys.readouterr().out == ""
