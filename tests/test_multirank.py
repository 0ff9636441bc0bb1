"""The replica mode of the benchmark with two gloo ranks on CPU: every rank
learns the slowest rank's time, and the whole-job rate counts all ranks' work."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, size, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=size)
    from paper_2312_14907_gb300 import replicas
    r, s = replicas.world()
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    slowest = replicas.max_over_ranks(local_ms)
    rate = replicas.whole_job_rate(2883, 4, s, slowest)
    q.put((r, s, slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 15.0 for o in out)
    assert all(abs(o[3] - 2883 * 4 * 2 / 0.015) < 1e-6 * o[3] for o in out)


def test_single_process_defaults():
    from paper_2312_14907_gb300 import replicas
    assert replicas.world() == (0, 1)
    assert replicas.max_over_ranks(3.5) == 3.5
    with pytest.raises(ValueError):
        replicas.whole_job_rate(1, 1, 1, 0.0)
