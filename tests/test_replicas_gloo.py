"""The multi-rank host logic of the benchmark (max over ranks, whole-job throughput) on
world_size-2 gloo process groups on the CPU."""
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
    from paper_2006_02545_gb300.replicas import job_throughput, max_over_ranks
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    ms = 1000.0 + 250.0 * rank           # rank 1 is the slowest
    slowest = max_over_ranks(ms)
    out[rank] = (slowest, job_throughput(35840, 5, world, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    ctx = mp.get_context("spawn")
    world = 2
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    slowest, v = res[0]
    assert slowest == 1250.0
    assert v == pytest.approx(2 * 35840 * 5 / 1.25)


def test_single_process_passthrough():
    from paper_2006_02545_gb300.replicas import max_over_ranks
    assert max_over_ranks(3.5) == 3.5
