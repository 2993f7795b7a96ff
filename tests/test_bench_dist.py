"""Host logic of the multi-process bench (replicas: one process per GPU, no
collective on the data path): rank environment and the max-over-ranks timing
reduction, run as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    ws, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=ws)
    dist.barrier()
    # each replica's own step time; every rank must report the slowest one
    got = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    dist.destroy_process_group()
    out.put((r, ws, local, got))


@pytest.mark.timeout(120)
def test_two_gloo_ranks_report_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [(r, ws, local) for r, ws, local, _ in res] == [(0, 2, 0), (1, 2, 1)]
    assert all(got == 15.0 for *_, got in res)


def test_single_process_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
