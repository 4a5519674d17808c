"""The benchmark's multi-GPU path is replicas only: each rank searches its own
beam, and the only collectives are the timing barrier and the max over ranks.
This checks that host logic with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), SPS_BENCH_BACKEND="gloo")
    import bench
    r, w = bench.dist_init(world)
    bench.barrier(w)
    step_s = [0.010, 0.025][r]  # the second rank is slower
    slowest = bench.max_over_ranks(step_s, w)
    samples = 2048 * 12500
    value = w * samples * 4 / (4 * slowest)  # all ranks' samples over the slowest rank's time
    q.put((r, w, slowest, value))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2, 2]
    assert all(o[2] == pytest.approx(0.025) for o in out)
    assert all(o[3] == pytest.approx(2 * 2048 * 12500 / 0.025) for o in out)
