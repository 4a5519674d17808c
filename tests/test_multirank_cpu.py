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


def _search_rank(rank, world, port, q):
    """One replica: the rank's own beam (bench.rank_beam), searched by the oracle on
    the CPU over the 32 DM trials around its strongest pulse; then the barrier
    and the max over ranks that the benchmark takes."""
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), SPS_BENCH_BACKEND="gloo")
    import time

    import numpy as np

    import bench
    import oracle
    from paper_1811_04165_gb300 import synth
    r, w = bench.dist_init(world)
    wl = bench.rank_beam(r)
    strongest = max(wl.pulses, key=lambda p: p.amp * np.sqrt(p.width))
    i0 = int(np.clip(np.searchsorted(wl.dms, strongest.dm) - 16, 0, wl.dms.size - 32))
    dms = wl.dms[i0:i0 + 32]
    t = time.perf_counter()
    delays = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, dms)
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_t + int(delays.max()), wl.seed, wl.pulses)
    s, pt, _ = oracle.snr(oracle.dedisperse(x, delays, wl.n_t), wl.widths)
    bi, bw = oracle.detect(s)
    step_s = time.perf_counter() - t
    bench.barrier(w)
    slowest = bench.max_over_ranks(step_s, w)
    q.put((r, bench.local_device_index(), wl.seed, strongest.dm, float(dms[bi]), int(pt[bw, bi]), step_s, slowest))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_search_their_own_beams():
    """Each rank drives the GPU of its LOCAL_RANK and searches its own beam (seed
    2 + rank, its own pulses); the detections differ between ranks, each finds its
    own strongest pulse's DM, and both ranks report the slower rank's time."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_search_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [0, 1]           # device = LOCAL_RANK
    assert [o[2] for o in out] == [2, 3]           # beam seed = 2 + rank
    for _, _, _, dm_true, dm_found, _, _, _ in out:
        assert abs(dm_found - dm_true) <= 1.0      # within a few 0.2 trials of the injected DM
    assert out[0][3] != out[1][3] and (out[0][4], out[0][5]) != (out[1][4], out[1][5])
    slowest = max(o[6] for o in out)
    assert all(o[7] == pytest.approx(slowest) for o in out)
