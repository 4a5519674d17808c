"""Real-time serving through the C ABI (`sps_server_*`): streamed batches with
device-resident overlap tails must give exactly what an offline search of the
same overlap-save window gives, and what the oracle gives on that window;
batches are admitted by the HBM budget as memory frees up; every submitted
tag is reported once, with its status."""
import numpy as np
import pytest

import oracle

from paper_1811_04165_gb300 import synth

pytestmark = pytest.mark.gpu


def _beams(n=2):
    return synth.batch_beams(n, seed=12, n_t=1500, channels=(64, 48), dm_trials=(64, 128), dm_steps=(1.0, 2.0),
                             max_widths=3)


def _stream(wl, n_batches, tail):
    """A continuous synthetic stream of (tail + n_batches * N_t) samples; the
    first `tail` samples stand for the zeros before the first batch."""
    n = tail + n_batches * wl.n_t
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, n, wl.seed, wl.pulses)
    x[:, :tail] = 0
    return x


def _drain(srv, done, timeout=30.0):
    t_end = srv.clock() + timeout
    while srv.pending() and srv.clock() < t_end:
        for c in srv.poll():
            done[c.tag] = c
    assert srv.pending() == 0
    return done


def _batch(stream, p, wl, k):
    tail = p.input_samples - wl.n_t
    return np.ascontiguousarray(stream[:, tail + k * wl.n_t: tail + (k + 1) * wl.n_t])


def _check_window(lib, p, wl, stream, k, snr, best):
    """The batch's results equal an offline search of its overlap-save window
    and the oracle on that window."""
    import torch
    window = stream[:, k * wl.n_t: k * wl.n_t + p.input_samples]
    x = np.zeros((wl.channels, p.pitch), np.uint8)
    x[:, :p.input_samples] = window
    o = p.search(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(snr, o["snr"].cpu().numpy()), k
    assert np.array_equal(best, o["best"].cpu().numpy()), k
    _, so, pto, pvo, (bi, bw) = oracle.search_brute(np.ascontiguousarray(window), wl.f_lo, wl.f_hi, wl.t_samp,
                                                    wl.dms, wl.widths, wl.n_t)
    assert np.all(np.abs(snr - so) <= 1e-5 * np.abs(so) + 1e-9), k
    assert best.tolist() == [bi, bw, int(pto[bw, bi]), int(pvo[bw, bi])], k


@pytest.mark.parametrize("inflight", [1, 3])
def test_streamed_batches_equal_offline_windows(lib, inflight):
    wls = _beams()
    plans = [lib.Plan.from_workload(wl) for wl in wls]
    srv = lib.Server(hbm_budget_bytes=8 << 30, max_inflight=inflight)
    ids = [srv.add_beam(p) for p in plans]
    n_batches = 3
    streams = [_stream(wl, n_batches, p.input_samples - wl.n_t) for p, wl in zip(plans, wls)]
    subs, tag = [], 0
    for k in range(n_batches):
        for b, (p, wl) in enumerate(zip(plans, wls)):
            snr = np.full((p.n_widths, p.n_dms), -1.0)
            best = np.full(4, -1, np.int32)
            srv.submit(ids[b], _batch(streams[b], p, wl, k), snr, best, tag=tag)
            subs.append((tag, b, k, snr, best))
            tag += 1
    done = _drain(srv, {})
    assert sorted(done) == [t for t, *_ in subs]
    assert all(c.status == 0 for c in done.values())
    for t, b, k, snr, best in subs:
        _check_window(lib, plans[b], wls[b], streams[b], k, snr, best)
    # completion times are on the server clock and ordered per beam
    for b in range(len(plans)):
        ts = [done[t].done_s for t, bb, *_ in subs if bb == b]
        assert ts == sorted(ts)
    st = srv.stats()
    assert st["admitted"] == len(subs) and st["failed"] == 0 and st["batch_bytes"] == 0


def _sizes(lib, p):
    """(tail bytes, batch bytes) the server takes for a beam of plan p."""
    srv = lib.Server(hbm_budget_bytes=4 << 30, max_inflight=1)
    b = srv.add_beam(p)
    tail = srv.stats()["resident_bytes"]
    srv.submit(b, np.zeros((p.channels, p.n_samples), np.uint8), tag=0)
    batch = srv.stats()["batch_bytes"]
    _drain(srv, {})
    return tail, batch


def test_batches_wait_for_memory_and_beams_leave(lib):
    """A budget that holds every beam's tail but one batch at a time: the second
    beam's batch waits for memory until the first completes (continuous
    batching by HBM budget), and both equal the oracle.  A beam refused for
    budget is admitted once another beam has been removed and its tail freed."""
    # three beams of one shape (tail t, batch bytes m each): a budget of 2 t + m holds
    # two tails and one batch; a third beam needs its tail and a batch beside them
    wls = [synth.Workload(f"serve-same-{b}", 64, 1250.0, 1550.0, 81.92e-6, 1500, synth.dm_grid(96, 1.0),
                          np.array([1, 2, 4], np.int32), seed=40 + b,
                          pulses=[synth.Pulse(30.0 + 20 * b, 4.0, 40.0, 300.0 + 200 * b)]) for b in range(3)]
    plans = [lib.Plan.from_workload(wl) for wl in wls]
    sizes = [_sizes(lib, p) for p in plans]
    assert len(set(sizes)) == 1
    tail, batch = sizes[0]
    budget = 2 * tail + batch
    srv = lib.Server(hbm_budget_bytes=budget, max_inflight=4)
    ids = [srv.add_beam(p) for p in plans[:2]]
    with pytest.raises(lib.SpsError) as e:  # the third beam's tail and batch do not fit beside them
        srv.add_beam(plans[2])
    assert e.value.status == 2 and "budget" in str(e.value)
    streams = [_stream(wl, 2, p.input_samples - wl.n_t) for p, wl in zip(plans, wls)]
    subs, tag = [], 0
    for k in range(2):
        for b in range(2):
            p, wl = plans[b], wls[b]
            snr, best = np.full((p.n_widths, p.n_dms), -1.0), np.full(4, -1, np.int32)
            srv.submit(ids[b], _batch(streams[b], p, wl, k), snr, best, tag=tag)
            subs.append((tag, b, k, snr, best))
            tag += 1
            assert srv.stats()["inflight"] <= 1
    done = _drain(srv, {})
    assert all(c.status == 0 for c in done.values()) and len(done) == 4
    assert srv.stats()["waits_for_memory"] > 0
    for t, b, k, snr, best in subs:
        _check_window(lib, plans[b], wls[b], streams[b], k, snr, best)
    # beam 0 leaves: its tail returns to the arena and beam 2 now fits
    before = srv.stats()["resident_bytes"]
    srv.remove_beam(ids[0])
    assert srv.stats()["resident_bytes"] == before - sizes[0][0]
    with pytest.raises(lib.SpsError):
        srv.submit(ids[0], _batch(streams[0], plans[0], wls[0], 0), tag=99)  # removed: refused
    b2 = srv.add_beam(plans[2])
    p, wl = plans[2], wls[2]
    snr, best = np.full((p.n_widths, p.n_dms), -1.0), np.full(4, -1, np.int32)
    srv.submit(b2, _batch(streams[2], p, wl, 0), snr, best, tag=100)
    done = _drain(srv, {})
    assert done[100].status == 0
    _check_window(lib, p, wl, streams[2], 0, snr, best)


def test_admission_respects_the_budget(lib):
    wls = _beams()
    plans = [lib.Plan.from_workload(wl) for wl in wls]
    srv = lib.Server(hbm_budget_bytes=1 << 20, max_inflight=2)  # 1 MiB: too small for any beam
    with pytest.raises(lib.SpsError) as e:
        srv.add_beam(plans[0])
    assert e.value.status == 2 and "budget" in str(e.value)
    big = lib.Server(hbm_budget_bytes=8 << 30, max_inflight=2)
    assert [big.add_beam(p) for p in plans] == [0, 1]
    assert big.stats()["used_bytes"] == big.stats()["resident_bytes"] > 0


def test_a_batch_that_fails_at_dispatch_is_reported_by_poll(lib):
    """A plan reconfigured after its beam was added needs a larger block than
    the server sized: its queued batch fails when dispatched.  submit() still
    returns normally (the batch was queued), poll() reports the tag with the
    error, its memory is released, and the next batch runs once the plan is
    back on its configuration."""
    # a fine DM grid keeps the pre-summed kernels' tuples per tile few on 4.7 MHz channels
    wl = synth.Workload("serve-fail", 64, 1250.0, 1550.0, 81.92e-6, 1500, synth.dm_grid(40, 0.1),
                        np.array([1, 4], np.int32), seed=21)
    p = lib.Plan.from_workload(wl)
    cfg = {"single": p.config, "quads": p.config}
    cfg["single"].brute.presum = 0
    cfg["quads"].brute = lib.DedispConfig(4, 16, 8, 1, 8, 2)
    sizes = {}
    for name, c in cfg.items():
        p.config = c
        sizes[name] = _sizes(lib, p)[1]
    lo, hi = sorted(sizes, key=sizes.get)
    assert sizes[lo] < sizes[hi]
    p.config = cfg[lo]
    srv = lib.Server(hbm_budget_bytes=1 << 30, max_inflight=1)
    b = srv.add_beam(p)
    x = np.zeros((wl.channels, wl.n_t), np.uint8)
    srv.submit(b, x, tag=1)           # dispatched at once on a block sized for cfg[lo]
    p.config = cfg[hi]                # now the plan needs more memory per batch
    srv.submit(b, x, tag=2)           # queued behind tag 1: fails at dispatch
    done = _drain(srv, {})
    assert done[1].status == 0 and done[2].status == 1
    assert srv.stats()["failed"] == 1 and srv.stats()["batch_bytes"] == 0
    p.config = cfg[lo]
    srv.submit(b, x, tag=2)           # the reported tag is free again
    done = _drain(srv, {})
    assert done[2].status == 0


def test_submit_refuses_a_tag_in_flight_and_bad_buffers(lib):
    wls = _beams()
    p = lib.Plan.from_workload(wls[0])
    srv = lib.Server(hbm_budget_bytes=8 << 30, max_inflight=2)
    b = srv.add_beam(p)
    x = np.zeros((wls[0].channels, wls[0].n_t), np.uint8)
    snr = np.zeros((p.n_widths, p.n_dms))
    srv.submit(b, x, snr, tag=7)
    with pytest.raises(ValueError):  # tag 7 has not been polled yet: its buffers stay referenced
        srv.submit(b, x, snr, tag=7)
    with pytest.raises(ValueError):
        srv.submit(b, x[:-1], tag=8)  # one channel row short
    with pytest.raises(ValueError):
        srv.submit(b, x, np.zeros((p.n_widths, p.n_dms), np.float32), tag=9)  # 4-byte S/N elements
    with pytest.raises(lib.SpsError):
        srv.submit(b, x[:, :10].copy(), tag=10)  # pitch below N_t: refused by the library
    done = _drain(srv, {})
    assert 7 in done and done[7].status == 0
    srv.submit(b, x, snr, tag=10)  # the refused tag is free again
    _drain(srv, {})
