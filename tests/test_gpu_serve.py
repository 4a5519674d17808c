"""Real-time serving through the C ABI (`sps_server_*`): streamed batches with
device-resident overlap tails must give exactly what an offline search of the
same overlap-save window gives, and what the oracle gives on that window;
admission respects the HBM budget."""
import numpy as np
import pytest

import oracle

from paper_1811_04165_gb300 import synth

pytestmark = pytest.mark.gpu


def _beams():
    return synth.batch_beams(2, seed=12, n_t=1500, channels=(64, 48), dm_trials=(64, 128), dm_steps=(1.0, 2.0),
                             max_widths=3)


def _stream(wl, n_batches, tail):
    """A continuous synthetic stream of (tail + n_batches * N_t) samples; the
    first `tail` samples stand for the zeros before the first batch."""
    n = tail + n_batches * wl.n_t
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, n, wl.seed, wl.pulses)
    x[:, :tail] = 0
    return x


@pytest.mark.parametrize("inflight", [1, 3])
def test_streamed_batches_equal_offline_windows(lib, inflight):
    import torch
    wls = _beams()
    plans = [lib.Plan.from_workload(wl) for wl in wls]
    srv = lib.Server(hbm_budget_bytes=8 << 30, max_inflight=inflight)
    ids = [srv.add_beam(p) for p in plans]
    n_batches = 3
    streams, subs = [], []
    for p, wl in zip(plans, wls):
        tail = p.input_samples - wl.n_t
        streams.append(_stream(wl, n_batches, tail))
    tag = 0
    for k in range(n_batches):
        for b, (p, wl) in enumerate(zip(plans, wls)):
            tail = p.input_samples - wl.n_t
            new = np.ascontiguousarray(streams[b][:, tail + k * wl.n_t: tail + (k + 1) * wl.n_t])
            snr = np.full((p.n_widths, p.n_dms), -1.0)
            best = np.full(4, -1, np.int32)
            srv.submit(ids[b], new, snr, best, tag=tag)
            subs.append((tag, b, k, snr, best, new))
            tag += 1
    done = {}
    t_end = srv.clock() + 30.0
    while len(done) < len(subs) and srv.clock() < t_end:
        for t, s in srv.poll():
            done[t] = s
    assert len(done) == len(subs) and srv.pending() == 0
    for t, b, k, snr, best, _ in subs:
        p, wl = plans[b], wls[b]
        tail = p.input_samples - wl.n_t
        window = streams[b][:, k * wl.n_t: k * wl.n_t + p.input_samples]
        x = np.zeros((wl.channels, p.pitch), np.uint8)
        x[:, :p.input_samples] = window
        o = p.search(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(snr, o["snr"].cpu().numpy()), (b, k)
        assert np.array_equal(best, o["best"].cpu().numpy()), (b, k)
        # and what the oracle computes on that window
        _, so, pto, pvo, (bi, bw) = oracle.search_brute(np.ascontiguousarray(window), wl.f_lo, wl.f_hi, wl.t_samp,
                                                        wl.dms, wl.widths, wl.n_t)
        assert np.all(np.abs(snr - so) <= 1e-5 * np.abs(so) + 1e-9), (b, k)
        assert best.tolist() == [bi, bw, int(pto[bw, bi]), int(pvo[bw, bi])], (b, k)
    # completion times are on the server clock and ordered per beam
    for b in range(len(plans)):
        ts = [done[t] for t, bb, *_ in subs if bb == b]
        assert ts == sorted(ts)


def test_admission_respects_the_budget(lib):
    wls = _beams()
    plans = [lib.Plan.from_workload(wl) for wl in wls]
    srv = lib.Server(hbm_budget_bytes=1 << 20, max_inflight=2)  # 1 MiB: too small for any beam
    with pytest.raises(lib.SpsError) as e:
        srv.add_beam(plans[0])
    assert e.value.status == 2 and "budget" in str(e.value)
    big = lib.Server(hbm_budget_bytes=8 << 30, max_inflight=2)
    assert [big.add_beam(p) for p in plans] == [0, 1]


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
    done = {}
    t_end = srv.clock() + 30.0
    while srv.pending() and srv.clock() < t_end:
        done.update(srv.poll())
    assert 7 in done and srv.pending() == 0
    srv.submit(b, x, snr, tag=10)  # the refused tag is free again
    while srv.pending() and srv.clock() < t_end:
        srv.poll()
