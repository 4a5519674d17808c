"""Batched beams through the C ABI (`sps_batch_*`): one CUDA-graph launch must
give every beam exactly what its own sps_search gives, launch after launch,
with beams of different shapes and kernel configurations on concurrent
branches; the oracle checks one beam outright."""
import numpy as np
import pytest

import oracle
from paper_1811_04165_gb300 import synth

pytestmark = pytest.mark.gpu


def _beams():
    return synth.batch_beams(6, seed=9, n_t=2000, channels=(96, 48), dm_trials=(64, 256), dm_steps=(0.5, 2.0),
                             max_widths=4)


def _setup(lib, wls):
    import torch
    plans = [lib.Plan.from_workload(wl) for wl in wls]
    xs = []
    for p, wl in zip(plans, wls):
        x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, p.input_samples, wl.seed, wl.pulses,
                             pitch=p.pitch)
        xs.append(torch.from_numpy(x).cuda())
    return plans, xs


def _alone(plans, xs):
    import torch
    ref = []
    for p, x in zip(plans, xs):
        o = p.search(x)
        torch.cuda.synchronize()
        ref.append({k: v.clone() for k, v in o.items()})
    return ref


def _mixed_beams(lib):
    """Beams of several shapes on several kernels: two pre-summed configurations
    shared by beams of different channel counts, DM counts and lengths (fine DM
    grids keep the pre-summed tables small on these wide channels), one on
    pairs, and beams on the single-channel kernel."""
    specs = [  # channels, DM trials, DM step, samples, brute-force configuration (None: single channels)
        (96, 96, 0.10, 2000, (4, 16, 8, 1, 8, 2)), (64, 160, 0.08, 1777, (4, 16, 8, 1, 8, 2)),
        (96, 64, 0.12, 1531, (2, 16, 4, 2, 8, 2)), (64, 40, 0.10, 2000, (2, 16, 4, 2, 8, 2)),
        (96, 72, 0.10, 1900, (4, 16, 8, 1, 8, 1)), (96, 200, 1.00, 2000, None), (48, 64, 2.00, 1200, None)]
    wls, cfgs = [], []
    for b, (ch, n_dm, step, n_t, cfg) in enumerate(specs):
        dms = synth.dm_grid(n_dm, step)
        wls.append(synth.Workload(f"mix{b}", ch, 1250.0, 1550.0, 81.92e-6, n_t, dms,
                                  np.array([1, 2, 4, 8][: 1 + b % 4], np.int32), seed=60 + b,
                                  pulses=[synth.Pulse(float(dms[n_dm // 2]), 2.0, 30.0, n_t / 3.0)]))
        cfgs.append(cfg)
    plans, xs = _setup(lib, wls)
    for p, cfg in zip(plans, cfgs):
        c = p.config
        c.brute = lib.DedispConfig(*cfg) if cfg else lib.DedispConfig(4, 16, 8, 1, 16, 0)
        p.config = c
    return wls, plans, xs


@pytest.mark.parametrize("branches", [1, 3, 8])
def test_batch_matches_each_beam_alone(lib, branches):
    import torch
    wls, plans, xs = _mixed_beams(lib)
    ref = _alone(plans, xs)
    batch = lib.Batch(plans, xs, branches=branches)
    # the pre-summed beams share their pass: one launch per kernel configuration
    # (and occupancy class, which may split one)
    keys = {p.config.brute.as_tuple() for p in plans if p.config.brute.presum}
    assert len(keys) == 3 and 3 <= batch.list_launches <= 5
    for _ in range(2):  # a replay finds the previous launch's contents everywhere
        for o in batch.outs:
            o["D"].fill_(-1)
            o["snr"].fill_(-1.0)
        batch.launch()
        torch.cuda.synchronize()
        for b, (o, r) in enumerate(zip(batch.outs, ref)):
            for k in ("D", "peak_t", "peak_val", "best"):
                assert torch.equal(o[k], r[k]), (b, k)
            assert torch.equal(o["snr"], r["snr"]), b  # same kernels, same arithmetic
    for p in plans:
        assert p.status() == 0


def test_batch_mixes_smoothing_modes_and_zapping(lib):
    """A decimating, RFI-zapped beam in the same graph as plain ones."""
    import torch
    wls = _beams()[:3]
    b = wls[1]
    rng = np.random.Generator(np.random.PCG64(4))
    b.zap = (rng.random(b.channels) < 0.25).astype(np.uint8)
    b.smoothing = lib.SMOOTH_DECIMATE
    b.widths = np.array([1, 3, 16], np.int32)
    plans, xs = _setup(lib, wls)
    ref = _alone(plans, xs)
    batch = lib.Batch(plans, xs, branches=3)
    batch.launch()
    torch.cuda.synchronize()
    for o, r in zip(batch.outs, ref):
        for k in ("D", "snr", "peak_t", "peak_val", "best"):
            assert torch.equal(o[k], r[k]), k
    x = xs[1].cpu().numpy()
    want = oracle.dedisperse(oracle.zap_channels(x, b.zap),
                             oracle.delay_table(b.f_lo, b.f_hi, b.channels, b.t_samp, b.dms), b.n_t)
    assert np.array_equal(batch.outs[1]["D"].cpu().numpy(), want)
    s, pt, pv = oracle.snr_decimated(want, b.widths)
    assert np.allclose(batch.outs[1]["snr"].cpu().numpy(), s, rtol=1e-5, atol=1e-9)
    assert np.array_equal(batch.outs[1]["peak_t"].cpu().numpy(), pt)


@pytest.mark.parametrize("b", [1, 2, 5])
def test_batch_beam_against_the_oracle(lib, b):
    """Beams of the two shared pre-summed passes and an unbatched beam, each
    against the oracle outright."""
    import torch
    wls, plans, xs = _mixed_beams(lib)
    batch = lib.Batch(plans, xs, branches=2)
    batch.launch()
    torch.cuda.synchronize()
    wl, x = wls[b], xs[b].cpu().numpy()
    D = batch.outs[b]["D"].cpu().numpy()
    want = oracle.dedisperse(x, oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms), wl.n_t)
    assert np.array_equal(D, want)
    s, pt, pv = oracle.snr(want, wl.widths)
    got = batch.outs[b]["snr"].cpu().numpy()
    assert np.allclose(got, s, rtol=1e-5, atol=1e-9)
    assert np.array_equal(batch.outs[b]["peak_t"].cpu().numpy(), pt)
    assert np.array_equal(batch.outs[b]["peak_val"].cpu().numpy(), pv)
    oi, ow = oracle.detect(s)
    assert batch.outs[b]["best"].cpu().numpy()[:2].tolist() == [oi, ow]


def test_batch_refuses_a_reconfigured_plan(lib):
    wls = _beams()[:2]
    plans, xs = _setup(lib, wls)
    batch = lib.Batch(plans, xs, branches=2)
    c = plans[0].config
    c.snr.threads = 128 if c.snr.threads != 128 else 256
    plans[0].config = c
    with pytest.raises(lib.SpsError) as e:
        batch.launch()
    assert e.value.status == 1 and "reconfigured" in str(e.value)
