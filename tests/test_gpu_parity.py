"""CUDA path against the CPU oracle, element by element, through the C ABI.

Integer results (D, Y, B, peak_t, peak_val, the detection) must be bit-exact;
S/N within relative 1e-5 of the FP64 oracle (absolute 1e-9 near zero).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1811_04165_gb300 import synth
from tests import oracle_rows

pytestmark = pytest.mark.gpu

SNR_RTOL = 1e-5
SNR_ATOL = 1e-9


def _torch():
    import torch
    return torch


def _plan(lib, wl, mode=None, **kw):
    return lib.Plan.from_workload(wl, mode=mode) if not kw else lib.Plan(**kw)


def _x_for(plan, wl, seed=None, pulses=None):
    n_in = plan.input_samples
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, n_in, wl.seed if seed is None else seed,
                         wl.pulses if pulses is None else pulses, pitch=plan.pitch)
    return x


def _to_np(t):
    torch = _torch()
    if t.dtype == torch.uint16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def _check_snr(got_snr, got_pt, got_pv, want_snr, want_pt, want_pv):
    assert np.array_equal(got_pt, want_pt)
    assert np.array_equal(got_pv, want_pv)
    err = np.abs(got_snr - want_snr)
    assert np.all(err <= SNR_RTOL * np.abs(want_snr) + SNR_ATOL), float(err.max())


# ----------------------------------------------------------------------------- tables
def test_plan_tables_equal_oracle(lib):
    wl = synth.apertif_beam()
    p = lib.Plan.from_workload(wl)
    want = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    assert np.array_equal(p.delay_table(), want)
    assert p.input_samples == wl.n_t + want.max()
    ws = synth.apertif_beam(subband=True)
    ps = lib.Plan.from_workload(ws)
    d1, d2 = oracle.subband_tables(ws.f_lo, ws.f_hi, ws.channels, ws.t_samp, ws.n_subbands, ws.coarse_dms,
                                   ws.dms)
    g1, g2 = ps.subband_tables()
    assert np.array_equal(g1, d1) and np.array_equal(g2, d2)
    n_1, n_in = oracle.subband_lengths(ws.n_t, d1, d2)
    assert (ps.step1_samples, ps.input_samples) == (n_1, n_in)


# ----------------------------------------------------------------------------- brute force
def test_tiny_brute_whole_path(lib):
    torch = _torch()
    wl = synth.tiny_brute()
    p = lib.Plan.from_workload(wl)
    x = _x_for(p, wl)
    out = p.search(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    D, s, pt, pv, (bi, bw) = oracle.search_brute(x[:, :p.input_samples], wl.f_lo, wl.f_hi, wl.t_samp,
                                                  wl.dms, wl.widths, wl.n_t)
    assert np.array_equal(_to_np(out["D"]), D)
    _check_snr(_to_np(out["snr"]), _to_np(out["peak_t"]), _to_np(out["peak_val"]), s, pt, pv)
    assert _to_np(out["best"]).tolist() == [bi, bw, int(pt[bw, bi]), int(pv[bw, bi])]
    assert (bi, int(wl.widths[bw])) == (25, 4)
    assert p.status() == 0


CONFIGS = [  # (dms_per_thread, samples_per_thread, warps_dm, warps_time, chunk)
    (1, 4, 1, 1, 2), (1, 8, 2, 2, 6), (2, 4, 4, 2, 16), (2, 16, 2, 1, 32), (4, 4, 2, 2, 10),
    (4, 8, 4, 2, 16), (4, 16, 8, 1, 16), (8, 4, 2, 4, 8), (8, 8, 1, 8, 6), (1, 32, 16, 1, 4),
    (2, 32, 4, 1, 8),
]


PRESUM_CONFIGS = [  # (dms_per_thread, samples_per_thread, warps_dm, warps_time, chunk, presum)
    (1, 4, 1, 1, 2, 1), (1, 8, 2, 2, 6, 1), (2, 4, 4, 2, 16, 1), (2, 32, 2, 1, 8, 1), (4, 8, 2, 2, 10, 1),
    (4, 16, 8, 1, 8, 1), (8, 4, 2, 4, 8, 1), (8, 8, 4, 2, 4, 1), (1, 32, 16, 1, 4, 1), (4, 8, 4, 4, 6, 1),
    (1, 4, 1, 1, 2, 2), (1, 8, 2, 2, 8, 2), (2, 4, 4, 2, 16, 2), (2, 32, 2, 1, 8, 2), (4, 8, 2, 2, 12, 2),
    (4, 16, 8, 1, 4, 2), (8, 4, 2, 4, 8, 2), (8, 8, 4, 2, 4, 2), (1, 32, 16, 1, 4, 2), (4, 8, 4, 4, 6, 2),
]


@pytest.mark.parametrize("cfg", CONFIGS + PRESUM_CONFIGS)
def test_brute_configs_ragged(lib, cfg):
    # 37 channels (odd, not a multiple of any chunk), 29 DMs, 1003 samples: ragged everywhere.
    # The pre-summed kernels get a finer DM grid: with 5.4 MHz channels a coarse
    # grid spreads the relative delays too far for one tile's staging.
    torch = _torch()
    dms = synth.dm_grid(29, 0.31 if len(cfg) > 5 and cfg[5] else 3.1)
    p = lib.Plan(37, 1300.0, 1500.0, 65.536e-6, 1003, dms, [1, 3, 8, 50])
    c = p.config
    c.brute = lib.DedispConfig(*cfg)
    p.config = c
    x = synth.filterbank(37, 1300.0, 1500.0, 65.536e-6, p.input_samples, 99, pitch=p.pitch + 32)
    xd = torch.from_numpy(x).cuda()
    D = torch.full((29, 1003), -7, dtype=torch.int32, device="cuda")
    lib.sps_dedisperse(p, xd, D)
    torch.cuda.synchronize()
    want = oracle.dedisperse(x, oracle.delay_table(1300.0, 1500.0, 37, 65.536e-6, dms), 1003)
    assert np.array_equal(_to_np(D), want)


@pytest.mark.parametrize("fill", [0x00, 0xFF, 0x5A])
@pytest.mark.parametrize("presum", [1, 2])
def test_presum_ignores_stale_workspace(lib, fill, presum):
    """The pre-pass writes each series only over the samples its trials read
    for valid outputs; whatever the workspace held elsewhere must not reach an
    output (odd N_t: the last valid sample shares a 32-bit word with one that
    is not)."""
    torch = _torch()
    dms = synth.dm_grid(29, 0.31)
    p = lib.Plan(40, 1300.0, 1500.0, 65.536e-6, 1003, dms, [1, 3])
    c = p.config
    c.brute = lib.DedispConfig(4, 8, 2, 2, 12, presum)
    p.config = c
    x = synth.filterbank(40, 1300.0, 1500.0, 65.536e-6, p.input_samples, 13, pitch=p.pitch)
    ws = torch.full((p.workspace_bytes,), fill, dtype=torch.uint8, device="cuda")
    D = torch.full((29, 1003), -7, dtype=torch.int32, device="cuda")
    lib.sps_dedisperse(p, torch.from_numpy(x).cuda(), D, workspace=ws)
    torch.cuda.synchronize()
    want = oracle.dedisperse(x, oracle.delay_table(1300.0, 1500.0, 40, 65.536e-6, dms), 1003)
    assert np.array_equal(_to_np(D), want)


@pytest.mark.parametrize("C", [38, 39, 40])
@pytest.mark.parametrize("cfg", [(1, 4, 1, 1, 2, 2), (4, 8, 2, 2, 12, 2)])
def test_quads_short_last_unit(lib, C, cfg):
    """Channel counts ending in a unit of 2, 3 or 4 channels."""
    torch = _torch()
    dms = synth.dm_grid(29, 0.31)
    p = lib.Plan(C, 1300.0, 1500.0, 65.536e-6, 1003, dms, [1, 3])
    c = p.config
    c.brute = lib.DedispConfig(*cfg)
    p.config = c
    x = synth.filterbank(C, 1300.0, 1500.0, 65.536e-6, p.input_samples, 5 + C, pitch=p.pitch)
    D = torch.full((29, 1003), -7, dtype=torch.int32, device="cuda")
    lib.sps_dedisperse(p, torch.from_numpy(x).cuda(), D)
    torch.cuda.synchronize()
    want = oracle.dedisperse(x, oracle.delay_table(1300.0, 1500.0, C, 65.536e-6, dms), 1003)
    assert np.array_equal(_to_np(D), want)


def test_brute_saturated_and_edges(lib):
    torch = _torch()
    # all-255 input: every sum is 255 * C, exercising the 16-bit lanes at their limit
    dms = synth.dm_grid(16, 5.0)
    C = 600  # more than two 16-bit folds
    p = lib.Plan(C, 1250.0, 1550.0, 81.92e-6, 500, dms, [1, 7])
    x = np.full((C, p.pitch), 255, np.uint8)
    D = torch.empty((16, 500), dtype=torch.int32, device="cuda")
    lib.sps_dedisperse(p, torch.from_numpy(x).cuda(), D)
    torch.cuda.synchronize()
    assert np.all(_to_np(D) == 255 * C)
    c = p.config
    c.brute = lib.DedispConfig(4, 16, 8, 1, 4, 1)  # pair sums at their limit: 128 pairs of 510 per 16-bit lane
    p.config = c
    D.fill_(0)
    lib.sps_dedisperse(p, torch.from_numpy(x).cuda(), D)
    torch.cuda.synchronize()
    assert np.all(_to_np(D) == 255 * C)
    # quad sums at their limit: 64 quads of 1020 per 16-bit lane, 4 quads per chunk
    # (a finer DM grid keeps one tile's quad tuples within shared memory)
    pq = lib.Plan(C, 1250.0, 1550.0, 81.92e-6, 500, synth.dm_grid(16, 0.5), [1, 7])
    c = pq.config
    c.brute = lib.DedispConfig(4, 16, 8, 1, 16, 2)
    pq.config = c
    D.fill_(0)
    lib.sps_dedisperse(pq, torch.from_numpy(x).cuda(), D)
    torch.cuda.synchronize()
    assert np.all(_to_np(D) == 255 * C)
    # single channels at their limit: 256 channels of 255 per fold (chunks of 16 fold at exactly 256, chunks
    # of 6 at 252), every byte of a word at 255, so the whole-word sums wrap and the even lanes come back only
    # through the odd-lane sums
    c = p.config
    for cfg in [(4, 16, 8, 1, 16, 0), (4, 8, 2, 2, 6, 0)]:
        c.brute = lib.DedispConfig(*cfg)
        p.config = c
        D.fill_(0)
        lib.sps_dedisperse(p, torch.from_numpy(x).cuda(), D)
        torch.cuda.synchronize()
        assert np.all(_to_np(D) == 255 * C), cfg
    # a single channel, single DM, single sample
    p1 = lib.Plan(1, 1250.0, 1550.0, 81.92e-6, 1, [0.0], [1])
    x1 = np.zeros((1, 16), np.uint8)
    x1[0, 0] = 201
    D1 = torch.empty((1, 1), dtype=torch.int32, device="cuda")
    lib.sps_dedisperse(p1, torch.from_numpy(x1).cuda(), D1)
    torch.cuda.synchronize()
    assert _to_np(D1).tolist() == [[201]]


@pytest.mark.parametrize("cfg", [(4, 16, 8, 1, 16, 0), (4, 16, 8, 1, 8, 1), (4, 16, 8, 1, 16, 2)])
def test_brute_4096_channels(lib, cfg):
    """A LOFAR-sized band of 4096 channels: sixteen 16-bit folds for single
    channels, 32 for pairs, 16 for quads per row, ragged time tail."""
    torch = _torch()
    dms = synth.dm_grid(24, 0.25)
    p = lib.Plan(4096, 1100.0, 1500.0, 65.536e-6, 601, dms, [1, 4, 16])
    c = p.config
    c.brute = lib.DedispConfig(*cfg)
    p.config = c
    x = synth.filterbank(4096, 1100.0, 1500.0, 65.536e-6, p.input_samples, 41, pitch=p.pitch)
    out = p.search(torch.from_numpy(x).cuda(), workspace=p.workspace())
    torch.cuda.synchronize()
    want = oracle.dedisperse(x, oracle.delay_table(1100.0, 1500.0, 4096, 65.536e-6, dms), 601)
    assert np.array_equal(_to_np(out["D"]), want)
    s, pt, pv = oracle.snr(want, [1, 4, 16])
    _check_snr(_to_np(out["snr"]), _to_np(out["peak_t"]), _to_np(out["peak_val"]), s, pt, pv)


def test_quads_with_long_relative_delays(lib):
    """Quads whose channels lie up to 33346 samples apart (100-200 MHz, 10 us
    samples): too far to stage a unit's rows in shared memory, so the
    pre-pass reads the rows from global memory."""
    torch = _torch()
    dms = np.array([0.0, 1.0, 2.0])
    p = lib.Plan(8, 100.0, 200.0, 1e-5, 100, dms, [1, 5])
    c = p.config
    c.brute = lib.DedispConfig(1, 4, 1, 1, 4, 2)  # one trial per tile: no delay spread inside a tile
    p.config = c
    x = synth.filterbank(8, 100.0, 200.0, 1e-5, p.input_samples, 77, pitch=p.pitch)
    D = torch.full((3, 100), -7, dtype=torch.int32, device="cuda")
    lib.sps_dedisperse(p, torch.from_numpy(x).cuda(), D, workspace=p.workspace())
    torch.cuda.synchronize()
    d = oracle.delay_table(100.0, 200.0, 8, 1e-5, dms)
    assert int(d[2, 0] - d[2, 3]) == 33346
    assert np.array_equal(_to_np(D), oracle.dedisperse(x, d, 100))


@pytest.fixture(scope="module")
def apertif_brute_oracle():
    """The beam's input and the oracle's whole-table results: D, S/N, peaks and
    the detection over all 2048 DM trials (rows split over the host cores)."""
    wl = synth.apertif_beam()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    n_in = wl.n_t + int(d.max())
    pitch = (n_in + 15) // 16 * 16
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, n_in, wl.seed, wl.pulses, pitch=pitch)
    D = oracle_rows.dedisperse(x, d, wl.n_t)
    s, pt, pv = oracle_rows.snr(D, wl.widths)
    return wl, x, D, s, pt, pv, oracle.detect(s)


@pytest.mark.parametrize("presum", [0, 1, 2])
def test_apertif_brute_full_tables(lib, apertif_brute_oracle, presum):
    """The full Apertif-shaped beam in the launch configurations the benchmark
    times: every row of D, every (width, DM) entry of the S/N, peak_t and
    peak_val tables, and the detection against the oracle's over the whole table."""
    torch = _torch()
    wl, x, Do, s, pt, pv, (bi, bw) = apertif_brute_oracle
    p = lib.Plan.from_workload(wl)
    assert p.pitch == x.shape[1]
    c = p.config
    c.brute.presum = presum
    p.config = c
    out = p.search(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(_to_np(out["D"]), Do)
    _check_snr(_to_np(out["snr"]), _to_np(out["peak_t"]), _to_np(out["peak_val"]), s, pt, pv)
    assert _to_np(out["best"]).tolist() == [bi, bw, int(pt[bw, bi]), int(pv[bw, bi])]
    # the detection is the strongest injected pulse
    strongest = max(wl.pulses, key=lambda q: q.amp * np.sqrt(q.width))
    assert abs(wl.dms[bi] - strongest.dm) <= 0.2 + 1e-9
    assert abs(int(pt[bw, bi]) - strongest.t0) <= strongest.width
    assert p.status() == 0


# ----------------------------------------------------------------------------- subband
def _small_subband(S, n_dms=48, n_coarse=6, C=96, n_t=777):
    dms = synth.dm_grid(n_dms, 1.7)
    return synth.Workload("small-subband", C, 1250.0, 1550.0, 81.92e-6, n_t, dms,
                          np.array([1, 2, 5], np.int32), seed=20 + S, n_subbands=S,
                          coarse_dms=dms[::n_dms // n_coarse].copy())


@pytest.mark.parametrize("S", [1, 2, 8, 32, 96])
def test_subband_small_exact(lib, S):
    torch = _torch()
    wl = _small_subband(S)
    p = lib.Plan.from_workload(wl)
    x = _x_for(p, wl, pulses=[synth.Pulse(40.0, 3.0, 30.0, 300.0)])
    xd = torch.from_numpy(x).cuda()
    Y = torch.empty(p.y_shape, dtype=torch.uint16, device="cuda")
    lib.sps_subband_step1(p, xd, Y)
    D = torch.empty((wl.dms.size, wl.n_t), dtype=torch.int32, device="cuda")
    lib.sps_subband_step2(p, Y, D)
    D2 = torch.empty_like(D)
    lib.sps_dedisperse(p, xd, D2, workspace=p.workspace())
    torch.cuda.synchronize()
    d1, d2 = oracle.subband_tables(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, S, wl.coarse_dms, wl.dms)
    n_1, _ = oracle.subband_lengths(wl.n_t, d1, d2)
    Yo = oracle.subband_step1(x, d1, S, n_1)
    k = oracle.coarse_index(wl.dms.size, wl.coarse_dms.size)
    Do = oracle.subband_step2(Yo, d2, k, wl.n_t)
    assert np.array_equal(_to_np(Y)[:, :, :n_1].astype(np.int32), Yo)
    assert np.array_equal(_to_np(D), Do)
    assert np.array_equal(_to_np(D2), Do)
    # the plan's composed table reproduces the same sums in one pass
    assert np.array_equal(oracle.dedisperse(x, p.delay_table(), wl.n_t), Do)


@pytest.mark.parametrize("C,S", [(63, 3), (60, 5), (60, 6)])
def test_subband_step1_blocks_walking_several_subbands(lib, C, S):
    """Step-one blocks walk several subbands in turn when the grid has tiles to
    spare (here 16 coarse DMs x about 37 time tiles of 128 samples, so up to four
    subbands per block); subband counts that leave the last block fewer, and a
    group of 21 channels whose last chunk holds one, give Y and D equal to the
    oracle's (step two on single-trial tiles of 128 samples)."""
    torch = _torch()
    n_coarse, per = 16, 4
    dms = synth.dm_grid(n_coarse * per, 1.3)
    wl = synth.Workload("walk-subbands", C, 1250.0, 1550.0, 81.92e-6, 4100, dms, np.array([1, 2, 4], np.int32),
                        seed=40 + S, n_subbands=S, coarse_dms=dms[::per].copy())
    p = lib.Plan.from_workload(wl)
    c = p.config
    c.step1 = lib.DedispConfig(1, 4, 1, 1, 4)
    c.step2 = lib.DedispConfig(1, 4, 1, 1, 2)
    p.config = c
    x = _x_for(p, wl, pulses=[synth.Pulse(60.0, 2.0, 25.0, 900.0)])
    xd = torch.from_numpy(x).cuda()
    Y = torch.empty(p.y_shape, dtype=torch.uint16, device="cuda")
    lib.sps_subband_step1(p, xd, Y)
    D = torch.empty((wl.dms.size, wl.n_t), dtype=torch.int32, device="cuda")
    lib.sps_subband_step2(p, Y, D)
    torch.cuda.synchronize()
    d1, d2 = oracle.subband_tables(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, S, wl.coarse_dms, wl.dms)
    n_1, _ = oracle.subband_lengths(wl.n_t, d1, d2)
    Yo = oracle.subband_step1(x, d1, S, n_1)
    assert np.array_equal(_to_np(Y)[:, :, :n_1].astype(np.int32), Yo)
    Do = oracle.subband_step2(Yo, d2, oracle.coarse_index(wl.dms.size, wl.coarse_dms.size), wl.n_t)
    assert np.array_equal(_to_np(D), Do)


@pytest.mark.parametrize("cfg1,cfg2", [
    # pre-summed kernels on 4.7 MHz channels: relative delays vary widely, so small chunks
    ((1, 4, 1, 1, 2, 1), (1, 4, 1, 1, 1)),
    ((4, 16, 8, 1, 2, 1), (4, 16, 8, 1, 8)),
    ((2, 8, 2, 2, 2, 1), (8, 4, 4, 2, 5)),
    ((1, 4, 1, 1, 4, 2), (1, 4, 1, 1, 1)),
    ((4, 16, 8, 1, 4, 2), (4, 16, 8, 1, 8)),
    ((2, 8, 2, 2, 8, 2), (8, 4, 4, 2, 5)),
    ((1, 4, 1, 1, 2), (1, 4, 1, 1, 1)),
    ((2, 8, 2, 2, 6), (2, 8, 2, 2, 3)),
    ((4, 16, 8, 1, 16), (8, 4, 4, 2, 5)),
    ((8, 8, 1, 4, 8), (4, 16, 2, 4, 4)),
])
def test_subband_configs(lib, cfg1, cfg2):
    torch = _torch()
    wl = _small_subband(8, n_dms=40, n_coarse=5, C=64, n_t=1001)
    p = lib.Plan.from_workload(wl)
    c = p.config
    c.step1 = lib.DedispConfig(*cfg1)
    c.step2 = lib.DedispConfig(*cfg2)
    p.config = c
    x = _x_for(p, wl)
    D = torch.empty((wl.dms.size, wl.n_t), dtype=torch.int32, device="cuda")
    lib.sps_dedisperse(p, torch.from_numpy(x).cuda(), D, workspace=p.workspace())
    torch.cuda.synchronize()
    assert np.array_equal(_to_np(D), oracle.dedisperse(x, p.delay_table(), wl.n_t))
    d1, d2 = oracle.subband_tables(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, 8, wl.coarse_dms, wl.dms)
    n_1, _ = oracle.subband_lengths(wl.n_t, d1, d2)
    Do = oracle.subband_step2(oracle.subband_step1(x, d1, 8, n_1), d2,
                              oracle.coarse_index(wl.dms.size, wl.coarse_dms.size), wl.n_t)
    assert np.array_equal(_to_np(D), Do)


@pytest.mark.parametrize("presum", [1, 2])
def test_subband_presum_ignores_stale_workspace(lib, presum):
    """Step one over pre-summed series (range-limited, N_1 outputs per row)
    with a workspace full of 0xFF bytes."""
    torch = _torch()
    wl = _small_subband(8, n_dms=40, n_coarse=5, C=64, n_t=1001)
    p = lib.Plan.from_workload(wl)
    c = p.config
    c.step1 = lib.DedispConfig(1, 4, 1, 1, 2, presum)
    p.config = c
    x = _x_for(p, wl)
    ws = torch.full((p.workspace_bytes,), 0xFF, dtype=torch.uint8, device="cuda")
    D = torch.full((wl.dms.size, wl.n_t), -7, dtype=torch.int32, device="cuda")
    lib.sps_dedisperse(p, torch.from_numpy(x).cuda(), D, workspace=ws)
    torch.cuda.synchronize()
    d1, d2 = oracle.subband_tables(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, 8, wl.coarse_dms, wl.dms)
    n_1, _ = oracle.subband_lengths(wl.n_t, d1, d2)
    Do = oracle.subband_step2(oracle.subband_step1(x, d1, 8, n_1), d2,
                              oracle.coarse_index(wl.dms.size, wl.coarse_dms.size), wl.n_t)
    assert np.array_equal(_to_np(D), Do)


@pytest.fixture(scope="module")
def apertif_subband_oracle():
    """The beam's two-step path in the oracle: Y over all 64 coarse DMs, D over
    all 2048 trials, the S/N tables and the detection."""
    wl = synth.apertif_beam(subband=True)
    d1, d2 = oracle.subband_tables(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.n_subbands, wl.coarse_dms,
                                   wl.dms)
    n_1, n_in = oracle.subband_lengths(wl.n_t, d1, d2)
    pitch = (n_in + 15) // 16 * 16
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, n_in, wl.seed, wl.pulses, pitch=pitch)
    k = oracle.coarse_index(wl.dms.size, wl.coarse_dms.size)
    Y = oracle_rows.subband_step1(x, d1, wl.n_subbands, n_1)
    D = oracle_rows.subband_step2(Y, d2, k, wl.n_t)
    s, pt, pv = oracle_rows.snr(D, wl.widths)
    return wl, x, n_1, Y, D, s, pt, pv, oracle.detect(s)


@pytest.mark.parametrize("presum", [0, 1, 2])
def test_apertif_subband_full_tables(lib, apertif_subband_oracle, presum):
    """Every element of Y and D, the S/N tables and the detection of the beam's
    two-step path against the oracle."""
    torch = _torch()
    wl, x, n_1, Yo, Do, s, pt, pv, (bi, bw) = apertif_subband_oracle
    p = lib.Plan.from_workload(wl)
    assert p.pitch == x.shape[1] and p.step1_samples == n_1
    c = p.config
    # quads on the widely spaced coarse trials: smaller DM tiles keep a chunk's tuples in shared memory
    c.step1 = lib.DedispConfig(1, 16, 8, 1, 8, 2) if presum == 2 else lib.DedispConfig(4, 16, 8, 1, 16, presum)
    p.config = c
    xd = torch.from_numpy(x).cuda()
    Y = torch.empty(p.y_shape, dtype=torch.uint16, device="cuda")
    lib.sps_subband_step1(p, xd, Y)
    out = p.search(xd)
    torch.cuda.synchronize()
    assert np.array_equal(_to_np(Y)[:, :, :n_1].astype(np.int32), Yo)
    assert np.array_equal(_to_np(out["D"]), Do)
    _check_snr(_to_np(out["snr"]), _to_np(out["peak_t"]), _to_np(out["peak_val"]), s, pt, pv)
    assert _to_np(out["best"]).tolist() == [bi, bw, int(pt[bw, bi]), int(pv[bw, bi])]
    assert p.status() == 0


# ----------------------------------------------------------------------------- boxcar, S/N
def test_integrate_and_snr_exact(lib):
    torch = _torch()
    rng = np.random.Generator(np.random.PCG64(3))
    n_dms, n_t = 37, 2003
    widths = [1, 2, 3, 16, 64, 2003]
    # D within the plan's range: sums of 1536 uint8 channels
    p = lib.Plan(1536, 1250.0, 1550.0, 81.92e-6, n_t, synth.dm_grid(n_dms, 1.0), widths)
    D = rng.integers(0, 255 * 1536 + 1, (n_dms, n_t)).astype(np.int32)
    D[3] = 7  # constant row: S/N 0
    D[4] = 0
    D[4, 1000] = 123456  # single spike: closed form
    Dd = torch.from_numpy(D).cuda()
    B = torch.empty((len(widths), n_dms, n_t), dtype=torch.int32, device="cuda")
    lib.sps_integrate(p, Dd, B)
    out = p.alloc_outputs()
    lib.sps_snr(p, Dd, out["snr"], out["peak_t"], out["peak_val"], out["best"])
    torch.cuda.synchronize()
    Bn = _to_np(B)
    for wi, w in enumerate(widths):
        for i in range(n_dms):
            want = oracle.boxcar(D[i], w)
            assert np.array_equal(Bn[wi, i, :want.size], want)
            assert np.all(Bn[wi, i, want.size:] == 0)
    s, pt, pv = oracle.snr(D, widths)
    _check_snr(_to_np(out["snr"]), _to_np(out["peak_t"]), _to_np(out["peak_val"]), s, pt, pv)
    bi, bw = oracle.detect(s)
    assert _to_np(out["best"]).tolist() == [bi, bw, int(pt[bw, bi]), int(pv[bw, bi])]
    assert np.all(_to_np(out["snr"])[:, 3] == 0.0)


@pytest.mark.parametrize("threads", [32, 256, 512])
def test_snr_fast_form_long_widths(lib, threads):
    """Few channels keep every boxcar small, so the fast form (64-bit partials,
    no flushes) serves widths up to the whole row: threads whose samples end past
    some widths' last valid start, a width with a single valid start."""
    torch = _torch()
    rng = np.random.Generator(np.random.PCG64(threads + 7))
    n_dms, n_t, widths = 11, 1001, [1, 5, 300, 997, 1001]
    p = lib.Plan(8, 1250.0, 1550.0, 81.92e-6, n_t, synth.dm_grid(n_dms, 1.0), widths)
    c = p.config
    c.snr = lib.SnrConfig(threads)
    p.config = c
    D = rng.integers(0, 255 * 8 + 1, (n_dms, n_t)).astype(np.int32)
    D[1] = 255 * 8          # constant at the largest value: S/N 0, every sample a maximum
    D[2] = 0
    D[2, 1000] = 77         # a spike in the last sample
    D[3] = 0
    D[3, 0] = D[3, 1] = 5   # two in the first samples (a lower S/N: no tie with row 2 for the detection)
    out = p.alloc_outputs()
    lib.sps_snr(p, torch.from_numpy(D).cuda(), out["snr"], out["peak_t"], out["peak_val"], out["best"])
    torch.cuda.synchronize()
    s, pt, pv = oracle.snr(D, widths)
    _check_snr(_to_np(out["snr"]), _to_np(out["peak_t"]), _to_np(out["peak_val"]), s, pt, pv)
    bi, bw = oracle.detect(s)
    assert _to_np(out["best"]).tolist() == [bi, bw, int(pt[bw, bi]), int(pv[bw, bi])]


@pytest.mark.parametrize("threads", [32, 96, 256, 512])
def test_snr_thread_counts(lib, threads):
    torch = _torch()
    rng = np.random.Generator(np.random.PCG64(threads))
    n_dms, n_t = 9, 12500
    p = lib.Plan(1536, 1250.0, 1550.0, 81.92e-6, n_t, synth.dm_grid(n_dms, 1.0), [1, 2, 4, 8, 16, 32, 64])
    c = p.config
    c.snr = lib.SnrConfig(threads)
    p.config = c
    D = rng.integers(150000, 250000, (n_dms, n_t)).astype(np.int32)
    D[:, 5000:5008] += 40000  # a burst so that maxima are distinct
    D[0, :] = 255 * 1536      # the largest value the plan allows: exercises the partial-sum flushes
    out = p.alloc_outputs()
    lib.sps_snr(p, torch.from_numpy(D).cuda(), out["snr"], out["peak_t"], out["peak_val"], out["best"])
    torch.cuda.synchronize()
    s, pt, pv = oracle.snr(D, p.widths)
    _check_snr(_to_np(out["snr"]), _to_np(out["peak_t"]), _to_np(out["peak_val"]), s, pt, pv)


# ----------------------------------------------------------------------------- host entry point
def test_search_host_matches_device_path(lib):
    torch = _torch()
    wl = synth.tiny_brute()
    p = lib.Plan.from_workload(wl)
    x = _x_for(p, wl)
    dev = p.search(torch.from_numpy(x).cuda())
    out = p.alloc_outputs()
    shp = (p.n_widths, p.n_dms)
    hs = torch.empty(shp, dtype=torch.float64).pin_memory()
    ht = torch.empty(shp, dtype=torch.int32).pin_memory()
    hv = torch.empty(shp, dtype=torch.int32).pin_memory()
    hb = torch.empty(4, dtype=torch.int32).pin_memory()
    xh = torch.from_numpy(x).pin_memory()
    xd = torch.empty_like(xh, device="cuda")
    lib.sps_search_host(p, xh, xd, out["D"], out["snr"], out["peak_t"], out["peak_val"], out["best"],
                        hs, ht, hv, hb)
    torch.cuda.synchronize()
    assert np.array_equal(hs.numpy(), _to_np(dev["snr"]))
    assert np.array_equal(ht.numpy(), _to_np(dev["peak_t"]))
    assert np.array_equal(hb.numpy(), _to_np(dev["best"]))


def test_argument_errors(lib):
    torch = _torch()
    wl = synth.tiny_brute()
    p = lib.Plan.from_workload(wl)
    x = torch.zeros((wl.channels, p.pitch), dtype=torch.uint8, device="cuda")
    D = torch.empty((wl.dms.size, wl.n_t), dtype=torch.int32, device="cuda")
    with pytest.raises(lib.SpsError) as e:
        lib.sps_dedisperse(p, x[:, : p.pitch - 16].contiguous(), D)
    assert e.value.status == 1
    with pytest.raises(ValueError):  # one row short: refused before the library would read past it
        lib.sps_dedisperse(p, x[:-1].contiguous(), D)
    xs = torch.zeros(wl.channels * p.pitch + 16, dtype=torch.uint8, device="cuda")[1:1 + wl.channels * p.pitch]
    with pytest.raises(lib.SpsError):
        lib.sps_dedisperse(p, xs.view(wl.channels, p.pitch), D)
    c = p.config
    c.brute = lib.DedispConfig(3, 4, 1, 1, 2)  # no compiled variant
    with pytest.raises(lib.SpsError):
        p.config = c
    # both modes need their workspace (shifted copies, and Y in subband mode)
    L = lib.lib()
    for wl in (synth.tiny_brute(), synth.apertif_beam(subband=True)):
        ps = lib.Plan.from_workload(wl)
        xs = torch.zeros((wl.channels, ps.pitch), dtype=torch.uint8, device="cuda")
        Ds = torch.empty((wl.dms.size, wl.n_t), dtype=torch.int32, device="cuda")
        small = torch.empty(1024, dtype=torch.uint8, device="cuda")  # far below what the plan needs
        import ctypes
        assert L.sps_dedisperse(ps.handle, ctypes.c_void_p(xs.data_ptr()), ps.pitch,
                                ctypes.c_void_p(Ds.data_ptr()), None, 0, None) == 1
        assert L.sps_dedisperse(ps.handle, ctypes.c_void_p(xs.data_ptr()), ps.pitch,
                                ctypes.c_void_p(Ds.data_ptr()), ctypes.c_void_p(small.data_ptr()),
                                small.numel(), None) == 1
    assert p.status() == 0  # no kernel's bounded wait ran out


def test_bounded_wait_runs_out_and_reports(lib):
    """Failure detection without a fault: a wait on an mbarrier that nothing
    arrives at gives up after its poll bound, sets the plan's status word, and
    the context still serves a correct search afterwards."""
    torch = _torch()
    wl = synth.tiny_brute()
    p = lib.Plan.from_workload(wl)
    assert p.status() == 0
    lib.sps_plan_check_wait_timeout(p, polls=1000)
    torch.cuda.synchronize()
    assert p.status(clear=False) == 1          # kStatusWaitTimeout, read without clearing
    assert p.status() == 1                     # read and cleared
    assert p.status() == 0
    with pytest.raises(lib.SpsError):
        lib.sps_plan_check_wait_timeout(p, polls=0)
    x = _x_for(p, wl)
    out = p.search(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    want = oracle.dedisperse(x, oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms), wl.n_t)
    assert np.array_equal(_to_np(out["D"]), want)
    assert p.status() == 0


def test_int_add_rate_is_plausible(lib):
    """The measured integer add rate (the roofline's measured denominator) lies
    between 1e12 adds/s and 2.5 x the 152 SM x 128 lane x 2.07 GHz unit count."""
    r = lib.sps_measure_int_add_rate()
    assert 1e12 < r < 2.5 * 152 * 128 * 2.07e9


@pytest.mark.parametrize("n_t", [64, 100, 1000, 4096, 12500])
@pytest.mark.parametrize("n_w", [1, 3, 7])
@pytest.mark.parametrize("threads", [32, 96, 256, 512])
def test_snr_power_of_two_widths_edges(lib, n_t, n_w, threads):
    """Widths 1, 2, ..., 2^(n_w - 1) take the vector form with the detection
    folded in: rows whose maximum sits at the first or last valid
    sample of a width, a maximum repeated in many segments (the first must
    win), constant and zero rows, the largest value the plan allows, and two
    identical rows (the detection takes the smaller DM index)."""
    torch = _torch()
    widths = [1 << k for k in range(n_w)]
    if widths[-1] > n_t:
        pytest.skip("widest boxcar longer than the row")
    rng = np.random.Generator(np.random.PCG64(n_t * 10 + n_w))
    C = 1536
    n_dms = 12
    p = lib.Plan(C, 1250.0, 1550.0, 81.92e-6, n_t, synth.dm_grid(n_dms, 1.0), widths)
    c = p.config
    c.snr = lib.SnrConfig(threads)
    p.config = c
    D = rng.integers(180000, 220000, (n_dms, n_t)).astype(np.int32)
    D[0] = 7                          # constant: S/N 0 everywhere, peak at t = 0
    D[1] = 0
    D[1, 0] = 255 * C                 # spike at the first sample
    D[2] = 0
    D[2, n_t - 1] = 255 * C           # spike at the last sample: only width 1 sees it at t = n_t - 1
    D[2, n_t // 3] = 3                # (and a small one: no exact S/N tie with row 1, which FP64
                                      # rounding in the oracle's two-pass sigma could break either way)
    D[3] = 0
    D[3, ::37] = 1000                 # the same maximum in many segments
    D[4] = 255 * C                    # the largest value everywhere
    D[5, :] = np.arange(n_t) % 251    # a ramp
    D[6] = D[7]                       # identical rows: a detection tie goes to the smaller index
    D[7, n_t // 2] = 255 * C
    D[6] = D[7]
    out = p.alloc_outputs()
    out["best"].fill_(-5)
    lib.sps_snr(p, torch.from_numpy(D).cuda(), out["snr"], out["peak_t"], out["peak_val"], out["best"])
    torch.cuda.synchronize()
    s, pt, pv = oracle.snr(D, widths)
    _check_snr(_to_np(out["snr"]), _to_np(out["peak_t"]), _to_np(out["peak_val"]), s, pt, pv)
    bi, bw = oracle.detect(s)
    assert _to_np(out["best"]).tolist() == [bi, bw, int(pt[bw, bi]), int(pv[bw, bi])]
    assert p.status() == 0


@pytest.mark.parametrize("S", [16, 64])
def test_apertif_subband_counts_full_tables(lib, S):
    """The beam's two-step path with 16 and 64 subbands (the counts the joint
    tuner explores beside 32): every element of D and the S/N tables against
    the oracle's two steps with that subband count."""
    torch = _torch()
    wl = synth.apertif_beam(subband=True)
    wl.n_subbands = S
    d1, d2 = oracle.subband_tables(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, S, wl.coarse_dms, wl.dms)
    n_1, n_in = oracle.subband_lengths(wl.n_t, d1, d2)
    p = lib.Plan.from_workload(wl)
    assert (p.step1_samples, p.input_samples) == (n_1, n_in)
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, n_in, wl.seed, wl.pulses, pitch=p.pitch)
    out = p.search(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    Y = oracle_rows.subband_step1(x, d1, S, n_1)
    Do = oracle_rows.subband_step2(Y, d2, oracle.coarse_index(wl.dms.size, wl.coarse_dms.size), wl.n_t)
    assert np.array_equal(_to_np(out["D"]), Do)
    s, pt, pv = oracle_rows.snr(Do, wl.widths)
    _check_snr(_to_np(out["snr"]), _to_np(out["peak_t"]), _to_np(out["peak_val"]), s, pt, pv)
    assert p.status() == 0


@pytest.mark.parametrize("presum", [0, 2])
def test_one_plan_on_concurrent_streams(lib, presum):
    """A plan is read-only once configured, so one plan serves searches on several
    streams at once (each with its own workspace and outputs), as the benchmark's
    pipelined run does: four streams, three rounds of interleaved searches on
    different inputs, every result against the oracle."""
    torch = _torch()
    C, n_t, n_dms = 256, 3000, 96
    dms = synth.dm_grid(n_dms, 0.5)
    p = lib.Plan(C, 1250.0, 1550.0, 81.92e-6, n_t, dms, [1, 2, 4, 8, 16])
    c = p.config
    c.brute.presum = presum
    p.config = c
    streams = [torch.cuda.Stream() for _ in range(4)]
    xs, wss, outs = [], [], []
    for k in range(4):
        x = synth.filterbank(C, 1250.0, 1550.0, 81.92e-6, p.input_samples, 300 + k,
                             [synth.Pulse(float(dms[20 + 15 * k]), 2.0 + k, 25.0, 500.0 + 400 * k)], pitch=p.pitch)
        xs.append(x)
        wss.append(torch.empty(p.workspace_bytes, dtype=torch.uint8, device="cuda"))
        outs.append(p.alloc_outputs())
    xd = [torch.from_numpy(x).cuda() for x in xs]
    torch.cuda.synchronize()
    for _ in range(3):
        for k, s in enumerate(streams):
            o = outs[k]
            lib.sps_search(p, xd[k], o["D"], o["snr"], o["peak_t"], o["peak_val"], o["best"], workspace=wss[k],
                           stream=s)
    torch.cuda.synchronize()
    delays = oracle.delay_table(1250.0, 1550.0, C, 81.92e-6, dms)
    for k in range(4):
        Do = oracle.dedisperse(xs[k], delays, n_t)
        assert np.array_equal(_to_np(outs[k]["D"]), Do), k
        s, pt, pv = oracle.snr(Do, [1, 2, 4, 8, 16])
        _check_snr(_to_np(outs[k]["snr"]), _to_np(outs[k]["peak_t"]), _to_np(outs[k]["peak_val"]), s, pt, pv)
        bi, bw = oracle.detect(s)
        assert _to_np(outs[k]["best"]).tolist() == [bi, bw, int(pt[bw, bi]), int(pv[bw, bi])]
    assert p.status() == 0


@pytest.mark.parametrize("threads", [64, 256])
def test_snr_rows_longer_than_shared_memory(lib, threads):
    """Rows too long to stage whole in shared memory (70000 samples, 280 KB) take
    the streaming S/N form: edge rows and noise rows against the oracle, and a
    whole search on such rows; a width set without a streaming form is refused
    with UNSUPPORTED rather than run."""
    torch = _torch()
    n_t, C, n_dms = 70000, 256, 8
    widths = [1, 2, 4, 8, 16, 32, 64]
    dms = synth.dm_grid(n_dms, 2.0)
    p = lib.Plan(C, 1250.0, 1550.0, 81.92e-6, n_t, dms, widths)
    c = p.config
    c.snr = lib.SnrConfig(threads)
    p.config = c
    rng = np.random.Generator(np.random.PCG64(77))
    D = rng.integers(30000, 35000, (n_dms, n_t)).astype(np.int32)
    D[0] = 11                                   # constant row
    D[1] = 0
    D[1, 0] = 255 * C                           # spike at the first sample
    D[2] = 0
    D[2, n_t - 1] = 255 * C                     # spike at the last sample
    D[2, 12345] = 5
    D[3] = 0
    D[3, ::4097] = 999                          # the same maximum in many chunks
    D[4, n_t // 2: n_t // 2 + 40] += 20000      # a wide pulse
    out = p.alloc_outputs()
    lib.sps_snr(p, torch.from_numpy(D).cuda(), out["snr"], out["peak_t"], out["peak_val"], out["best"])
    torch.cuda.synchronize()
    s, pt, pv = oracle.snr(D, widths)
    _check_snr(_to_np(out["snr"]), _to_np(out["peak_t"]), _to_np(out["peak_val"]), s, pt, pv)
    bi, bw = oracle.detect(s)
    assert _to_np(out["best"]).tolist() == [bi, bw, int(pt[bw, bi]), int(pv[bw, bi])]
    # a whole search on such rows
    x = synth.filterbank(C, 1250.0, 1550.0, 81.92e-6, p.input_samples, 78,
                         [synth.Pulse(float(dms[5]), 8.0, 20.0, 40000.0)], pitch=p.pitch)
    o = p.search(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    Do = oracle.dedisperse(x, oracle.delay_table(1250.0, 1550.0, C, 81.92e-6, dms), n_t)
    assert np.array_equal(_to_np(o["D"]), Do)
    s, pt, pv = oracle.snr(Do, widths)
    _check_snr(_to_np(o["snr"]), _to_np(o["peak_t"]), _to_np(o["peak_val"]), s, pt, pv)
    assert p.status() == 0
    # widths that are not 1, 2, 4, ... on such rows: refused
    q = lib.Plan(C, 1250.0, 1550.0, 81.92e-6, n_t, dms, [1, 3, 9])
    oq = q.alloc_outputs()
    with pytest.raises(lib.SpsError) as e:
        lib.sps_snr(q, torch.from_numpy(D).cuda(), oq["snr"], oq["peak_t"], oq["peak_val"], oq["best"])
    assert e.value.status == 2
