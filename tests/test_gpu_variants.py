"""AMBER-style variants against the oracle: decimating downsampling with S/N on
every downsampled series (Table 2 DOWNSAMPLING / NRSAMPLES, Sec. 5), and RFI
channel zapping (Sec. 2 footnote)."""
import numpy as np
import pytest

import oracle
from paper_1811_04165_gb300 import synth
from tests import oracle_rows

pytestmark = pytest.mark.gpu


def _x(p, wl, seed=None):
    return synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, p.input_samples, wl.seed if seed is None else seed,
                            wl.pulses, pitch=p.pitch)


def _small(factors, smoothing, zap=None, n_t=2003, step=1.5):
    dms = synth.dm_grid(40, step)
    wl = synth.Workload("small", 64, 1250.0, 1550.0, 81.92e-6, n_t, dms, np.array(factors, np.int32), seed=17,
                        pulses=[synth.Pulse(30.0, 8.0, 60.0, 700.0)], smoothing=smoothing, zap=zap)
    return wl


@pytest.mark.parametrize("factors", [[1, 3, 10, 64, 100], [1, 2, 4, 7, 9, 16, 33, 50, 128, 1000]])
def test_decimated_snr_matches_the_oracle(lib, factors):
    import torch
    wl = _small(factors, lib.SMOOTH_DECIMATE)
    p = lib.Plan.from_workload(wl)
    x = _x(p, wl)
    out = p.search(torch.from_numpy(x).cuda())
    B = torch.empty((len(factors), wl.dms.size, wl.n_t), dtype=torch.int32, device="cuda")
    lib.sps_integrate(p, out["D"], B)
    torch.cuda.synchronize()
    D = oracle.dedisperse(x, oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms), wl.n_t)
    assert np.array_equal(out["D"].cpu().numpy(), D)
    s, pt, pv = oracle.snr_decimated(D, factors)
    assert np.allclose(out["snr"].cpu().numpy(), s, rtol=1e-5, atol=1e-9)
    assert np.array_equal(out["peak_t"].cpu().numpy(), pt)
    assert np.array_equal(out["peak_val"].cpu().numpy(), pv)
    assert out["best"].cpu().numpy()[:2].tolist() == list(oracle.detect(s))
    Bh = B.cpu().numpy()
    for k, f in enumerate(factors):
        X = oracle.decimate(D, f)
        assert np.array_equal(Bh[k, :, :X.shape[1]], X)
        assert not Bh[k, :, X.shape[1]:].any()


@pytest.mark.parametrize("presum", [0, 1, 2])
def test_zapped_channels_contribute_nothing(lib, presum):
    import torch
    rng = np.random.Generator(np.random.PCG64(presum + 3))
    zap = (rng.random(64) < 0.2).astype(np.uint8)
    zap[0] = zap[63] = 1  # the reference and the most delayed channel too
    # a fine DM grid keeps the pre-summed kernels' tuples per tile few on 4.7 MHz channels
    wl = _small([1, 4, 16], lib.SMOOTH_SLIDING, zap=zap, step=0.1)
    p = lib.Plan.from_workload(wl)
    c = p.config
    if presum:
        c.brute = lib.DedispConfig(4, 16, 8, 1, 8, presum)
    else:
        c.brute.presum = 0
    p.config = c
    x = _x(p, wl)
    out = p.search(torch.from_numpy(x).cuda(), workspace=p.workspace())
    torch.cuda.synchronize()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    want = oracle.dedisperse(oracle.zap_channels(x, zap), d, wl.n_t)
    assert np.array_equal(out["D"].cpu().numpy(), want)
    s, pt, pv = oracle.snr(want, wl.widths)
    assert np.allclose(out["snr"].cpu().numpy(), s, rtol=1e-5, atol=1e-9)
    assert np.array_equal(out["peak_t"].cpu().numpy(), pt)


def test_zapping_in_subband_mode(lib):
    import torch
    zap = np.zeros(64, np.uint8)
    zap[[5, 6, 7, 20, 41]] = 1
    dms = synth.dm_grid(48, 1.3)
    wl = synth.Workload("sub", 64, 1250.0, 1550.0, 81.92e-6, 1500, dms, np.array([1, 4], np.int32), seed=8,
                        n_subbands=8, coarse_dms=dms[::8].copy(), zap=zap)
    p = lib.Plan.from_workload(wl)
    x = _x(p, wl)
    out = p.search(torch.from_numpy(x).cuda(), workspace=p.workspace())
    torch.cuda.synchronize()
    d1, d2 = oracle.subband_tables(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, 8, wl.coarse_dms, wl.dms)
    n_1, _ = oracle.subband_lengths(wl.n_t, d1, d2)
    xz = oracle.zap_channels(x, zap)
    Do = oracle.subband_step2(oracle.subband_step1(xz, d1, 8, n_1), d2,
                              oracle.coarse_index(wl.dms.size, wl.coarse_dms.size), wl.n_t)
    assert np.array_equal(out["D"].cpu().numpy(), Do)


def test_apertif_beam_decimated_and_zapped(lib):
    """The full beam with the paper's downsampling range (Table 2: 10 .. 3200)
    plus the raw series, and an RFI mask: every row of D and every S/N, peak and
    the detection against the oracle."""
    import torch
    base = synth.apertif_beam()
    rng = np.random.Generator(np.random.PCG64(99))
    zap = (rng.random(base.channels) < 0.05).astype(np.uint8)
    factors = [1, 10, 20, 40, 80, 160, 320, 640, 1280, 2560]
    wl = synth.Workload(base.name, base.channels, base.f_lo, base.f_hi, base.t_samp, base.n_t, base.dms,
                        np.array(factors, np.int32), seed=base.seed, pulses=base.pulses,
                        smoothing=lib.SMOOTH_DECIMATE, zap=zap)
    p = lib.Plan.from_workload(wl)
    x = _x(p, wl)
    out = p.search(torch.from_numpy(x).cuda(), workspace=p.workspace())
    torch.cuda.synchronize()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    want = oracle_rows.dedisperse(oracle.zap_channels(x, zap), d, wl.n_t)
    assert np.array_equal(out["D"].cpu().numpy(), want)
    s, pt, pv = oracle_rows.snr_decimated(want, factors)
    assert np.allclose(out["snr"].cpu().numpy(), s, rtol=1e-5, atol=1e-9)
    assert np.array_equal(out["peak_t"].cpu().numpy(), pt)
    assert np.array_equal(out["peak_val"].cpu().numpy(), pv)
    bi, bw = oracle.detect(s)
    assert out["best"].cpu().numpy().tolist() == [bi, bw, int(pt[bw, bi]), int(pv[bw, bi])]
    assert p.status() == 0
