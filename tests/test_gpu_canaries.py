"""Out-of-bounds writes: every output buffer and the workspace sit between
256-byte guard regions filled with a known pattern; after a search the guards
must be untouched and the results must still equal the oracle's.  Covers the
single-channel, pair and quad de-dispersion kernels with their pre-pass, the
subband steps, decimating S/N with zapped channels, and the integrate kernel."""
import numpy as np
import pytest

import oracle
from paper_1811_04165_gb300 import synth

pytestmark = pytest.mark.gpu

GUARD_BYTES = 256
FILL = 0xA5


def _guarded(torch, shape, dtype):
    """(byte buffer, tensor of `shape` and `dtype` between two guards)."""
    nbytes = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
    buf = torch.full((nbytes + 2 * GUARD_BYTES,), FILL, dtype=torch.uint8, device="cuda")
    return buf, buf[GUARD_BYTES:GUARD_BYTES + nbytes].view(dtype).view(*shape)


def _intact(buf):
    b = buf.cpu().numpy()
    return bool(np.all(b[:GUARD_BYTES] == FILL) and np.all(b[-GUARD_BYTES:] == FILL))


def _search_guarded(lib, p, x):
    import torch
    shp = (p.n_widths, p.n_dms)
    bufs = {}
    out = {}
    for k, shape, dt in (("D", (p.n_dms, p.n_samples), torch.int32), ("snr", shp, torch.float64),
                         ("peak_t", shp, torch.int32), ("peak_val", shp, torch.int32), ("best", (4,), torch.int32)):
        bufs[k], out[k] = _guarded(torch, shape, dt)
    wbuf, ws = _guarded(torch, (p.workspace_bytes,), torch.uint8)
    p.search(torch.from_numpy(x).cuda(), out=out, workspace=ws)
    torch.cuda.synchronize()
    for k, buf in bufs.items():
        assert _intact(buf), f"write outside {k}"
    assert _intact(wbuf), "write outside the workspace"
    assert p.status() == 0
    return {k: v.cpu().numpy() for k, v in out.items()}


def _x(p, wl):
    return synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, p.input_samples, wl.seed, wl.pulses,
                            pitch=p.pitch)


@pytest.mark.parametrize("presum", [0, 1, 2])
def test_brute_force_writes_stay_inside(lib, presum):
    dms = synth.dm_grid(37, 0.31)
    wl = synth.Workload("guard", 61, 1300.0, 1500.0, 65.536e-6, 1003, dms, np.array([1, 3, 50], np.int32), seed=3)
    p = lib.Plan.from_workload(wl)
    c = p.config
    c.brute = lib.DedispConfig(4, 8, 2, 2, 12, presum)
    p.config = c
    x = _x(p, wl)
    got = _search_guarded(lib, p, x)
    want = oracle.dedisperse(x, oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, dms), wl.n_t)
    assert np.array_equal(got["D"], want)
    s, pt, pv = oracle.snr(want, wl.widths)
    assert np.allclose(got["snr"], s, rtol=1e-5, atol=1e-9) and np.array_equal(got["peak_t"], pt)


def test_apertif_quads_writes_stay_inside(lib):
    wl = synth.apertif_beam()
    p = lib.Plan.from_workload(wl)
    x = _x(p, wl)
    got = _search_guarded(lib, p, x)
    rows = np.array([0, 1023, 2047])
    want = oracle.dedisperse(x, oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)[rows], wl.n_t)
    assert np.array_equal(got["D"][rows], want)


def test_subband_writes_stay_inside(lib):
    import torch
    dms = synth.dm_grid(48, 1.3)
    wl = synth.Workload("guard-sub", 64, 1250.0, 1550.0, 81.92e-6, 999, dms, np.array([1, 4], np.int32), seed=8,
                        n_subbands=8, coarse_dms=dms[::8].copy())
    p = lib.Plan.from_workload(wl)
    x = _x(p, wl)
    got = _search_guarded(lib, p, x)
    d1, d2 = oracle.subband_tables(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, 8, wl.coarse_dms, wl.dms)
    n_1, _ = oracle.subband_lengths(wl.n_t, d1, d2)
    Yo = oracle.subband_step1(x, d1, 8, n_1)
    Do = oracle.subband_step2(Yo, d2, oracle.coarse_index(wl.dms.size, wl.coarse_dms.size), wl.n_t)
    assert np.array_equal(got["D"], Do)
    # step one alone into a guarded Y
    ybuf, Y = _guarded(torch, p.y_shape, torch.uint16)
    lib.sps_subband_step1(p, torch.from_numpy(x).cuda(), Y)
    torch.cuda.synchronize()
    assert _intact(ybuf)
    assert np.array_equal(Y.cpu().numpy()[:, :, :n_1].astype(np.int32), Yo)


def test_decimated_zapped_and_integrate_writes_stay_inside(lib):
    import torch
    dms = synth.dm_grid(40, 1.5)
    zap = np.zeros(64, np.uint8)
    zap[[0, 9, 33, 63]] = 1
    factors = np.array([1, 3, 10, 100], np.int32)
    wl = synth.Workload("guard-dec", 64, 1250.0, 1550.0, 81.92e-6, 2003, dms, factors, seed=17,
                        pulses=[synth.Pulse(30.0, 8.0, 60.0, 700.0)], smoothing=lib.SMOOTH_DECIMATE, zap=zap)
    p = lib.Plan.from_workload(wl)
    x = _x(p, wl)
    got = _search_guarded(lib, p, x)
    D = oracle.dedisperse(oracle.zap_channels(x, zap),
                          oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, dms), wl.n_t)
    assert np.array_equal(got["D"], D)
    s, pt, pv = oracle.snr_decimated(D, factors)
    assert np.allclose(got["snr"], s, rtol=1e-5, atol=1e-9) and np.array_equal(got["peak_t"], pt)
    bbuf, B = _guarded(torch, (factors.size, dms.size, wl.n_t), torch.int32)
    lib.sps_integrate(p, torch.from_numpy(got["D"]).cuda(), B)
    torch.cuda.synchronize()
    assert _intact(bbuf)
    for k, f in enumerate(factors):
        X = oracle.decimate(D, int(f))
        assert np.array_equal(B.cpu().numpy()[k, :, :X.shape[1]], X)
