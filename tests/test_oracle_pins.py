"""Pins for the CPU oracle: values and properties fixed by the mathematics and by
the paper, each independent of the oracle's own code.

Every plausible slip in the oracle (a dropped channel, a sign or index error in
a delay, a transposed table, an off-by-one in a boxcar, sample instead of
population sigma, a wrong tie-break) fails at least one test here.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1811_04165_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------- frequencies
def test_channel_grid_matches_table2_bandwidth():
    # Table 2: 1536 channels of 0.1953125 MHz; the Apertif beam spans 300 MHz.
    g = json.load(open(os.path.join(GOLDEN, "table2_survey.json")))
    wl = synth.apertif_beam()
    f = oracle.channel_freqs(wl.f_lo, wl.f_hi, wl.channels)
    assert wl.channels == g["CHANNELS"]
    assert np.all(np.diff(f) == g["CHANNEL_BANDWIDTH_MHZ"])
    assert f[0] == wl.f_lo + g["CHANNEL_BANDWIDTH_MHZ"] / 2  # centre of the lowest channel


# --------------------------------------------------------------------------- delays
def _exact_delay(f_lo, f_hi, channels, t_samp, dm, c):
    """Exact rational delay (same double inputs, no rounding inside)."""
    F = Fraction
    df = (F(f_hi) - F(f_lo)) / channels
    fc = F(f_lo) + (F(c) + F(1, 2)) * df
    fr = F(f_lo) + (F(channels - 1) + F(1, 2)) * df
    return F(oracle.K_DM) * F(dm) * (1 / (fc * fc) - 1 / (fr * fr)) / F(t_samp)


def _round_half_away(q: Fraction) -> int:
    n = int(abs(q) + Fraction(1, 2))
    return n if q >= 0 else -n


def test_delay_table_against_exact_rationals():
    wl = synth.tiny_brute()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    for i in range(wl.dms.size):
        for c in range(wl.channels):
            q = _exact_delay(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, float(wl.dms[i]), c)
            frac = q - int(q)
            if abs(frac - Fraction(1, 2)) < Fraction(1, 10**6):
                continue  # FP64 may legitimately round a near-half either way
            assert d[i, c] == _round_half_away(q), (i, c, float(q))


def test_delay_table_sampled_apertif_exact():
    wl = synth.apertif_beam()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    r = _rng(5)
    for i, c in zip(r.integers(0, wl.dms.size, 400).tolist(), r.integers(0, wl.channels, 400).tolist()):
        q = _exact_delay(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, float(wl.dms[i]), c)
        if abs(q - int(q) - Fraction(1, 2)) < Fraction(1, 10**6):
            continue
        assert d[i, c] == _round_half_away(q)


def test_delay_textbook_units():
    # Textbook form: delay_ms = 4.148808 ms * DM * (nu_lo^-2 - nu_hi^-2), nu in GHz.
    wl = synth.tiny_brute()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    f = oracle.channel_freqs(wl.f_lo, wl.f_hi, wl.channels) / 1e3
    dm = wl.dms[25]
    ms = 4.148808 * dm * (f[0] ** -2 - f[-1] ** -2)
    assert abs(d[25, 0] - ms * 1e-3 / wl.t_samp) <= 0.5


def test_delay_special_cases_and_monotone():
    wl = synth.apertif_beam()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    assert np.all(d[:, -1] == 0)            # the top channel is the reference
    assert np.all(d[0, :] == 0)             # DM 0 has no sweep
    assert np.all(np.diff(d, axis=1) <= 0)  # lower frequency arrives later
    assert np.all(np.diff(d, axis=0) >= 0)  # larger DM, longer sweep
    assert d.max() == d[-1, 0]


# --------------------------------------------------------------------------- dedispersion
def test_dedisperse_hand_example():
    # Four channels, eight samples, two DM rows, worked by hand.
    x = np.array([[1, 2, 3, 4, 5, 6, 7, 8],
                  [10, 20, 30, 40, 50, 60, 70, 80],
                  [100, 0, 100, 0, 100, 0, 100, 0],
                  [7, 7, 7, 7, 7, 7, 7, 7]], np.uint8)
    delays = np.array([[0, 0, 0, 0], [3, 2, 1, 0]], np.int32)
    D = oracle.dedisperse(x, delays, 4)
    assert D.tolist() == [
        [1 + 10 + 100 + 7, 2 + 20 + 0 + 7, 3 + 30 + 100 + 7, 4 + 40 + 0 + 7],
        [4 + 30 + 0 + 7, 5 + 40 + 100 + 7, 6 + 50 + 0 + 7, 7 + 60 + 100 + 7]]


def test_dedisperse_dm0_is_channel_sum():
    wl = synth.tiny_brute()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_t + int(d.max()), 3)
    D = oracle.dedisperse(x, d, wl.n_t)
    assert np.array_equal(D[0], x[:, :wl.n_t].astype(np.int64).sum(axis=0))


@pytest.mark.parametrize("seed", range(6))
def test_dedisperse_against_slice_sums(seed):
    r = _rng(seed)
    C, n_t, n_dm = int(r.integers(1, 9)), int(r.integers(1, 33)), int(r.integers(1, 6))
    delays = r.integers(0, 12, (n_dm, C)).astype(np.int32)
    x = r.integers(0, 256, (C, n_t + 12)).astype(np.uint8)
    x[0, :min(256, x.shape[1])] = np.arange(min(256, x.shape[1]))  # include many byte values
    want = np.zeros((n_dm, n_t), np.int64)
    for i in range(n_dm):
        for c in range(C):
            want[i] += x[c, delays[i, c]:delays[i, c] + n_t]
    assert np.array_equal(oracle.dedisperse(x, delays, n_t), want)


def test_dedisperse_saturated_input():
    wl = synth.apertif_beam()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms[::128])
    x = np.full((wl.channels, 64 + int(d.max())), 255, np.uint8)
    assert np.all(oracle.dedisperse(x, d, 64) == 255 * wl.channels)


def test_injected_pulse_recovered_tiny():
    # One pulse at DM 50 (trial 25), width 4, leading edge at sample 1024 of the top channel.
    wl = synth.tiny_brute()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_t + int(d.max()), wl.seed,
                         wl.pulses)
    D = oracle.dedisperse(x, d, wl.n_t)
    s, pt, pv = oracle.snr(D, wl.widths)
    i, w = oracle.detect(s)
    assert (i, int(wl.widths[w]), int(pt[w, i])) == (25, 4, 1024)
    assert s[w, i] > 20


@pytest.mark.slow
def test_injected_pulse_recovered_apertif_strongest():
    wl = synth.apertif_beam()
    dms = wl.dms
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, dms)
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_t + int(d.max()), wl.seed,
                         wl.pulses)
    strongest = max(wl.pulses, key=lambda p: p.amp * np.sqrt(p.width))
    near = int(round(strongest.dm / 0.2))
    rows = np.arange(max(near - 40, 0), min(near + 41, dms.size))
    D = oracle.dedisperse(x, d[rows], wl.n_t)
    s, pt, pv = oracle.snr(D, wl.widths)
    i, w = oracle.detect(s)
    assert abs(dms[rows[i]] - strongest.dm) <= 0.2 + 1e-9
    assert strongest.width / 2 <= wl.widths[w] <= strongest.width * 2
    assert abs(pt[w, i] - strongest.t0) <= strongest.width


# --------------------------------------------------------------------------- subband
def _small_band(C=48, n_t=300):
    return dict(f_lo=1250.0, f_hi=1550.0, channels=C, t_samp=81.92e-6, n_t=n_t)


def _subband_D(x, b, S, coarse, dms, coarse_of):
    d1, d2 = oracle.subband_tables(b["f_lo"], b["f_hi"], b["channels"], b["t_samp"], S, coarse, dms)
    n_1 = b["n_t"] + int(d2.max())
    Y = oracle.subband_step1(x, d1, S, n_1)
    return oracle.subband_step2(Y, d2, coarse_of, b["n_t"]), d1, d2


def test_subband_with_one_channel_per_subband_is_brute_force():
    b = _small_band()
    dms = synth.dm_grid(24, 1.5)
    d = oracle.delay_table(b["f_lo"], b["f_hi"], b["channels"], b["t_samp"], dms)
    x = synth.filterbank(b["channels"], b["f_lo"], b["f_hi"], b["t_samp"], b["n_t"] + 800, 11)
    coarse = dms[::4]
    D_sub, d1, d2 = _subband_D(x, b, b["channels"], coarse, dms, oracle.coarse_index(24, 6))
    assert np.all(d1 == 0) and np.array_equal(d2, d)
    assert np.array_equal(D_sub, oracle.dedisperse(x, d, b["n_t"]))


def test_subband_with_one_subband_is_brute_force_at_coarse_dm():
    b = _small_band()
    dms = synth.dm_grid(24, 1.5)
    coarse = dms[::6]
    k = oracle.coarse_index(24, 4)
    x = synth.filterbank(b["channels"], b["f_lo"], b["f_hi"], b["t_samp"], b["n_t"] + 800, 12)
    D_sub, d1, d2 = _subband_D(x, b, 1, coarse, dms, k)
    assert np.all(d2 == 0)
    d_coarse = oracle.delay_table(b["f_lo"], b["f_hi"], b["channels"], b["t_samp"], coarse)
    assert np.array_equal(D_sub, oracle.dedisperse(x, d_coarse[k], b["n_t"]))


@pytest.mark.parametrize("S", [2, 4, 8, 16])
def test_subband_composition_identity(S):
    # Two integer shifts compose: step one then step two equals one pass with
    # the composed delay d1[k(i), c] + d2[i, s(c)].
    b = _small_band()
    dms = synth.dm_grid(32, 1.25)
    coarse = dms[::8]
    k = oracle.coarse_index(32, 4)
    x = synth.filterbank(b["channels"], b["f_lo"], b["f_hi"], b["t_samp"], b["n_t"] + 800, 13 + S)
    D_sub, d1, d2 = _subband_D(x, b, S, coarse, dms, k)
    s_of_c = np.arange(b["channels"]) // (b["channels"] // S)
    composed = d1[k] + d2[:, s_of_c]
    assert np.array_equal(D_sub, oracle.dedisperse(x, composed, b["n_t"]))
    # each subband's top channel carries no intra-subband delay; the top subband none across
    assert np.all(d1[:, (np.arange(S) + 1) * (b["channels"] // S) - 1] == 0)
    assert np.all(d2[:, -1] == 0)
    # the coarse trial itself equals brute force where the delays coincide (DM 0)
    assert np.array_equal(D_sub[0], x[:, :b["n_t"]].astype(np.int64).sum(axis=0))


def test_coarse_index_hand_example():
    # k(i) = floor(i / (n_dms / n_coarse)): each coarse DM serves the block of
    # consecutive fine trials that starts at it (Sec. 2, first footnote: step one
    # at the coarse DM, step two at the trial's own DM).  Worked by hand.
    assert oracle.coarse_index(8, 2).tolist() == [0, 0, 0, 0, 1, 1, 1, 1]
    assert oracle.coarse_index(6, 3).tolist() == [0, 0, 1, 1, 2, 2]
    assert oracle.coarse_index(5, 5).tolist() == [0, 1, 2, 3, 4]
    assert oracle.coarse_index(4, 1).tolist() == [0, 0, 0, 0]


def test_coarse_index_apertif_grid():
    # The beam's two-step grid: 64 coarse DMs 6.4 apart, each followed by 32
    # fine trials 0.2 apart, so DM_i = 6.4 k + 0.2 j with i = 32 k + j; the
    # coarse DM of trial i is 6.4 floor(i / 32) and the fine offset 0.2 (i mod 32).
    wl = synth.apertif_beam(subband=True)
    k = oracle.coarse_index(wl.dms.size, wl.coarse_dms.size)
    i = np.arange(2048)
    assert np.allclose(wl.coarse_dms[k], 6.4 * (i // 32), rtol=0, atol=1e-9)
    assert np.allclose(wl.dms - wl.coarse_dms[k], 0.2 * (i % 32), rtol=0, atol=1e-9)
    # each coarse DM lies at or below every trial it serves, and serves 32 of them
    assert np.all(wl.coarse_dms[k] <= wl.dms + 1e-12)
    assert np.array_equal(np.bincount(k), np.full(64, 32))


def _exact_k(f_lo, f_hi, channels, t_samp, c, c_ref):
    """Exact rational delay per unit DM of channel c against channel c_ref."""
    F = Fraction
    df = (F(f_hi) - F(f_lo)) / channels
    fc = F(f_lo) + (F(c) + F(1, 2)) * df
    fr = F(f_lo) + (F(c_ref) + F(1, 2)) * df
    return F(oracle.K_DM) * (1 / (fc * fc) - 1 / (fr * fr)) / F(t_samp)


def test_subband_lengths_hand_example():
    # Step two reads Y[k][s][t + d2] for t < N_t, so N_1 = N_t + max d2; step one
    # reads x[c][t' + d1] for t' < N_1, so N_in = N_1 + max d1.  By hand:
    # N_t = 10, max d2 = 5 -> N_1 = 15; max d1 = 3 -> N_in = 18.
    d1 = np.array([[0, 3], [1, 0]], np.int32)
    d2 = np.array([[2], [5]], np.int32)
    assert oracle.subband_lengths(10, d1, d2) == (15, 18)
    assert oracle.subband_lengths(7, np.zeros((1, 4), np.int32), np.array([[9]], np.int32)) == (16, 16)


def test_subband_apertif_lengths():
    # The beam's subband path from the delay law in exact rationals: the largest
    # step-one delay is at the largest coarse DM (403.2), the largest step-two
    # delay at the largest trial DM (409.4): 190 and 4444 samples, so
    # N_1 = 12500 + 4444 = 16944 and N_in = 16944 + 190 = 17134.
    wl = synth.apertif_beam(subband=True)
    C, S = wl.channels, 32
    per = C // S
    d1, d2 = oracle.subband_tables(wl.f_lo, wl.f_hi, C, wl.t_samp, S, wl.coarse_dms, wl.dms)
    assert (d1.shape, d2.shape) == ((64, 1536), (2048, 32))
    exact_d1 = max(_round_half_away(Fraction(float(wl.coarse_dms[-1])) *
                                    _exact_k(wl.f_lo, wl.f_hi, C, wl.t_samp, c, (c // per + 1) * per - 1))
                   for c in range(C))
    exact_d2 = max(_round_half_away(Fraction(float(wl.dms[-1])) *
                                    _exact_k(wl.f_lo, wl.f_hi, C, wl.t_samp, (s + 1) * per - 1, C - 1))
                   for s in range(S))
    assert (exact_d1, exact_d2) == (190, 4444)
    assert (int(d1.max()), int(d2.max())) == (190, 4444)
    assert oracle.subband_lengths(wl.n_t, d1, d2) == (16944, 17134)


# --------------------------------------------------------------------------- boxcar
@pytest.mark.parametrize("w", [1, 2, 3, 8, 17])
def test_boxcar_is_valid_convolution(w):
    D = _rng(w).integers(0, 400000, 64).astype(np.int32)
    B = oracle.boxcar(D, w)
    assert np.array_equal(B, np.convolve(D.astype(np.int64), np.ones(w, np.int64), "valid"))


def test_boxcar_width_one_and_full():
    D = _rng(3).integers(-5, 5, 33).astype(np.int32)
    assert np.array_equal(oracle.boxcar(D, 1), D)
    assert oracle.boxcar(D, 33).tolist() == [int(D.astype(np.int64).sum())]


# --------------------------------------------------------------------------- S/N
def test_snr_hand_example():
    D = np.array([[41, 152, 63, 174]], np.int32)
    s, pt, pv = oracle.snr(D, [1, 2])
    # w = 2: B = (193, 215, 237), mean 215, sigma = 22 sqrt(2/3) -> S/N = sqrt(3/2)
    assert (pt[1, 0], pv[1, 0]) == (2, 237)
    assert s[1, 0] == pytest.approx(np.sqrt(1.5), rel=1e-14)
    # w = 1: mean 107.5, sum of squared deviations 12805 over N = 4
    assert s[0, 0] == pytest.approx(66.5 / np.sqrt(12805 / 4), rel=1e-14)


def test_snr_constant_series_is_zero():
    s, pt, pv = oracle.snr(np.full((2, 50), 7, np.int32), [1, 5, 50])
    assert np.all(s == 0) and np.all(pt == 0)
    assert pv[:, 0].tolist() == [7, 35, 350]


@pytest.mark.parametrize("n,h,w", [(100, 1, 1), (4096, 255, 1), (1000, 12345, 4)])
def test_snr_single_spike_closed_form(n, h, w):
    # A spike of height h on zeros: every width-w boxcar that covers it equals h,
    # so with N = n - w + 1 valid samples and w of them at h the S/N is
    # (1 - w/N) / sqrt(w/N (1 - w/N)) = sqrt((N - w) / w), independent of h.
    D = np.zeros((1, n), np.int32)
    D[0, n // 2] = h
    s, pt, pv = oracle.snr(D, [w])
    N = n - w + 1
    assert s[0, 0] == pytest.approx(np.sqrt((N - w) / w), rel=1e-12)
    assert pt[0, 0] == n // 2 - w + 1 and pv[0, 0] == h


def test_snr_against_numpy_population_std():
    D = _rng(9).integers(0, 391680, (5, 777)).astype(np.int32)
    widths = [1, 3, 16, 64]
    s, pt, pv = oracle.snr(D, widths)
    for wi, w in enumerate(widths):
        for i in range(5):
            B = np.convolve(D[i].astype(np.int64), np.ones(w, np.int64), "valid").astype(np.float64)
            assert s[wi, i] == pytest.approx((B.max() - B.mean()) / B.std(ddof=0), rel=1e-12)
            assert pt[wi, i] == int(np.argmax(B)) and pv[wi, i] == int(B.max())


def test_peak_ties_take_the_first_sample():
    D = np.array([[0, 9, 1, 9, 0, 9]], np.int32)
    s, pt, pv = oracle.snr(D, [1])
    assert (pt[0, 0], pv[0, 0]) == (1, 9)


def test_detect_tie_break():
    s = np.zeros((3, 4))
    s[2, 1] = s[1, 3] = s[0, 3] = 5.0
    assert oracle.detect(s) == (1, 2)
    s[1, 1] = 5.0
    assert oracle.detect(s) == (1, 1)




def test_snr_values_order_like_their_bit_patterns():
    """The detection compares S/N values by their IEEE-754 bit patterns read as
    signed 64-bit integers.  That ordering equals the values' own ordering
    exactly when every value is a finite double >= +0, which the definition
    guarantees (the peak is never below the mean; a constant series gives 0).
    Checked on the oracle's S/N of random rows, constant rows and single spikes,
    and on values one ulp apart."""
    rng = np.random.default_rng(11)
    D = rng.integers(0, 391681, size=(40, 300), dtype=np.int64).astype(np.int32)
    D[3] = 7
    D[5] = 0
    D[8, 150] = 391680
    s, _, _ = oracle.snr(D, [1, 2, 4, 8, 300])
    v = s.ravel()
    assert np.all(np.isfinite(v)) and np.all(v >= 0.0) and not np.any(np.signbit(v))
    k = v.view(np.int64)
    assert np.array_equal(np.argsort(v, kind="stable"), np.argsort(k, kind="stable"))
    near = np.array([0.0, 5e-324, 1.0, np.nextafter(1.0, 2.0), 28.97, np.nextafter(28.97, 0.0)])
    for a in near:
        for b in near:
            assert (a > b) == (np.float64(a).view(np.int64) > np.float64(b).view(np.int64))


# ----------------------------------------------------------------------------- RFI zapping, downsampling
def test_zapping_is_linear_in_the_channel_set():
    """Zapped + zapped-only de-dispersions add up to the full one; zapping every
    channel gives zeros (Sec. 2 footnote: zapped channels are left out)."""
    rng = np.random.Generator(np.random.PCG64(41))
    C, n_t = 12, 40
    d = rng.integers(0, 9, size=(5, C)).astype(np.int32)
    x = rng.integers(0, 256, size=(C, n_t + 9)).astype(np.uint8)
    m = rng.integers(0, 2, size=C).astype(np.uint8)
    a = oracle.dedisperse(oracle.zap_channels(x, m), d, n_t)
    b = oracle.dedisperse(oracle.zap_channels(x, 1 - m), d, n_t)
    assert np.array_equal(a.astype(np.int64) + b, oracle.dedisperse(x, d, n_t))
    assert not oracle.dedisperse(oracle.zap_channels(x, np.ones(C)), d, n_t).any()


@pytest.mark.parametrize("f", [1, 2, 3, 7, 10, 40])
def test_decimated_series_is_the_boxcar_at_stride_f(f):
    """X_f[j] = B_f[j f]: decimation samples the sliding boxcar (an independent
    code path, the C boxcar) at multiples of f; the trailing partial window is
    dropped, so the sums telescope to the first (n_t // f) f samples."""
    rng = np.random.Generator(np.random.PCG64(f))
    D = rng.integers(0, 5000, size=(4, 97)).astype(np.int32)
    X = oracle.decimate(D, f)
    n = 97 // f
    assert X.shape == (4, n)
    for i in range(4):
        assert np.array_equal(X[i], oracle.boxcar(D[i], f)[::f][:n])
    assert np.array_equal(X.sum(axis=1), D[:, :n * f].astype(np.int64).sum(axis=1))


@pytest.mark.parametrize("f,t0", [(1, 0), (4, 13), (10, 99), (7, 96), (7, 99)])
def test_decimated_snr_single_spike_closed_form(f, t0):
    """One spike of height h in a zero series: one non-zero bin among N = n_t // f,
    so S/N = sqrt(N - 1) whatever h, at peak_t = f * (t0 // f)."""
    n_t, h = 100, 777
    D = np.zeros((1, n_t), np.int32)
    D[0, t0] = h
    s, pt, pv = oracle.snr_decimated(D, [f])
    N = n_t // f
    if t0 < N * f:
        assert s[0, 0] == pytest.approx(np.sqrt(N - 1), rel=1e-12)
        assert pt[0, 0] == f * (t0 // f) and pv[0, 0] == h
    else:  # the spike falls in the dropped tail: a constant (zero) series
        assert s[0, 0] == 0.0 and pv[0, 0] == 0
