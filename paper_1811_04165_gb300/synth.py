"""Seeded synthetic inputs: uint8 filterbanks with injected dispersed pulses.

This module is shared by the tests, ``bench.py`` and the smoke check.  It
simulates the sky and the digitiser only; it holds none of the search's own
arithmetic (no integer delay tables, no sums over channels, no boxcars, no
S/N).  A pulse is modelled in continuous time: its leading edge reaches the
centre frequency f of a channel k_DM * DM * (f^-2 - f_top^-2) / t_samp samples
after it reaches the top channel, it lasts ``width`` samples, and each sample
bin receives the amplitude times the fraction of the bin the pulse covers.
Noise is Gaussian (mean 128, sd 16) from numpy's PCG64; the sum is rounded and
clipped to 0..255.  The paper's own test data were generated noise with an
injected single pulse (Sec. 4), so no dataset is needed.

The named workloads below are the shapes the library is measured and checked
on: a tiny 64-channel search and one Apertif-shaped 1536-channel beam
(Table 2: 1536 channels of 0.1953125 MHz, 32 subbands; 1.024 s batches).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

K_DM_PHYS = 4.148808e3  # s MHz^2 pc^-1 cm^3 (cold-plasma dispersion law)


@dataclass(frozen=True)
class Pulse:
    dm: float        # pc cm^-3
    width: float     # samples
    amp: float       # digitiser units added per fully covered channel-sample
    t0: float        # arrival of the leading edge at the top channel, in samples


@dataclass
class Workload:
    name: str
    channels: int
    f_lo: float
    f_hi: float
    t_samp: float
    n_t: int
    dms: np.ndarray
    widths: np.ndarray
    seed: int
    pulses: list = field(default_factory=list)
    n_subbands: int = 0
    coarse_dms: np.ndarray | None = None
    smoothing: int = 0                 # 0 sliding boxcars, 1 decimating downsampling
    zap: np.ndarray | None = None      # per-channel RFI flags (non-zero = zapped)

    @property
    def dm_trial_samples(self) -> int:
        return int(self.dms.size) * int(self.n_t)


def dm_grid(n: int, step: float, first: float = 0.0) -> np.ndarray:
    """DM trials first + step * i, i < n, each computed directly (no running sum)."""
    return first + step * np.arange(n, dtype=np.float64)


def pulse_amplitude(snr: float, channels: int, width: float, sd: float = 16.0) -> float:
    """Per channel-sample amplitude that gives a matched-filter S/N of ``snr``."""
    return snr * sd / np.sqrt(channels * width)


def _centre_freqs(f_lo: float, f_hi: float, channels: int) -> np.ndarray:
    return f_lo + (np.arange(channels) + 0.5) * ((f_hi - f_lo) / channels)


def filterbank(channels: int, f_lo: float, f_hi: float, t_samp: float, n_in: int, seed: int,
               pulses=(), pitch: int | None = None, mean: float = 128.0,
               sd: float = 16.0) -> np.ndarray:
    """uint8 [channels, pitch] channel-major filterbank; samples >= n_in are 0."""
    if pitch is None:
        pitch = (n_in + 15) // 16 * 16
    if pitch < n_in:
        raise ValueError("pitch < n_in")
    rng = np.random.Generator(np.random.PCG64(seed))
    sky = rng.standard_normal((channels, n_in), dtype=np.float32)
    sky *= np.float32(sd)
    sky += np.float32(mean)
    if pulses:
        f = _centre_freqs(f_lo, f_hi, channels)
        inv_top = 1.0 / (f[-1] * f[-1])
        for p in pulses:
            lead = p.t0 + K_DM_PHYS * p.dm * (1.0 / (f * f) - inv_top) / t_samp
            for c in range(channels):
                a, b = lead[c], lead[c] + p.width
                j0, j1 = int(np.floor(a)), int(np.ceil(b))
                if j1 <= 0 or j0 >= n_in:
                    continue
                j = np.arange(max(j0, 0), min(j1, n_in))
                cover = np.minimum(j + 1.0, b) - np.maximum(j * 1.0, a)
                sky[c, j] += np.float32(p.amp) * cover.astype(np.float32)
    out = np.zeros((channels, pitch), np.uint8)
    np.clip(np.rint(sky), 0, 255, out=sky)
    out[:, :n_in] = sky.astype(np.uint8)
    return out


def tiny_brute() -> Workload:
    """64 channels over 1250-1550 MHz, 81.92 us, 4096 samples; 32 DMs 0..62 step 2;
    widths {1,2,4,8}; one pulse at DM 50, width 4, 3 sd per channel-sample."""
    return Workload("tiny-64ch-4096s-32dm", 64, 1250.0, 1550.0, 81.92e-6, 4096,
                    dm_grid(32, 2.0), np.array([1, 2, 4, 8], np.int32), seed=1,
                    pulses=[Pulse(50.0, 4.0, 48.0, 1024.0)])


def apertif_beam(seed: int = 2, subband: bool = False) -> Workload:
    """One Apertif-shaped beam: 1536 channels of 0.1953125 MHz over 1250-1550 MHz,
    81.92 us, a 1.024 s batch of 12500 samples; 2048 DMs 0..409.4 step 0.2;
    widths 1..64 (powers of two); five pulses with DM in U(10, 400), widths in
    {1,..,32}, S/N in U(6, 20), one per fifth of the batch.  With ``subband`` the
    two-step path uses 32 subbands and 64 coarse DMs (the first fine DM of each
    group of 32)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    n_t, channels = 12500, 1536
    pulses = []
    slot = (n_t - 64) / 5.0
    for k in range(5):
        dm = float(rng.uniform(10.0, 400.0))
        w = float(2 ** int(rng.integers(0, 6)))
        snr = float(rng.uniform(6.0, 20.0))
        t0 = float(np.floor(k * slot + rng.uniform(0.0, slot - 64.0)))
        pulses.append(Pulse(dm, w, pulse_amplitude(snr, channels, w), t0))
    dms = dm_grid(2048, 0.2)
    wl = Workload("apertif-1536ch-12500s-2048dm", channels, 1250.0, 1550.0, 81.92e-6, n_t, dms,
                  np.array([1, 2, 4, 8, 16, 32, 64], np.int32), seed=seed, pulses=pulses)
    if subband:
        wl.name += "-subband32"
        wl.n_subbands = 32
        wl.coarse_dms = dms[::32].copy()
    return wl


def batch_beams(n_beams: int = 40, seed: int = 4, n_t: int = 12500, channels=(1536, 384),
                dm_trials=(512, 4096), dm_steps=(0.1, 0.5), max_widths: int = 7) -> list:
    """Beams for one batch: alternately ``channels[0]`` and ``channels[1]``
    channels over 1250-1550 MHz, 81.92 us, ``n_t`` samples; per beam a DM count
    uniform in ``dm_trials`` (a multiple of 32), a step uniform in ``dm_steps``
    (0.01 resolution), the first 1..``max_widths`` widths of 1, 2, 4, ..., 64,
    and two pulses (DM within the beam's range, width 2^U{0..5}, S/N U(8, 20))."""
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    out = []
    for b in range(n_beams):
        ch = int(channels[b % len(channels)])
        n_dm = int(rng.integers(dm_trials[0] // 32, dm_trials[1] // 32 + 1)) * 32
        step = round(float(rng.uniform(*dm_steps)), 2)
        k = int(rng.integers(1, max_widths + 1))
        widths = np.array([2 ** i for i in range(k)], np.int32)
        dms = dm_grid(n_dm, step)
        pulses = []
        for _ in range(2):
            dm = float(rng.uniform(0.05, 0.9) * dms[-1])
            w = float(2 ** int(rng.integers(0, 6)))
            snr = float(rng.uniform(8.0, 20.0))
            t0 = float(np.floor(rng.uniform(0.0, n_t - 64.0)))
            pulses.append(Pulse(dm, w, pulse_amplitude(snr, ch, w), t0))
        out.append(Workload(f"beam{b}-{ch}ch-{n_t}s-{n_dm}dm-step{step}", ch, 1250.0, 1550.0, 81.92e-6, n_t, dms,
                            widths, seed=seed * 1000 + b, pulses=pulses))
    return out
