"""CPU oracle for the single-pulse-search hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never imports it and shares no code with it.

The arithmetic lives in plain C (``sps_oracle.c``, FP64, no FMA contraction);
this module compiles it on first use with gcc and wraps it with numpy.  The GA
tuner's oracle is pure Python in ``ga.py``.

What each function computes, and the paper passage it follows (Mikhailov &
Sclocco, AMBER auto-tuning with genetic algorithms):
  channel_freqs      Table 2 (MIN_FREQ, CHANNEL_BANDWIDTH); centres, ascending
  delay_table        Sec. 1 ("shift" of channels); k_DM dispersion law
  subband_tables     Sec. 2, first footnote; Table 2 SUBBANDS / DM grid
  dedisperse         Sec. 1 and the one-step path of Sec. 5
  subband_step1/2    Sec. 2, first footnote (two-step de-dispersion)
  boxcar             Sec. 2 "downsampling (smoothing)", as a sliding boxcar
  snr                Sec. 2 S/N step; (peak - mean) / population sigma
  detect             argmax over (DM, width) of the S/N table
  zap_channels       Sec. 2, footnote: channels zapped for terrestrial RFI
  decimate           Table 2 DOWNSAMPLING / NRSAMPLES: decimating downsampling
  snr_decimated      Sec. 2 S/N, Sec. 5: on every downsampled series (factor 1 =
                     the series itself)

Parity pins for every function are in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sps_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

K_DM = 4.148808e3  # s MHz^2 pc^-1 cm^3


def build(force: bool = False) -> str:
    """Compile the oracle's C source into liboracle.so (gcc, -O2, no FMA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    p = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.oracle_channel_freq.restype = f64
    lib.oracle_channel_freq.argtypes = [f64, f64, i32, i32]
    lib.oracle_delay_table.restype = None
    lib.oracle_delay_table.argtypes = [f64, f64, i32, f64, p, i32, p]
    lib.oracle_subband_tables.restype = None
    lib.oracle_subband_tables.argtypes = [f64, f64, i32, f64, i32, p, i32, p, i32, p, p]
    lib.oracle_dedisperse.restype = None
    lib.oracle_dedisperse.argtypes = [p, i64, i32, i32, p, i32, p]
    lib.oracle_subband_step1.restype = None
    lib.oracle_subband_step1.argtypes = [p, i64, i32, i32, i32, p, i32, p]
    lib.oracle_subband_step2.restype = None
    lib.oracle_subband_step2.argtypes = [p, i32, i32, i32, p, p, i32, i32, p]
    lib.oracle_boxcar.restype = None
    lib.oracle_boxcar.argtypes = [p, i32, i32, p]
    lib.oracle_snr.restype = None
    lib.oracle_snr.argtypes = [p, i32, i32, p, i32, p, p, p]
    lib.oracle_detect.restype = None
    lib.oracle_detect.argtypes = [p, i32, i32, p, p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def channel_freqs(f_lo: float, f_hi: float, channels: int) -> np.ndarray:
    """Channel centre frequencies in MHz, channel 0 lowest (Table 2 reading)."""
    lib = _load()
    return np.array([lib.oracle_channel_freq(f_lo, f_hi, channels, c) for c in range(channels)])


def delay_table(f_lo, f_hi, channels, t_samp, dms) -> np.ndarray:
    """int32 [n_dms, channels]: round-half-away(DM * k_DM (f^-2 - f_ref^-2) / t_samp)."""
    lib = _load()
    dms = _c(dms, np.float64)
    d = np.empty((dms.size, channels), np.int32)
    lib.oracle_delay_table(f_lo, f_hi, channels, t_samp, _ptr(dms), dms.size, _ptr(d))
    return d


def subband_tables(f_lo, f_hi, channels, t_samp, n_subbands, coarse_dms, dms):
    """(d1 int32 [n_coarse, channels], d2 int32 [n_dms, n_subbands])."""
    if channels % n_subbands:
        raise ValueError("subbands must divide channels")
    lib = _load()
    coarse = _c(coarse_dms, np.float64)
    dms = _c(dms, np.float64)
    d1 = np.empty((coarse.size, channels), np.int32)
    d2 = np.empty((dms.size, n_subbands), np.int32)
    lib.oracle_subband_tables(f_lo, f_hi, channels, t_samp, n_subbands, _ptr(coarse), coarse.size,
                              _ptr(dms), dms.size, _ptr(d1), _ptr(d2))
    return d1, d2


def _check_x(x: np.ndarray, n_needed: int):
    if x.dtype != np.uint8 or x.ndim != 2:
        raise ValueError("x must be a 2-D uint8 array [channels, samples]")
    if x.shape[1] < n_needed:
        raise ValueError(f"x has {x.shape[1]} samples per channel, needs {n_needed}")
    if x.strides[1] != 1:
        raise ValueError("x rows must be contiguous")


def dedisperse(x: np.ndarray, delays: np.ndarray, n_t: int) -> np.ndarray:
    """int32 [n_dms, n_t]: D[i, t] = sum_c x[c, t + delays[i, c]]."""
    lib = _load()
    delays = _c(delays, np.int32)
    n_dms, channels = delays.shape
    if x.shape[0] != channels:
        raise ValueError("channel count mismatch")
    if delays.size and delays.min() < 0:
        raise ValueError("negative delay")
    _check_x(x, n_t + (int(delays.max()) if delays.size else 0))
    out = np.empty((n_dms, n_t), np.int32)
    lib.oracle_dedisperse(_ptr(x), x.strides[0], channels, n_t, _ptr(delays), n_dms, _ptr(out))
    return out


def subband_step1(x: np.ndarray, d1: np.ndarray, n_subbands: int, n_1: int) -> np.ndarray:
    """int32 [n_coarse, n_subbands, n_1]: Y[k, s, t] = sum_{c in s} x[c, t + d1[k, c]]."""
    lib = _load()
    d1 = _c(d1, np.int32)
    n_coarse, channels = d1.shape
    _check_x(x, n_1 + int(d1.max()))
    y = np.empty((n_coarse, n_subbands, n_1), np.int32)
    lib.oracle_subband_step1(_ptr(x), x.strides[0], channels, n_subbands, n_1, _ptr(d1), n_coarse,
                             _ptr(y))
    return y


def subband_step2(y: np.ndarray, d2: np.ndarray, coarse_of: np.ndarray, n_t: int) -> np.ndarray:
    """int32 [n_dms, n_t]: D[i, t] = sum_s Y[k(i), s, t + d2[i, s]]."""
    lib = _load()
    y = _c(y, np.int32)
    d2 = _c(d2, np.int32)
    coarse_of = _c(coarse_of, np.int32)
    n_coarse, n_subbands, n_1 = y.shape
    if n_t + int(d2.max()) > n_1:
        raise ValueError("Y rows too short for the step-two delays")
    out = np.empty((d2.shape[0], n_t), np.int32)
    lib.oracle_subband_step2(_ptr(y), n_coarse, n_subbands, n_1, _ptr(d2), _ptr(coarse_of),
                             d2.shape[0], n_t, _ptr(out))
    return out


def boxcar(series: np.ndarray, w: int) -> np.ndarray:
    """int32 [n_t - w + 1]: B[t] = sum_{u<w} D[t + u] (valid part only)."""
    lib = _load()
    series = _c(series, np.int32)
    n_t = series.size
    if not 1 <= w <= n_t:
        raise ValueError("width out of range")
    out = np.empty(n_t - w + 1, np.int32)
    lib.oracle_boxcar(_ptr(series), n_t, w, _ptr(out))
    return out


def snr(D: np.ndarray, widths) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """S/N, peak sample and peak value per (width, DM), each laid out [n_w, n_dms]."""
    lib = _load()
    D = _c(D, np.int32)
    widths = _c(widths, np.int32)
    n_dms, n_t = D.shape
    if widths.size == 0 or widths.min() < 1 or widths.max() > n_t:
        raise ValueError("widths must lie in [1, n_t]")
    s = np.empty((widths.size, n_dms), np.float64)
    pt = np.empty((widths.size, n_dms), np.int32)
    pv = np.empty((widths.size, n_dms), np.int32)
    lib.oracle_snr(_ptr(D), n_dms, n_t, _ptr(widths), widths.size, _ptr(s), _ptr(pt), _ptr(pv))
    return s, pt, pv


def detect(snr_table: np.ndarray) -> tuple[int, int]:
    """(DM index, width index) of the largest S/N; ties -> smaller DM, then width."""
    lib = _load()
    s = _c(snr_table, np.float64)
    n_w, n_dms = s.shape
    bi, bw = ctypes.c_int32(), ctypes.c_int32()
    lib.oracle_detect(_ptr(s), n_dms, n_w, ctypes.byref(bi), ctypes.byref(bw))
    return bi.value, bw.value


def zap_channels(x: np.ndarray, zap) -> np.ndarray:
    """x with every zapped channel's row set to 0 (zap: one flag per channel,
    non-zero = zapped): such channels add nothing to any sum."""
    out = np.array(x, copy=True)
    out[np.asarray(zap).astype(bool)] = 0
    return out


def decimate(D: np.ndarray, f: int) -> np.ndarray:
    """Downsampling by factor f: X[i][j] = sum_{u<f} D[i][j * f + u] for
    j < n_t // f (the trailing n_t mod f samples form no sample), int64."""
    D = np.asarray(D)
    if not 1 <= f <= D.shape[1]:
        raise ValueError("factor out of range")
    n = D.shape[1] // f
    return D[:, :n * f].astype(np.int64).reshape(D.shape[0], n, f).sum(axis=2)


def snr_decimated(D: np.ndarray, factors) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """S/N of every downsampled series, laid out [n_factors, n_dms]: for factor
    f, (max X - mean X) / population sigma over the n_t // f samples of
    X = decimate(D, f); peak_t = f * (first j with X[j] = max), in input
    samples; peak_val = max X."""
    D = np.asarray(D)
    factors = [int(f) for f in factors]
    s = np.empty((len(factors), D.shape[0]), np.float64)
    pt = np.empty((len(factors), D.shape[0]), np.int32)
    pv = np.empty((len(factors), D.shape[0]), np.int32)
    for k, f in enumerate(factors):
        X = decimate(D, f)
        if X.size and (X.max() > np.iinfo(np.int32).max or X.min() < 0):
            raise ValueError("downsampled sums outside [0, 2^31)")
        sk, ptk, pvk = snr(X.astype(np.int32), [1])
        s[k], pt[k], pv[k] = sk[0], ptk[0] * f, pvk[0]
    return s, pt, pv


def coarse_index(n_dms: int, n_coarse: int) -> np.ndarray:
    """Default fine-to-coarse DM map k(i) = floor(i / (n_dms / n_coarse))."""
    if n_dms % n_coarse:
        raise ValueError("n_coarse must divide n_dms")
    return (np.arange(n_dms) // (n_dms // n_coarse)).astype(np.int32)


def subband_lengths(n_t: int, d1: np.ndarray, d2: np.ndarray) -> tuple[int, int]:
    """(n_1, n_in) for the two-step path: n_1 = n_t + max d2, n_in = n_1 + max d1."""
    n_1 = n_t + int(d2.max())
    return n_1, n_1 + int(d1.max())


def search_brute(x, f_lo, f_hi, t_samp, dms, widths, n_t):
    """Whole one-step path: delays -> D -> (snr, peak_t, peak_val, (dm, w))."""
    d = delay_table(f_lo, f_hi, x.shape[0], t_samp, dms)
    D = dedisperse(x, d, n_t)
    s, pt, pv = snr(D, widths)
    return D, s, pt, pv, detect(s)
