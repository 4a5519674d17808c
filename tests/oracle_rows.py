"""The oracle over whole tables at once, for full-size parity tests: independent
rows (DM trials, coarse DMs) are split into contiguous parts run on host
threads.  The oracle's C routines release the interpreter lock and each row is
computed on its own, so the result is exactly that of one call."""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


def host_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return os.cpu_count() or 1


def _split(n: int, threads: int | None):
    threads = threads or host_threads()
    return [p for p in np.array_split(np.arange(n), min(threads, max(n, 1))) if p.size]


def _run(fn, parts):
    with ThreadPoolExecutor(len(parts)) as ex:
        return list(ex.map(fn, parts))


def dedisperse(x: np.ndarray, delays: np.ndarray, n_t: int, threads: int | None = None) -> np.ndarray:
    """oracle.dedisperse over every row of `delays`."""
    parts = _split(delays.shape[0], threads)
    return np.concatenate(_run(lambda p: oracle.dedisperse(x, delays[p], n_t), parts), axis=0)


def snr(D: np.ndarray, widths, threads: int | None = None):
    """oracle.snr over every DM row of D: (snr, peak_t, peak_val), [n_w, n_dms]."""
    parts = _split(D.shape[0], threads)
    res = _run(lambda p: oracle.snr(D[p], widths), parts)
    return tuple(np.concatenate([r[k] for r in res], axis=1) for k in range(3))


def snr_decimated(D: np.ndarray, factors, threads: int | None = None):
    """oracle.snr_decimated over every DM row of D."""
    parts = _split(D.shape[0], threads)
    res = _run(lambda p: oracle.snr_decimated(D[p], factors), parts)
    return tuple(np.concatenate([r[k] for r in res], axis=1) for k in range(3))


def subband_step1(x: np.ndarray, d1: np.ndarray, n_subbands: int, n_1: int, threads: int | None = None):
    """oracle.subband_step1 over every coarse DM of d1: Y [n_coarse, S, n_1]."""
    parts = _split(d1.shape[0], threads)
    return np.concatenate(_run(lambda p: oracle.subband_step1(x, d1[p], n_subbands, n_1), parts), axis=0)


def subband_step2(Y: np.ndarray, d2: np.ndarray, coarse_of: np.ndarray, n_t: int, threads: int | None = None):
    """oracle.subband_step2 over every DM trial of d2."""
    parts = _split(d2.shape[0], threads)
    return np.concatenate(_run(lambda p: oracle.subband_step2(Y, d2[p], coarse_of[p], n_t), parts), axis=0)
