"""The oracle's pins must catch plausible mistakes.

Each case below plants one slip in a temporary copy of the oracle's C source
(on the CPU; the real oracle is untouched), compiles it, binds it in place of
the real library and runs the pin suite: at least one pin must fail.
"""
import ctypes
import inspect
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sps_oracle.c")

MUTANTS = {
    "delay sign flipped": ("(inv_f - inv_r)", "(inv_r - inv_f)"),
    "channel edge instead of centre": ("((double)c + 0.5) * df", "((double)c) * df"),
    "bottom channel as reference": (
        "double f_ref = oracle_channel_freq(f_lo, f_hi, channels, channels - 1);\n  for (int32_t c = 0; c < channels; c++) {\n    double kc",
        "double f_ref = oracle_channel_freq(f_lo, f_hi, channels, 0);\n  for (int32_t c = 0; c < channels; c++) {\n    double kc"),
    "delays truncated": ("(int32_t)llround(dms[i] * kc)", "(int32_t)(dms[i] * kc)"),
    "first channel dropped": (
        "for (int32_t c = 0; c < channels; c++) {\n      const uint8_t* xr",
        "for (int32_t c = 1; c < channels; c++) {\n      const uint8_t* xr"),
    "delay table transposed": ("d[(int64_t)i * channels + c];\n      for", "d[(int64_t)c * n_dms + i];\n      for"),
    "subband ref at its bottom channel": (
        "double f_top = oracle_channel_freq(f_lo, f_hi, channels, (s + 1) * per - 1);\n    double k1",
        "double f_top = oracle_channel_freq(f_lo, f_hi, channels, s * per);\n    double k1"),
    "step two with the fine offset only": ("(int32_t)llround(dms[i] * k2)",
                                           "(int32_t)llround((dms[i] - coarse_dms[0]) * k2 * 0.5)"),
    "step two reads the wrong coarse row": ("((int64_t)coarse_of[i] * n_subbands + s)",
                                            "((int64_t)(coarse_of[i] > 0 ? coarse_of[i] - 1 : 0) * n_subbands + s)"),
    "boxcar one short": ("for (int32_t u = 0; u < w; u++) s += D[t + u];",
                         "for (int32_t u = 0; u + 1 < w; u++) s += D[t + u];"),
    "sample sigma": ("sqrt(ss / (double)N)", "sqrt(ss / (double)(N - 1))"),
    "last peak on ties": ("if (B[t] > pv)", "if (B[t] >= pv)"),
    "valid length off by one": ("int32_t N = n_t - w + 1;", "int32_t N = n_t - w;"),
    "detect prefers later DMs": ("if (v > best)", "if (v >= best)"),
}


def _pin_tests():
    out = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        marks = getattr(fn, "pytestmark", [])
        params = [m for m in marks if m.name == "parametrize"]
        if params:
            argnames, values = params[0].args[0], params[0].args[1]
            argnames = [a.strip() for a in argnames.split(",")]
            for v in values:
                v = v if isinstance(v, tuple) else (v,)
                out.append((name, fn, dict(zip(argnames, v))))
        else:
            out.append((name, fn, {}))
    return out


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant, tmp_path):
    old, new = MUTANTS[mutant]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {mutant!r} not unique"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(path), "-lm"])
    saved = oracle._load()
    oracle._lib = oracle._bind(ctypes.CDLL(str(so)))
    failed = []
    try:
        for name, fn, kw in _pin_tests():
            if name == "test_injected_pulse_recovered_apertif_strongest":
                continue
            try:
                fn(**kw) if "tmp_path" not in inspect.signature(fn).parameters else fn(tmp_path=tmp_path, **kw)
            except Exception:  # an assertion or an out-of-range check in the wrapper
                failed.append(name)
                break
    finally:
        oracle._lib = saved
    assert failed, f"no pin caught the planted mistake {mutant!r}"
