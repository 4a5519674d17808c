"""The C ABI without a GPU: the library loads, exports every symbol the headers
declare, and rejects bad descriptors with the documented status codes."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(sps_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = _declared()
    for required in ("sps_plan_create", "sps_dedisperse", "sps_integrate", "sps_snr", "sps_search",
                     "sps_search_host", "sps_subband_step1", "sps_subband_step2"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    L = ctypes.CDLL(lib.lib_path())
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(lib):
    from paper_1811_04165_gb300 import _lib
    assert set(_declared()) <= set(_lib.SIGNATURES)


def test_status_strings(lib):
    L = lib.lib()
    assert L.sps_status_string(0) == b"ok"
    assert L.sps_status_string(6) == b"no device"
    assert L.sps_abi_version() >= 100


def _desc(lib, **over):
    dms = np.asarray(over.pop("dms", np.arange(8) * 1.0), np.float64)
    widths = np.asarray(over.pop("widths", [1, 2]), np.int32)
    d = lib.PlanDesc()
    d.channels, d.f_lo_mhz, d.f_hi_mhz, d.t_samp_s, d.n_samples = 16, 1250.0, 1550.0, 81.92e-6, 100
    d.dms, d.n_dms = dms.ctypes.data, dms.size
    d.widths, d.n_widths = widths.ctypes.data, widths.size
    for k, v in over.items():
        setattr(d, k, v)
    return d, (dms, widths)


@pytest.mark.parametrize("over,status", [
    ({"channels": 0}, 1), ({"f_hi_mhz": 1000.0}, 1), ({"t_samp_s": 0.0}, 1), ({"n_samples": 0}, 1),
    ({"dms": [3.0, 1.0]}, 1), ({"dms": [-1.0]}, 1), ({"widths": [0]}, 1), ({"widths": [2, 2]}, 1),
    ({"widths": [101]}, 1), ({"mode": 7}, 1),
])
def test_bad_descriptors_rejected_before_device_use(lib, over, status):
    d, keep = _desc(lib, **over)
    h = ctypes.c_void_p()
    assert lib.lib().sps_plan_create(ctypes.byref(d), ctypes.byref(h)) == status
    assert not h.value
    assert lib.lib().sps_last_error()


def test_null_arguments(lib):
    L = lib.lib()
    assert L.sps_plan_create(None, None) == 1
    assert L.sps_dedisperse(None, None, 0, None, None, 0, None) == 1
    assert L.sps_snr(None, None, None, None, None, None, None) == 1
    assert L.sps_plan_destroy(None) == 0
    assert L.sps_plan_input_samples(None) == -1


def test_valid_descriptor_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    d, keep = _desc(lib)
    h = ctypes.c_void_p()
    assert lib.lib().sps_plan_create(ctypes.byref(d), ctypes.byref(h)) == 6  # SPS_ERR_NO_DEVICE


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1811_04165_gb300 import _lib
    monkeypatch.setattr(_lib, "_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.lib()


def test_binding_checks_host_array_lengths(lib):
    """Arrays the library reads by count from the descriptor are checked for
    length in the binding first (a short array would be read past its end)."""
    with pytest.raises(ValueError):
        lib.sps_plan_create(16, 1250.0, 1550.0, 81.92e-6, 100, [0.0, 1.0, 2.0, 3.0], [1], mode=lib.MODE_SUBBAND,
                            n_subbands=4, coarse_dms=[0.0, 2.0], coarse_of=[0, 0, 1])
    with pytest.raises(ValueError):
        lib.sps_plan_create(16, 1250.0, 1550.0, 81.92e-6, 100, [0.0], [1], zap=[0] * 15)
