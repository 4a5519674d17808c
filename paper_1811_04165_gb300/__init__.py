"""GB300 single-pulse search: the hot path of the AMBER pipeline as hand-written
sm_103a CUDA behind a C ABI (``include/sps.h``, ``libsps.so``).

This module is a thin ctypes binding: it checks tensors and passes raw device
pointers and the current CUDA stream to the library.  Every step of the path
runs in the library's kernels; there is no CPU fallback, and importing the
binding's first call fails loudly (ImportError) when ``libsps.so`` has not been
built.

Functions carry the C names (``sps_plan_create`` ... ``sps_search_host``);
:class:`Plan` wraps a plan handle.  Shapes follow the C ABI:
  x        uint8  [channels, pitch]   pitch >= plan.input_samples, pitch % 16 == 0
  D        int32  [n_dms, n_samples]
  Y        uint16 [n_coarse, n_subbands, y_pitch]   (subband step one)
  B        int32  [n_widths, n_dms, n_samples]
  snr      float64 [n_widths, n_dms]; peak_t, peak_val int32 [n_widths, n_dms]
  best     int32  [4] = (DM index, width index, peak_t, peak_val)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from ._lib import SpsError, check, lib, lib_path  # noqa: F401

MODE_BRUTE = 0
MODE_SUBBAND = 1
SPS_OK, SPS_ERR_INVALID_ARG, SPS_ERR_UNSUPPORTED, SPS_ERR_CUDA, SPS_ERR_OOM, SPS_ERR_TIMEOUT = 0, 1, 2, 3, 4, 5
# bits of the plan's device status word (Plan.status)
STATUS_WAIT_TIMEOUT = 1   # a kernel's bounded wait ran out
STATUS_BOUNDS = 2         # bounds-checked build: a staged read would have left its stage
SMOOTH_SLIDING = 0
SMOOTH_DECIMATE = 1


class DedispConfig(ctypes.Structure):
    _fields_ = [("dms_per_thread", ctypes.c_int32), ("samples_per_thread", ctypes.c_int32),
                ("warps_dm", ctypes.c_int32), ("warps_time", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("presum", ctypes.c_int32)]

    def as_tuple(self):
        return tuple(getattr(self, f) for f, _ in self._fields_)


class SnrConfig(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32)]

    def as_tuple(self):
        return (self.threads,)


class KernelConfig(ctypes.Structure):
    _fields_ = [("brute", DedispConfig), ("step1", DedispConfig), ("step2", DedispConfig),
                ("snr", SnrConfig)]

    def as_dict(self):
        return {k: getattr(self, k).as_tuple() for k, _ in self._fields_}


class PlanDesc(ctypes.Structure):
    _fields_ = [("channels", ctypes.c_int32), ("f_lo_mhz", ctypes.c_double),
                ("f_hi_mhz", ctypes.c_double), ("t_samp_s", ctypes.c_double),
                ("n_samples", ctypes.c_int32), ("dms", ctypes.c_void_p), ("n_dms", ctypes.c_int32),
                ("widths", ctypes.c_void_p), ("n_widths", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("n_subbands", ctypes.c_int32), ("coarse_dms", ctypes.c_void_p),
                ("n_coarse", ctypes.c_int32), ("coarse_of", ctypes.c_void_p), ("smoothing", ctypes.c_int32),
                ("zap", ctypes.c_void_p)]


class _Lazy:
    """Resolves libsps.so on first use; raises ImportError if it was not built."""

    def __getattr__(self, name):
        return getattr(lib(), name)


_L = _Lazy()


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, name, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _xdev(plan, x, name="x"):
    """A filterbank on the device: uint8 [channels][pitch], one row per channel
    (the library reads `channels` rows of the given pitch)."""
    t = _torch()
    if not isinstance(x, t.Tensor) or x.dim() != 2 or x.shape[0] != plan.channels:
        raise ValueError(f"{name} must be a 2-D tensor with one row per channel ({plan.channels})")
    return _dev(x, t.uint8, name)


def _host(a, dtype, name, shape=None):
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != dtype or not a.is_contiguous():
            raise TypeError(f"{name} must be a contiguous CPU tensor of {dtype}")
        if shape is not None and tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"{name} must be a torch CPU tensor")


@dataclass
class _Arrays:  # keeps the descriptor's host arrays alive during sps_plan_create
    dms: np.ndarray
    widths: np.ndarray
    coarse: np.ndarray | None
    coarse_of: np.ndarray | None
    zap: np.ndarray | None = None


def sps_plan_create(channels, f_lo_mhz, f_hi_mhz, t_samp_s, n_samples, dms, widths,
                    mode=MODE_BRUTE, n_subbands=0, coarse_dms=None, coarse_of=None, smoothing=SMOOTH_SLIDING,
                    zap=None):
    arr = _Arrays(np.ascontiguousarray(dms, np.float64), np.ascontiguousarray(widths, np.int32),
                  None if coarse_dms is None else np.ascontiguousarray(coarse_dms, np.float64),
                  None if coarse_of is None else np.ascontiguousarray(coarse_of, np.int32),
                  None if zap is None else (np.asarray(zap) != 0).astype(np.uint8))
    if arr.zap is not None and arr.zap.size != int(channels):
        raise ValueError("zap needs one flag per channel")
    if arr.coarse_of is not None and arr.coarse_of.size != arr.dms.size:
        raise ValueError("coarse_of needs one coarse-DM index per DM trial")
    d = PlanDesc()
    d.channels, d.f_lo_mhz, d.f_hi_mhz, d.t_samp_s = int(channels), float(f_lo_mhz), float(f_hi_mhz), float(t_samp_s)
    d.n_samples = int(n_samples)
    d.dms, d.n_dms = arr.dms.ctypes.data, arr.dms.size
    d.widths, d.n_widths = arr.widths.ctypes.data, arr.widths.size
    d.mode, d.n_subbands = int(mode), int(n_subbands)
    d.coarse_dms = arr.coarse.ctypes.data if arr.coarse is not None else None
    d.n_coarse = arr.coarse.size if arr.coarse is not None else 0
    d.coarse_of = arr.coarse_of.ctypes.data if arr.coarse_of is not None else None
    d.smoothing = int(smoothing)
    d.zap = arr.zap.ctypes.data if arr.zap is not None else None
    h = ctypes.c_void_p()
    check(_L.sps_plan_create(ctypes.byref(d), ctypes.byref(h)), "sps_plan_create")
    return h


def sps_plan_destroy(h):
    check(_L.sps_plan_destroy(h), "sps_plan_destroy")


def sps_dedisperse(plan, x, D, workspace=None, stream=None):
    p = plan.handle
    if workspace is None:
        workspace = plan.workspace()
    ws = _dev(workspace, workspace.dtype, "workspace") if workspace is not None else ctypes.c_void_p()
    wsb = workspace.numel() * workspace.element_size() if workspace is not None else 0
    check(_L.sps_dedisperse(p, _xdev(plan, x), ctypes.c_int64(x.shape[1]),
                            _dev(D, _torch().int32, "D", (plan.n_dms, plan.n_samples)), ws,
                            ctypes.c_size_t(wsb), _stream(stream)), "sps_dedisperse")


def sps_dedisperse_noalloc(plan, x, D, stream=None):
    """sps_dedisperse with the library's fixed static scratch instead of a workspace
    (for callers that cannot allocate device memory; see include/sps.h)."""
    t = _torch()
    check(_L.sps_dedisperse_noalloc(plan.handle, _xdev(plan, x), ctypes.c_int64(x.shape[1]),
                                    _dev(D, t.int32, "D", (plan.n_dms, plan.n_samples)), _stream(stream)),
          "sps_dedisperse_noalloc")


def sps_subband_step1(plan, x, Y, workspace=None, stream=None):
    if workspace is None:
        workspace = plan.workspace()
    check(_L.sps_subband_step1(plan.handle, _xdev(plan, x), ctypes.c_int64(x.shape[1]),
                               _dev(Y, _torch().uint16, "Y", plan.y_shape),
                               _dev(workspace, workspace.dtype, "workspace"),
                               ctypes.c_size_t(workspace.numel() * workspace.element_size()), _stream(stream)),
          "sps_subband_step1")


def sps_subband_step2(plan, Y, D, stream=None):
    check(_L.sps_subband_step2(plan.handle, _dev(Y, _torch().uint16, "Y", plan.y_shape),
                               _dev(D, _torch().int32, "D", (plan.n_dms, plan.n_samples)),
                               _stream(stream)), "sps_subband_step2")


def sps_integrate(plan, D, B, stream=None):
    check(_L.sps_integrate(plan.handle, _dev(D, _torch().int32, "D", (plan.n_dms, plan.n_samples)),
                           _dev(B, _torch().int32, "B", (plan.n_widths, plan.n_dms, plan.n_samples)),
                           _stream(stream)), "sps_integrate")


def sps_snr(plan, D, snr, peak_t, peak_val, best=None, stream=None):
    t = _torch()
    shp = (plan.n_widths, plan.n_dms)
    check(_L.sps_snr(plan.handle, _dev(D, t.int32, "D", (plan.n_dms, plan.n_samples)),
                     _dev(snr, t.float64, "snr", shp), _dev(peak_t, t.int32, "peak_t", shp),
                     _dev(peak_val, t.int32, "peak_val", shp),
                     _dev(best, t.int32, "best", (4,)) if best is not None else ctypes.c_void_p(),
                     _stream(stream)), "sps_snr")


def sps_search(plan, x, D, snr, peak_t, peak_val, best=None, workspace=None, stream=None):
    t = _torch()
    if workspace is None:
        workspace = plan.workspace()
    shp = (plan.n_widths, plan.n_dms)
    ws = _dev(workspace, workspace.dtype, "workspace") if workspace is not None else ctypes.c_void_p()
    wsb = workspace.numel() * workspace.element_size() if workspace is not None else 0
    check(_L.sps_search(plan.handle, _xdev(plan, x), ctypes.c_int64(x.shape[1]),
                        _dev(D, t.int32, "D", (plan.n_dms, plan.n_samples)), ws, ctypes.c_size_t(wsb),
                        _dev(snr, t.float64, "snr", shp), _dev(peak_t, t.int32, "peak_t", shp),
                        _dev(peak_val, t.int32, "peak_val", shp),
                        _dev(best, t.int32, "best", (4,)) if best is not None else ctypes.c_void_p(),
                        _stream(stream)), "sps_search")


def sps_search_host(plan, x_host, x_dev, D, snr_dev, peak_t_dev, peak_val_dev, best_dev,
                    snr_host, peak_t_host, peak_val_host, best_host, workspace=None, stream=None):
    t = _torch()
    if workspace is None:
        workspace = plan.workspace()
    shp = (plan.n_widths, plan.n_dms)
    ws = _dev(workspace, workspace.dtype, "workspace") if workspace is not None else ctypes.c_void_p()
    wsb = workspace.numel() * workspace.element_size() if workspace is not None else 0
    if tuple(x_host.shape) != tuple(x_dev.shape):
        raise ValueError("x_host and x_dev must have the same shape")
    check(_L.sps_search_host(
        plan.handle, _host(x_host, t.uint8, "x_host"), ctypes.c_int64(x_dev.shape[1]),
        _xdev(plan, x_dev, "x_dev"), _dev(D, t.int32, "D", (plan.n_dms, plan.n_samples)), ws,
        ctypes.c_size_t(wsb), _dev(snr_dev, t.float64, "snr_dev", shp),
        _dev(peak_t_dev, t.int32, "peak_t_dev", shp), _dev(peak_val_dev, t.int32, "peak_val_dev", shp),
        _dev(best_dev, t.int32, "best_dev", (4,)), _host(snr_host, t.float64, "snr_host", shp),
        _host(peak_t_host, t.int32, "peak_t_host", shp), _host(peak_val_host, t.int32, "peak_val_host", shp),
        _host(best_host, t.int32, "best_host", (4,)), _stream(stream)), "sps_search_host")


def _torch():
    import torch
    return torch


class Plan:
    """A search plan (frequencies, delay tables, kernel configuration) on the current device."""

    def __init__(self, channels, f_lo_mhz, f_hi_mhz, t_samp_s, n_samples, dms, widths,
                 mode=MODE_BRUTE, n_subbands=0, coarse_dms=None, coarse_of=None, smoothing=SMOOTH_SLIDING,
                 zap=None):
        self.handle = sps_plan_create(channels, f_lo_mhz, f_hi_mhz, t_samp_s, n_samples, dms, widths,
                                      mode, n_subbands, coarse_dms, coarse_of, smoothing, zap)
        self.smoothing = int(smoothing)
        self.channels = int(channels)
        self.n_samples = int(n_samples)
        self.dms = np.asarray(dms, np.float64).copy()
        self.widths = np.asarray(widths, np.int32).copy()
        self.n_dms = self.dms.size
        self.n_widths = self.widths.size
        self.mode = int(mode)
        self.n_subbands = int(n_subbands)
        self.n_coarse = 0 if coarse_dms is None else len(coarse_dms)
        self.f_lo, self.f_hi, self.t_samp = float(f_lo_mhz), float(f_hi_mhz), float(t_samp_s)

    @classmethod
    def from_workload(cls, wl, mode=None):
        if mode is None:
            mode = MODE_SUBBAND if wl.n_subbands else MODE_BRUTE
        extra = dict(smoothing=getattr(wl, "smoothing", SMOOTH_SLIDING), zap=getattr(wl, "zap", None))
        if mode == MODE_SUBBAND:
            return cls(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_t, wl.dms, wl.widths, MODE_SUBBAND,
                       wl.n_subbands, wl.coarse_dms, **extra)
        return cls(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_t, wl.dms, wl.widths, **extra)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _L.sps_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

    @property
    def input_samples(self) -> int:
        return int(_L.sps_plan_input_samples(self.handle))

    @property
    def step1_samples(self) -> int:
        return int(_L.sps_plan_step1_samples(self.handle))

    @property
    def pitch(self) -> int:
        return (self.input_samples + 15) // 16 * 16

    @property
    def y_shape(self):
        n1 = self.step1_samples
        return (self.n_coarse, self.n_subbands, (n1 + 7) // 8 * 8)

    @property
    def workspace_bytes(self) -> int:
        n = ctypes.c_size_t()
        check(_L.sps_plan_workspace_bytes(self.handle, ctypes.byref(n)), "sps_plan_workspace_bytes")
        return int(n.value)

    def workspace(self):
        """A device workspace tensor of the required size, cached per plan and used by
        the calls that get no workspace argument: it serves one stream at a time;
        searches on several streams at once need one workspace each."""
        import torch
        n = self.workspace_bytes
        ws = getattr(self, "_ws", None)
        if ws is None or ws.numel() < n:
            ws = torch.empty(max(n, 16), dtype=torch.uint8, device="cuda")
            self._ws = ws
        return ws

    def status(self, clear: bool = True) -> int:
        """Device status word: STATUS_WAIT_TIMEOUT when a kernel's bounded wait ran
        out, STATUS_BOUNDS (bounds-checked build only) when a staged read would
        have left its stage; synchronises."""
        v = ctypes.c_uint32()
        _L.sps_plan_status(self.handle, ctypes.byref(v), int(clear))
        return int(v.value)

    def delay_table(self) -> np.ndarray:
        out = np.empty((self.n_dms, self.channels), np.int32)
        check(_L.sps_plan_delay_table(self.handle, out.ctypes.data), "sps_plan_delay_table")
        return out

    def subband_tables(self):
        d1 = np.empty((self.n_coarse, self.channels), np.int32)
        d2 = np.empty((self.n_dms, self.n_subbands), np.int32)
        check(_L.sps_plan_subband_tables(self.handle, d1.ctypes.data, d2.ctypes.data),
              "sps_plan_subband_tables")
        return d1, d2

    @property
    def config(self) -> KernelConfig:
        c = KernelConfig()
        check(_L.sps_plan_get_config(self.handle, ctypes.byref(c)), "sps_plan_get_config")
        return c

    @config.setter
    def config(self, c: KernelConfig):
        check(_L.sps_plan_set_config(self.handle, ctypes.byref(c)), "sps_plan_set_config")

    def shape_key(self) -> dict:
        """What a tuned configuration depends on: the band, sampling, DM grid and
        widths, mode and subbands (the key of a saved configuration)."""
        return {"channels": self.channels, "f_lo_mhz": self.f_lo, "f_hi_mhz": self.f_hi, "t_samp_s": self.t_samp,
                "n_samples": self.n_samples, "n_dms": self.n_dms, "dm_first": float(self.dms[0]),
                "dm_last": float(self.dms[-1]), "widths": [int(w) for w in self.widths], "mode": self.mode,
                "n_subbands": self.n_subbands, "n_coarse": self.n_coarse, "smoothing": self.smoothing}

    def save_config(self, path):
        """Write the kernel configuration as JSON keyed by the GPU's name and the
        plan's shape (e.g. after sps_tune)."""
        import json
        import torch
        rec = {"gpu": torch.cuda.get_device_name(), "plan": self.shape_key(), "config": self.config.as_dict()}
        with open(path, "w") as f:
            json.dump(rec, f, indent=1)

    def load_config(self, path, strict=True):
        """Apply a configuration written by save_config.  With `strict`, one saved
        for another GPU or another plan shape is refused (ValueError); the
        library still checks the configuration itself (SpsError)."""
        import json
        import torch
        with open(path) as f:
            rec = json.load(f)
        if strict:
            if rec.get("gpu") != torch.cuda.get_device_name():
                raise ValueError(f"configuration saved for {rec.get('gpu')!r}")
            if rec.get("plan") != self.shape_key():
                raise ValueError("configuration saved for another plan shape")
        cfg = rec["config"]
        c = KernelConfig()
        for k in ("brute", "step1", "step2"):
            setattr(c, k, DedispConfig(*cfg[k]))
        c.snr = SnrConfig(*cfg["snr"])
        self.config = c

    # convenience wrappers allocating outputs
    def alloc_outputs(self):
        import torch
        shp = (self.n_widths, self.n_dms)
        return dict(D=torch.empty((self.n_dms, self.n_samples), dtype=torch.int32, device="cuda"),
                    snr=torch.empty(shp, dtype=torch.float64, device="cuda"),
                    peak_t=torch.empty(shp, dtype=torch.int32, device="cuda"),
                    peak_val=torch.empty(shp, dtype=torch.int32, device="cuda"),
                    best=torch.empty(4, dtype=torch.int32, device="cuda"))

    def search(self, x, out=None, workspace=None, stream=None):
        out = out or self.alloc_outputs()
        if workspace is None:
            workspace = self.workspace()
        sps_search(self, x, out["D"], out["snr"], out["peak_t"], out["peak_val"], out["best"],
                   workspace=workspace, stream=stream)
        return out


class BeamBuffers(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("x_pitch", ctypes.c_int64), ("D", ctypes.c_void_p), ("snr", ctypes.c_void_p),
                ("peak_t", ctypes.c_void_p), ("peak_val", ctypes.c_void_p), ("best", ctypes.c_void_p)]


def batch_workspace_bytes(plans, branches=8) -> int:
    """Workspace one Batch of these plans needs (`sps_batch_workspace_bytes`)."""
    arr = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
    nbytes = ctypes.c_size_t()
    check(_L.sps_batch_workspace_bytes(arr, len(plans), int(branches), ctypes.byref(nbytes)),
          "sps_batch_workspace_bytes")
    return int(nbytes.value)


class Batch:
    """A fixed set of beams searched by one CUDA-graph launch (`sps_batch_*`).

    plans: one Plan per beam; xs: each beam's device filterbank (uint8
    [channels][pitch]); outs: each beam's outputs as from Plan.alloc_outputs
    (allocated here when None).  The batch keeps references to everything the
    graph points at, so the buffers live as long as it does."""

    def __init__(self, plans, xs, outs=None, branches=8):
        t = _torch()
        if len(plans) != len(xs):
            raise ValueError("one input per plan")
        self.plans = list(plans)
        self.xs = list(xs)
        self.outs = list(outs) if outs is not None else [p.alloc_outputs() for p in self.plans]
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        self._arr = arr
        self.workspace = t.empty(max(batch_workspace_bytes(self.plans, branches), 256), dtype=t.uint8, device="cuda")
        bufs = (BeamBuffers * len(self.plans))()
        for b, (p, x, o) in enumerate(zip(self.plans, self.xs, self.outs)):
            shp = (p.n_widths, p.n_dms)
            bufs[b] = BeamBuffers(_xdev(p, x).value, int(x.shape[1]),
                                  _dev(o["D"], t.int32, "D", (p.n_dms, p.n_samples)).value,
                                  _dev(o["snr"], t.float64, "snr", shp).value,
                                  _dev(o["peak_t"], t.int32, "peak_t", shp).value,
                                  _dev(o["peak_val"], t.int32, "peak_val", shp).value,
                                  _dev(o["best"], t.int32, "best", (4,)).value)
        self._bufs = bufs
        h = ctypes.c_void_p()
        check(_L.sps_batch_create(arr, bufs, len(self.plans), int(branches), self.workspace.data_ptr(),
                                  ctypes.c_size_t(self.workspace.numel()), ctypes.byref(h)), "sps_batch_create")
        self.handle = h.value

    def launch(self, stream=None):
        check(_L.sps_batch_launch(self.handle, _stream(stream)), "sps_batch_launch")

    @property
    def list_launches(self) -> int:
        """Shared-pass launches in the graph (one per kernel configuration of
        the beams on the pre-summed brute-force kernel)."""
        n = ctypes.c_int32()
        check(_L.sps_batch_list_launches(self.handle, ctypes.byref(n)), "sps_batch_list_launches")
        return n.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                _L.sps_batch_destroy(h)
            except Exception:
                pass
            self.handle = None


class ServerDesc(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t),
                ("resident_bytes", ctypes.c_size_t), ("batch_bytes", ctypes.c_size_t),
                ("inflight", ctypes.c_int32), ("queued", ctypes.c_int32), ("admitted", ctypes.c_int64),
                ("waits_for_memory", ctypes.c_int64), ("failed", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


@dataclass
class Completion:
    """One finished batch as sps_server_poll reports it: its tag, its completion
    time on the server clock, and its status (SPS_OK, or the error that
    stopped it when it was dispatched)."""
    tag: int
    done_s: float
    status: int


class Server:
    """Real-time serving of streaming beams (`sps_server_*`).  Host buffers
    handed to submit() stay referenced here until poll() reports their tag."""

    def __init__(self, hbm_budget_bytes, max_inflight=4):
        h = ctypes.c_void_p()
        check(_L.sps_server_create(ctypes.byref(ServerDesc(int(hbm_budget_bytes), int(max_inflight))),
                                   ctypes.byref(h)), "sps_server_create")
        self.handle = h.value
        self.plans = []
        self._keep = {}

    def add_beam(self, plan) -> int:
        b = ctypes.c_int32()
        check(_L.sps_server_add_beam(self.handle, plan.handle, ctypes.byref(b)), "sps_server_add_beam")
        self.plans.append(plan)
        return b.value

    def remove_beam(self, beam):
        """No further batches for this beam; its queued and in-flight batches
        still run; its overlap tail returns to the arena once they are done."""
        check(_L.sps_server_remove_beam(self.handle, int(beam)), "sps_server_remove_beam")

    def submit(self, beam, x_host, snr_host=None, best_host=None, tag=0):
        """x_host: uint8 array [channels][pitch >= N_t] (pinned torch tensor or numpy)."""
        def ptr(a):
            if a is None:
                return None
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        def dense(a, itemsize, name):
            ok = a.is_contiguous() and a.element_size() == itemsize if hasattr(a, "is_contiguous") else \
                a.flags["C_CONTIGUOUS"] and a.itemsize == itemsize
            if not ok:
                raise ValueError(f"{name} must be C-contiguous with {itemsize}-byte elements")

        p = self.plans[int(beam)] if 0 <= int(beam) < len(self.plans) else None
        if p is not None:  # (an unknown beam is refused by the library)
            if len(x_host.shape) != 2 or x_host.shape[0] != p.channels:
                raise ValueError(f"x_host must be 2-D with one row per channel ({p.channels})")
            dense(x_host, 1, "x_host")
            for a, shape, size, name in ((snr_host, (p.n_widths, p.n_dms), 8, "snr_host"),
                                         (best_host, (4,), 4, "best_host")):
                if a is not None:
                    if tuple(a.shape) != shape:
                        raise ValueError(f"{name} must have shape {shape}")
                    dense(a, size, name)
        if int(tag) in self._keep:
            raise ValueError(f"tag {int(tag)} is still in flight")  # its buffers must stay referenced
        pitch = int(x_host.shape[1])
        self._keep[int(tag)] = (x_host, snr_host, best_host)
        st = _L.sps_server_submit(self.handle, int(beam), ptr(x_host), pitch, ptr(snr_host), ptr(best_host),
                                  ctypes.c_uint64(int(tag)))
        if st != SPS_OK:  # refused before it was queued: nothing of it remains in the library
            self._keep.pop(int(tag), None)
        check(st, "sps_server_submit")

    def poll(self, max_n=256):
        """Finished batches as a list of Completion (oldest first).  A batch
        whose dispatch failed is reported with its error status, not raised:
        every submitted tag is reported exactly once."""
        tags = (ctypes.c_uint64 * max_n)()
        done = (ctypes.c_double * max_n)()
        status = (ctypes.c_int32 * max_n)()
        n = ctypes.c_int32()
        check(_L.sps_server_poll(self.handle, tags, done, status, int(max_n), ctypes.byref(n)), "sps_server_poll")
        out = [Completion(int(tags[i]), float(done[i]), int(status[i])) for i in range(n.value)]
        for c in out:
            self._keep.pop(c.tag, None)
        return out

    def pending(self) -> int:
        n = ctypes.c_int32()
        check(_L.sps_server_pending(self.handle, ctypes.byref(n)), "sps_server_pending")
        return n.value

    def stats(self) -> dict:
        st = ServerStats()
        check(_L.sps_server_get_stats(self.handle, ctypes.byref(st)), "sps_server_get_stats")
        return st.as_dict()

    @staticmethod
    def clock() -> float:
        return float(_L.sps_server_clock())

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                _L.sps_server_destroy(h)
            except Exception:
                pass
            self.handle = None


def sps_plan_check_wait_timeout(plan, polls=1000, stream=None):
    """Launch the failure-detection self-check: a bounded wait that runs out and
    sets the plan's status word (see Plan.status)."""
    check(_L.sps_plan_check_wait_timeout(plan.handle, int(polls), _stream(stream)), "sps_plan_check_wait_timeout")


def sps_presum_tables_verify(delays, per, n_out, cfg: DedispConfig, read_n_out=None):
    """Host-only check of the pre-summed kernels' staging tables for a delay table
    (int32 [rows][channels]); raises SpsError naming the first violated invariant."""
    d = np.ascontiguousarray(delays, np.int32)
    check(_L.sps_presum_tables_verify(d.ctypes.data, d.shape[0], d.shape[1], int(per), int(n_out),
                                      int(n_out if read_n_out is None else read_n_out), ctypes.byref(cfg)),
          "sps_presum_tables_verify")


def sps_measure_int_add_rate(stream=None) -> float:
    """The device's measured 32-bit integer add rate, adds/s."""
    v = ctypes.c_double()
    check(_L.sps_measure_int_add_rate(ctypes.byref(v), _stream(stream)), "sps_measure_int_add_rate")
    return float(v.value)


def upload_filterbank(x_np: np.ndarray, pitch: int | None = None):
    """Copy a host uint8 [channels, samples] array into a pitched device tensor."""
    import torch
    C, n = x_np.shape
    pitch = pitch or (n + 15) // 16 * 16
    t = torch.zeros((C, pitch), dtype=torch.uint8)
    t[:, :n] = torch.from_numpy(np.ascontiguousarray(x_np))
    return t.to("cuda")


# ----------------------------------------------------------------------------- tuning
TUNE_GA, TUNE_RANDOM, TUNE_EXHAUSTIVE = 0, 1, 2
CROSS_UNIFORM, CROSS_ONE_POINT = 0, 1
SPACE_FULL, SPACE_REDUCED = 0, 1
TUNE_MAX_VALUES = 8

_VALID_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p)
_FITNESS_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p)
_TRACE_FN = ctypes.CFUNCTYPE(None, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.c_double, ctypes.c_void_p)


class SpaceDesc(ctypes.Structure):
    _fields_ = [("n_genes", ctypes.c_int32), ("n_values", ctypes.c_void_p), ("kernel_of", ctypes.c_void_p)]


class SearchDesc(ctypes.Structure):
    _fields_ = [("algorithm", ctypes.c_int32), ("crossover", ctypes.c_int32), ("population", ctypes.c_int32),
                ("max_generations", ctypes.c_int32), ("p_cross", ctypes.c_double), ("p_mut", ctypes.c_double),
                ("pool_fraction", ctypes.c_double), ("max_evaluations", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("known_points", ctypes.c_void_p), ("known_fitness", ctypes.c_void_p), ("n_known", ctypes.c_int64),
                ("final_population", ctypes.c_void_p), ("renew", ctypes.c_int32)]


def _with_final_population(desc, n_genes):
    """A copy of `desc` whose final_population points at a fresh [population][n_genes]
    array (returned beside it); the caller's descriptor is left as it was.  Known
    evaluations must have one value per gene (the engine reads n_genes per point)."""
    known = getattr(desc, "_known_arrays", None)
    if desc.n_known and (known is None or known[0].ndim != 2 or known[0].shape != (desc.n_known, n_genes)):
        raise ValueError(f"known evaluations need {n_genes} gene values per point")
    d = SearchDesc.from_buffer_copy(desc)
    d._known_arrays = getattr(desc, "_known_arrays", None)
    fp = np.full((max(1, desc.population), n_genes), -1, np.int32)
    d.final_population = fp.ctypes.data
    return d, fp


def _end_configurations(fp, algorithm):
    """Rows of a final_population array that hold individuals (exhaustive search fills none)."""
    if algorithm == TUNE_EXHAUSTIVE:
        return []
    return [tuple(int(v) for v in row) for row in fp if row[0] >= 0]


class SearchResult(ctypes.Structure):
    _fields_ = [("best_fitness", ctypes.c_double), ("evaluations", ctypes.c_int64), ("generations", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


def search_desc(algorithm=TUNE_GA, population=32, p_cross=0.8, p_mut=0.1, pool_fraction=0.2,
                crossover=CROSS_UNIFORM, max_evaluations=500, max_generations=1000, seed=1,
                known=None, renew=8) -> SearchDesc:
    """Search descriptor.  `known`: earlier evaluations [(point, fitness), ...]
    (e.g. read_tuning_log) served instead of measuring them: a search re-run
    with the same settings replays its log and continues (resume).  `renew`:
    GA renewal tries for offspring that repeat an evaluated individual (0: none)."""
    d = SearchDesc(int(algorithm), int(crossover), int(population), int(max_generations), float(p_cross),
                   float(p_mut), float(pool_fraction), int(max_evaluations), int(seed) & ((1 << 64) - 1))
    d.renew = int(renew)
    if known:
        pts = np.ascontiguousarray([list(p) for p, _ in known], np.int32)
        fit = np.ascontiguousarray([float(f) for _, f in known], np.float64)
        d._known_arrays = (pts, fit)  # kept alive with the descriptor
        d.known_points, d.known_fitness, d.n_known = pts.ctypes.data, fit.ctypes.data, len(known)
    return d


class TuningLog:
    """JSON-lines log of a search: one line per distinct evaluation
    {"eval", "point", "fitness"} (fitness null for +inf), flushed as it goes so
    that an interrupted search leaves a usable log, and a closing line
    {"best", "fitness", "evaluations", "generations"[, "config"]}."""

    def __init__(self, path):
        import json
        self._json = json
        self.f = open(path, "w") if path else None

    def evaluation(self, i, point, fitness):
        if self.f:
            f = None if not np.isfinite(fitness) else float(fitness)
            self.f.write(self._json.dumps({"eval": int(i), "point": [int(v) for v in point], "fitness": f}) + "\n")
            self.f.flush()

    def close(self, best, res, config=None):
        if self.f:
            line = {"best": [int(v) for v in best], "fitness": float(res.best_fitness),
                    "evaluations": int(res.evaluations), "generations": int(res.generations)}
            if config is not None:
                line["config"] = config
            self.f.write(self._json.dumps(line) + "\n")
            self.f.close()
            self.f = None


def read_tuning_log(path):
    """The evaluations of a tuning log as [(point, fitness)], in order (+inf for
    a logged failure); the closing line, if the search finished, is skipped."""
    import json
    out = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            try:
                rec = json.loads(line)
            except ValueError:  # a line cut by an interruption
                break
            if "eval" in rec:
                out.append((tuple(rec["point"]), float("inf") if rec["fitness"] is None else float(rec["fitness"])))
    return out


def sps_optimize(n_values, kernel_of, fitness, valid=None, desc: SearchDesc | None = None, log=None):
    """Host-only GA / random / exhaustive search with Python callbacks.
    Returns (best_point, SearchResult, trace) where trace lists (point, fitness)
    per distinct evaluation, in order; `log` names a JSON-lines tuning log to write."""
    nv = np.ascontiguousarray(n_values, np.int32)
    ko = np.ascontiguousarray(kernel_of, np.int32)
    if nv.ndim != 1 or ko.shape != nv.shape:
        raise ValueError("n_values and kernel_of need one entry per gene")
    sp = SpaceDesc(nv.size, nv.ctypes.data, ko.ctypes.data)
    desc = desc or search_desc()
    n = nv.size
    trace, errors = [], []

    def _pt(ptr):
        return tuple(ptr[g] for g in range(n))

    def _fit(ptr, _):
        try:
            return float(fitness(_pt(ptr)))
        except Exception as e:  # keep exceptions from crossing the C boundary
            errors.append(e)
            return float("inf")

    def _val(ptr, _):
        try:
            return 1 if valid(_pt(ptr)) else 0
        except Exception as e:
            errors.append(e)
            return 0

    lg = TuningLog(log)

    def _tr(i, ptr, f, _):
        trace.append((_pt(ptr), f))
        lg.evaluation(i, trace[-1][0], f)

    cf, cv, ct = _FITNESS_FN(_fit), _VALID_FN(_val) if valid else None, _TRACE_FN(_tr)
    best = np.zeros(n, np.int32)
    res = SearchResult()
    d, fp = _with_final_population(desc, n)
    st = _L.sps_optimize(ctypes.byref(sp), ctypes.byref(d), cv, cf, ct, None, best.ctypes.data, ctypes.byref(res))
    if errors:
        raise errors[0]
    check(st, "sps_optimize")
    res.final_population = _end_configurations(fp, desc.algorithm)
    lg.close(best, res)
    return tuple(int(v) for v in best), res, trace


def sps_tune_space(plan, which=SPACE_FULL):
    """(n_values, kernel_of, values) of the plan's tuning space."""
    n = ctypes.c_int32()
    check(_L.sps_tune_space(plan.handle, int(which), 0, ctypes.byref(n), None, None, None), "sps_tune_space")
    nv = np.zeros(n.value, np.int32)
    ko = np.zeros(n.value, np.int32)
    vals = np.zeros((n.value, TUNE_MAX_VALUES), np.int32)
    check(_L.sps_tune_space(plan.handle, int(which), n.value, ctypes.byref(n), nv.ctypes.data, ko.ctypes.data,
                            vals.ctypes.data), "sps_tune_space")
    return nv, ko, [list(vals[g, :nv[g]]) for g in range(n.value)]


def sps_tune_config(plan, which, point) -> KernelConfig:
    pt = np.ascontiguousarray(point, np.int32)
    c = KernelConfig()
    check(_L.sps_tune_config(plan.handle, int(which), pt.ctypes.data, ctypes.byref(c)), "sps_tune_config")
    return c


def sps_tune(plan, x, which=SPACE_FULL, desc: SearchDesc | None = None, reps=3, limit_ms=0.0, out=None,
             workspace=None, stream=None, log=None):
    """Live tuning of the plan's kernels on input x; leaves the plan on the best
    configuration.  Returns (best_point, SearchResult, trace).  `log` names a
    JSON-lines tuning log (resume with search_desc(known=read_tuning_log(path)))."""
    t = _torch()
    out = out or plan.alloc_outputs()
    if workspace is None:
        workspace = plan.workspace()
    n = int(sps_tune_space(plan, which)[0].size)
    trace = []
    lg = TuningLog(log)

    def _tr(i, ptr, f, _):
        trace.append((tuple(ptr[g] for g in range(n)), f))
        lg.evaluation(i, trace[-1][0], f)

    ct = _TRACE_FN(_tr)
    best = np.zeros(n, np.int32)
    res = SearchResult()
    shp = (plan.n_widths, plan.n_dms)
    desc = desc or search_desc()
    d, fp = _with_final_population(desc, n)
    check(_L.sps_tune(plan.handle, int(which), ctypes.byref(d), _xdev(plan, x),
                      ctypes.c_int64(x.shape[1]), _dev(out["D"], t.int32, "D", (plan.n_dms, plan.n_samples)),
                      _dev(workspace, workspace.dtype, "workspace"),
                      ctypes.c_size_t(workspace.numel() * workspace.element_size()),
                      _dev(out["snr"], t.float64, "snr", shp), _dev(out["peak_t"], t.int32, "peak_t", shp),
                      _dev(out["peak_val"], t.int32, "peak_val", shp), int(reps), float(limit_ms), ct, None,
                      best.ctypes.data, ctypes.byref(res), _stream(stream)), "sps_tune")
    res.final_population = _end_configurations(fp, desc.algorithm)
    lg.close(best, res, plan.config.as_dict())
    return tuple(int(v) for v in best), res, trace
