"""Benchmark of the single-pulse-search hot path on one Apertif-shaped beam.

One step = one 1.024 s batch (1536 channels x 12500 samples, uint8) searched
over 2048 DM trials (0..409.4, step 0.2) and 7 boxcar widths (1..64):
brute-force de-dispersion, then the fused boxcar + S/N + peak kernel and the
detection reduction.  The two-step subband path (32 subbands, 64 coarse DMs)
is timed on the same batch and reported beside it.

Metric: DM-trial samples per second (n_dms * n_samples per step / step time),
device time from CUDA events, inputs resident in HBM.  Headline: K steps on
--streams streams (four by default) in turn, eight distinct input batches (210 MB, more than L2)
rotated, events around all K steps.  Breakdown: the same steps on one stream,
events around each kernel call, L2 flushed (a 256 MiB write) before every
step outside the events.  `e2e` repeats the metric through the host entry
point (pinned host batch in, S/N tables out).

Multi-GPU (torchrun): independent replicas, one beam per GPU, no collective
on the data path; value = all ranks' samples / the slowest rank's time.

--impl reference times the CPU oracle (test infrastructure, never the product
path) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DM-trial samples/s (dedisp+boxcar+SNR)"
UNIT = "DM-trial samples/s"
N_SM = 152
INT32_LANES_PER_SM_CLK = 128
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 200 steps keep the timed region (two legs, ~0.4 s) long enough for several clock samples
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-subband", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dms", type=int, default=2048,
                    help="DM trials (fewer only for small profiling cases; bench lines use 2048)")
    ap.add_argument("--presum", type=int, choices=[0, 1, 2], default=None,
                    help="brute-force kernel: 0 single channels, 1 pairs, 2 quads (default: the plan's default)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-beam leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the real-time serving leg")
    ap.add_argument("--no-tuning", action="store_true", help="skip the tuning leg")
    ap.add_argument("--e2e-threads", type=int, default=12,
                    help="host threads taking the end-to-end leg's steps in turn")
    ap.add_argument("--streams", type=int, default=4,
                    help="streams the headline's (and the streamed two-step path's) batches take in turn")
    return ap.parse_args()


def dist_init(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("SPS_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world


def measured_hbm_gbs():
    """The copy bandwidth measured on this machine's GPUs (MEASURED_PEAKS.json,
    written by the driver), else the stated fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def local_device_index() -> int:
    """The GPU this rank drives: torchrun's LOCAL_RANK (one process per GPU)."""
    return int(os.environ.get("LOCAL_RANK", "0"))


def rank_beam(rank: int, dms: int = 2048):
    """The beam rank `rank` searches: replicas search independent beams (seed
    2 + rank), so no data moves between ranks."""
    from paper_1811_04165_gb300 import synth
    wl = synth.apertif_beam(seed=2 + rank)
    if dms != 2048:
        wl.dms = wl.dms[:dms].copy()
        wl.name += f"-first{dms}dm"
    return wl


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int, device=None) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), max=float(f[2]), power=float(f[3]), hw=f[5], hwt=f[6], swt=f[7],
                                 cap=f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        loaded = [r for r in rows if r["power"] > 200.0] or rows
        reasons = set()
        for r in loaded:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("cap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in loaded), "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": sorted(reasons), "samples": len(loaded)}


def profiled_traffic(kernel_src: str, summary: str):
    """DRAM bytes per launch recorded in a profile summary, or None when the
    kernel's source has changed since the counters were taken."""
    import hashlib
    import re
    try:
        data = open(os.path.join(ROOT, kernel_src), "rb").read()
        text = open(os.path.join(ROOT, summary)).read()
    except OSError:
        return None
    blob = hashlib.sha1(b"blob %d\0" % len(data) + data).hexdigest()
    t = re.search(r"traffic_bytes_per_launch: (\d+)", text)
    b = re.search(r"traffic_source_blob: ([0-9a-f]+)", text)
    return int(t.group(1)) if t and b and b.group(1) == blob else None


def host_threads():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rows_threaded(x, d, rows, n_t, widths, threads):
    """The oracle's dedispersion + S/N over the given DM rows, split into
    `threads` contiguous parts run concurrently (the oracle's C routines
    release the interpreter lock; every row is independent, so the results
    are those of one call)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    parts = [p for p in np.array_split(rows, threads) if p.size]

    def one(p):
        D = oracle.dedisperse(x, d[p], n_t)
        return oracle.snr(D, widths)

    with ThreadPoolExecutor(len(parts)) as ex:
        return list(ex.map(one, parts))


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, or implementer/part on Arm)."""
    import platform
    try:
        fields = {}
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip(), v.strip())
        if "model name" in fields:
            return fields["model name"]
        if "CPU part" in fields:
            names = {("0x41", "0xd4f"): "Arm Neoverse V2", ("0x41", "0xd40"): "Arm Neoverse V1"}
            key = (fields.get("CPU implementer", "?"), fields["CPU part"])
            return names.get(key, f"{platform.machine()} implementer {key[0]} part {key[1]}")
    except OSError:
        pass
    return platform.machine()


def cpu_oracle_tiny():
    """The oracle's whole search (dedispersion + S/N) on the tiny 64-channel
    configuration, single thread: DM-trial samples/s and seconds."""
    import oracle
    from paper_1811_04165_gb300 import synth
    wl = synth.tiny_brute()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_t + int(d.max()), wl.seed, wl.pulses)
    reps, t0 = 0, time.perf_counter()
    while reps < 3 or time.perf_counter() - t0 < 1.0:
        D = oracle.dedisperse(x, d, wl.n_t)
        oracle.snr(D, wl.widths)
        reps += 1
    dt = (time.perf_counter() - t0) / reps
    return wl.dms.size * wl.n_t / dt, dt


def cpu_oracle_all_cores(wl, x, threads):
    """DM-trial samples/s of the oracle on every host core, over the whole batch,
    and its (snr, peak_t, peak_val) tables [n_widths, n_dms]."""
    import oracle
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    rows = np.arange(wl.dms.size)
    t0 = time.perf_counter()
    parts = oracle_rows_threaded(x, d, rows, wl.n_t, wl.widths, threads)
    dt = time.perf_counter() - t0
    tables = tuple(np.concatenate([r[k] for r in parts], axis=1) for k in range(3))
    return rows.size * wl.n_t / dt, dt, tables


def check_outputs(wl, x, out, tables, n_rows=12):
    """The pipelined run's outputs for input x against the oracle: the whole
    S/N table (relative 1e-5), peak_t and peak_val (exact), the detection, and
    `n_rows` rows of D (exact)."""
    import oracle
    s, pt, pv = tables
    bi, bw = oracle.detect(s)
    rows = np.unique(np.linspace(0, wl.dms.size - 1, n_rows).astype(np.int64))
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    D_rows = oracle.dedisperse(x, d[rows], wl.n_t)
    g_s = out["snr"].cpu().numpy()
    err = np.abs(g_s - s)
    res = {"snr_entries": int(s.size), "D_rows": int(rows.size),
           "snr_ok": bool(np.all(err <= 1e-5 * np.abs(s) + 1e-9)),
           "max_rel_err": float(np.max(err / np.maximum(np.abs(s), 1e-300))),
           "peaks_ok": bool(np.array_equal(out["peak_t"].cpu().numpy(), pt) and
                            np.array_equal(out["peak_val"].cpu().numpy(), pv)),
           "best_ok": out["best"].cpu().numpy().tolist() == [bi, bw, int(pt[bw, bi]), int(pv[bw, bi])],
           "D_ok": bool(np.array_equal(out["D"].cpu().numpy()[rows], D_rows))}
    res["ok"] = res["snr_ok"] and res["peaks_ok"] and res["best_ok"] and res["D_ok"]
    return res


def cpu_oracle_rate(wl, x, target_s=12.0, max_rows=None):
    """DM-trial samples/s of the oracle (dedispersion + S/N) on a bounded row sample."""
    import oracle
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    probe_rows = np.arange(0, wl.dms.size, wl.dms.size // 8)[:8]
    t0 = time.perf_counter()
    D = oracle.dedisperse(x, d[probe_rows], wl.n_t)
    oracle.snr(D, wl.widths)
    per_row = (time.perf_counter() - t0) / probe_rows.size
    n = int(max(8, min(wl.dms.size if max_rows is None else max_rows, target_s / max(per_row, 1e-6))))
    rows = np.linspace(0, wl.dms.size - 1, n).astype(np.int64)
    t0 = time.perf_counter()
    D = oracle.dedisperse(x, d[rows], wl.n_t)
    oracle.snr(D, wl.widths)
    dt = time.perf_counter() - t0
    return rows.size * wl.n_t / dt, dt, rows.size


def run_reference(args, rank, world):
    """The CPU oracle as the reference arm, on the host cores (rank 0 only)."""
    from paper_1811_04165_gb300 import synth
    import oracle
    if rank != 0:
        return
    wl = synth.apertif_beam()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_t + int(d.max()), wl.seed, wl.pulses)
    threads = host_threads()
    rows_per_step = min(wl.dms.size, 16 * threads)
    rng = np.random.Generator(np.random.PCG64(11))
    times = []
    for s in range(args.warmup + args.steps):
        rows = np.sort(rng.choice(wl.dms.size, rows_per_step, replace=False))
        t0 = time.perf_counter()
        oracle_rows_threaded(x, d, rows, wl.n_t, wl.widths, threads)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    dt = sum(times)
    value = rows_per_step * wl.n_t * len(times) / dt
    sample = (f"{rows_per_step} random DM trials x {wl.n_t} samples x {wl.channels} channels per step, "
              f"split over {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": workload_config(wl, "brute", args.streams),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(wl, mode, streams):
    return {"workload": wl.name, "channels": wl.channels, "band_mhz": [wl.f_lo, wl.f_hi], "t_samp_s": wl.t_samp,
            "samples_per_batch": wl.n_t, "dm_trials": int(wl.dms.size), "dm_step": 0.2,
            "widths": [int(w) for w in wl.widths], "dedispersion": mode,
            "l2": "headline: 8 rotating input batches (210 MB > L2); kernel breakdown: L2 flushed before every "
                  "step (256 MiB write)",
            "pipeline": f"headline: consecutive batches on {streams} streams in turn (each batch's full path on its "
                        "stream, own workspace and outputs); kernel breakdown: one stream, sequential",
            "parallelism": "replicas (one beam per GPU)"}


def time_pipelined(torch, plan, xs, steps, warmup, n_streams=2):
    """Whole-job CUDA-event time (ms) of `steps` batches, each searched in full
    (sps_search) on the next of `n_streams` streams with its own workspace and
    outputs, so consecutive batches overlap; inputs rotate through xs.  Also
    returns, per stream, the outputs its last timed batch left and that
    batch's input index (checked against the oracle afterwards)."""
    import paper_1811_04165_gb300 as sps
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    outs = [plan.alloc_outputs() for _ in range(n_streams)]
    wss = [torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda") for _ in range(n_streams)]
    cur = torch.cuda.current_stream()

    def run(n, first):
        for s in range(n):
            i = s % n_streams
            o = outs[i]
            sps.sps_search(plan, xs[(first + s) % len(xs)], o["D"], o["snr"], o["peak_t"], o["peak_val"], o["best"],
                           workspace=wss[i], stream=streams[i])

    run(warmup, 0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for st in streams:
        st.wait_event(e0)
    run(steps, warmup)
    for st in streams:
        ev = torch.cuda.Event()
        ev.record(st)
        cur.wait_event(ev)
    e1.record(cur)
    torch.cuda.synchronize()
    held = []
    for i in range(min(n_streams, steps)):
        last = max(s for s in range(steps) if s % n_streams == i)
        held.append((last, outs[i], (warmup + last) % len(xs)))
    return e0.elapsed_time(e1), held


def e2e_pipelined(torch, plan, xh, steps, warmup, device, n_workers=8):
    """Wall time (s) of `steps` batches through the host entry point
    (sps_search_host: pinned host batch in, S/N tables and detection back,
    stream synchronised) on `n_workers` host threads, each with its own stream
    and device buffers, taking steps in turn; ctypes releases the GIL during
    the call, so one batch's copies overlap another's search."""
    import threading
    import paper_1811_04165_gb300 as sps
    shp = (plan.n_widths, plan.n_dms)
    workers = []
    for _ in range(n_workers):
        workers.append(dict(stream=torch.cuda.Stream(device=device),
                            xd=torch.empty((plan.channels, plan.pitch), dtype=torch.uint8, device=device),
                            out=plan.alloc_outputs(),
                            ws=torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=device),
                            hs=torch.empty(shp, dtype=torch.float64).pin_memory(),
                            ht=torch.empty(shp, dtype=torch.int32).pin_memory(),
                            hv=torch.empty(shp, dtype=torch.int32).pin_memory(),
                            hb=torch.empty(4, dtype=torch.int32).pin_memory()))
    errors = []

    def run(w, first, n):
        try:
            torch.cuda.set_device(device)
            o = workers[w]
            for s in range(first + w, first + n, n_workers):
                sps.sps_search_host(plan, xh[s % len(xh)], o["xd"], o["out"]["D"], o["out"]["snr"],
                                    o["out"]["peak_t"], o["out"]["peak_val"], o["out"]["best"], o["hs"], o["ht"],
                                    o["hv"], o["hb"], workspace=o["ws"], stream=o["stream"])
        except Exception as e:  # surfaced after join
            errors.append(e)

    def batch(first, n):
        ts = [threading.Thread(target=run, args=(w, first, n)) for w in range(n_workers)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        if errors:
            raise errors[0]

    batch(0, warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch(warmup, steps)
    return time.perf_counter() - t0


def launches_per_step(plan):
    """Kernels of one brute-force search: the pre-pass (pre-summed series, or the
    shifted copies) and the pass, then the S/N kernel (one launch for widths
    1, 2, 4, ...; one per eight widths otherwise) and the detection kernel."""
    pow2 = list(plan.widths) == [1 << k for k in range(plan.n_widths)] and plan.n_widths <= 7
    snr = 1 if pow2 and plan.smoothing == 0 else (plan.n_widths + 7) // 8
    return 2 + snr + 1


def device_noise(torch, shape, seed, dev):
    """uint8 Gaussian-like noise (mean 128, sd 16) drawn on the device: inputs for
    the legs whose timing and exactness checks do not depend on the values."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    x = torch.randn(shape, generator=g, device=dev).mul_(16).add_(128).round_().clamp_(0, 255)
    return x.to(torch.uint8)


def events_ms(torch, fn, reps, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def leg_batched(torch, dev, reps=5):
    """The batched-beam workload: 40 beams (alternately 1536 and 384 channels,
    512-4096 DM trials with steps 0.1-0.5, 1-7 widths) per 1.024 s batch, on the
    GA-tuned tiles stored per channel count, as one graph launch (sps_batch_*)
    against plain per-beam sps_search launches on one stream; every beam's
    batched outputs must equal its own search's."""
    import paper_1811_04165_gb300 as sps
    from paper_1811_04165_gb300 import synth
    from paper_1811_04165_gb300 import batch_study
    wls = synth.batch_beams(40)
    t0 = time.perf_counter()
    plans = [sps.Plan.from_workload(wl) for wl in wls]
    tuned = batch_study.apply_tuned(plans)
    plan_s = time.perf_counter() - t0
    xs = [device_noise(torch, (p.channels, p.pitch), 1000 + b, dev) for b, p in enumerate(plans)]
    ws = torch.empty(max(sps.batch_workspace_bytes([p], 1) for p in plans), dtype=torch.uint8, device=dev)
    outs = [p.alloc_outputs() for p in plans]

    def per_beam():
        for p, x, o in zip(plans, xs, outs):
            p.search(x, out=o, workspace=ws)

    t_beam = events_ms(torch, per_beam, reps)
    del ws
    batch = sps.Batch(plans, xs, branches=8)
    t_batch = events_ms(torch, batch.launch, reps)
    exact = all(torch.equal(o[k], r[k]) for o, r in zip(batch.outs, outs) for k in ("D", "snr", "peak_t",
                                                                                    "peak_val", "best"))
    samples = sum(wl.dm_trial_samples for wl in wls)
    res = {"workload": "40 beams, 1536/384 channels, 512-4096 DM trials, 1-7 widths, 12500 samples each",
           "value": samples / (t_batch * 1e-3), "unit": UNIT, "ms_per_batch": t_batch,
           "per_beam_ms_per_batch": t_beam, "speedup_vs_per_beam": t_beam / t_batch,
           "real_time_beams": len(wls) * 1024.0 / t_batch, "exact_vs_per_beam": exact,
           "shared_pass_launches": batch.list_launches,
           "kernel_configs": f"GA-tuned per channel count (stored), taken by {tuned} of {len(plans)} beams",
           "plan_s": plan_s, "inputs": "device-drawn noise (timing and exactness do not depend on values)"}
    del batch
    torch.cuda.empty_cache()
    return res


def leg_serving(torch, dev, seconds=3.0):
    """The real-time serving workload (sps_server_*): beams alternately 1536 and
    384 channels, 1024-4096 DM trials, widths 1..64, 1.024 s batches arriving
    as per-beam Poisson processes with +-50 ms jitter.  p50/p99 batch latency
    (GPU completion on the host clock minus arrival) against the 1.024 s
    deadline, for the server (8 slots, continuous batching) and for one batch
    at a time (plain per-beam processing): 48 beams in real time, then 96
    beams with the arrival period compressed to 96 ms, which emulates 1024
    beams."""
    import numpy as np
    import paper_1811_04165_gb300 as sps
    from paper_1811_04165_gb300 import serve_study
    wls = serve_study.serve_beams(96)
    t0 = time.perf_counter()
    plans = [sps.Plan.from_workload(wl) for wl in wls]
    plan_s = time.perf_counter() - t0
    rng = np.random.Generator(np.random.PCG64(1))
    host_x = {ch: torch.from_numpy(np.clip(np.rint(128 + 16 * rng.standard_normal((ch, 12500))), 0, 255)
                                   .astype(np.uint8)).pin_memory() for ch in (384, 1536)}
    budget = 32 << 30
    out = {"deadline_s": serve_study.DEADLINE_S, "plan_s": plan_s, "hbm_budget_bytes": budget}
    for name, n, period, dur in (("real_time_48_beams", 48, serve_study.DEADLINE_S, seconds),
                                 ("emulated_1024_beams", 96, 0.096, seconds * 0.096 / serve_study.DEADLINE_S * 4)):
        for mode, inflight in (("served", 8), ("per_beam", 1)):
            r = serve_study.run(plans[:n], host_x, period, dur, inflight, seed=n, budget=budget)
            r["period_s"] = period
            r["within_period"] = r["p99_s"] <= period
            out[f"{name}/{mode}"] = r
    return out


def leg_tuning(torch, dev):
    """The tuner against exhaustive search on this workload: the committed
    live-measured table of the beam's reduced brute-force space replayed with
    the GA and random search at 10 % of its valid points over 20 seeds each,
    and the table's optimum and the default configuration re-timed live."""
    import paper_1811_04165_gb300 as sps
    from paper_1811_04165_gb300 import synth, tune_study
    tab = tune_study.load_table(tune_study.BEAM_TABLE)
    res = tune_study.replay(tab, seeds=range(20), budget_frac=0.1)
    wl = synth.apertif_beam()
    plan = sps.Plan.from_workload(wl)
    default = plan.config
    x = device_noise(torch, (plan.channels, plan.pitch), 7, dev)
    o = plan.alloc_outputs()
    ws = plan.workspace()
    live = {}
    for name, point in (("optimum", tab["optimum_point"]), ("default", tab["default_point"])):
        if point is None:
            continue
        plan.config = sps.sps_tune_config(plan, sps.SPACE_REDUCED, point)
        live[name] = events_ms(torch, lambda: plan.search(x, out=o, workspace=ws), 20, warm=3)
    plan.config = default
    res["live_ms"] = live
    if "optimum" in live and "default" in live:
        res["live_default_over_optimum"] = live["default"] / live["optimum"]
    return res


def time_path(torch, plan, xs, outs, steps, warmup, ws, flush, with_events=True):
    """Per-step CUDA-event times (ms) of [dedisperse, snr+detect] on the current stream."""
    import paper_1811_04165_gb300 as sps
    st = torch.cuda.current_stream()
    res = []
    for s in range(warmup + steps):
        x = xs[s % len(xs)]
        flush.fill_(s & 0xFF)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        sps.sps_dedisperse(plan, x, outs["D"], workspace=ws, stream=st)
        e1.record(st)
        sps.sps_snr(plan, outs["D"], outs["snr"], outs["peak_t"], outs["peak_val"], outs["best"], stream=st)
        e2.record(st)
        if s >= warmup:
            res.append((e0, e1, e2))
    torch.cuda.synchronize()
    return [(a.elapsed_time(b), b.elapsed_time(c)) for a, b, c in res]


def main():
    args = parse()
    rank, world = dist_init(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import paper_1811_04165_gb300 as sps
    from paper_1811_04165_gb300 import synth

    local = local_device_index()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = rank_beam(rank, args.dms)
    plan = sps.Plan.from_workload(wl, mode=sps.MODE_BRUTE)
    if args.presum is not None:
        c = plan.config
        c.brute.presum = args.presum
        plan.config = c
    pitch = plan.pitch
    n_in = plan.input_samples
    n_batches = 8  # 8 x 26 MB: more input than the 126 MB L2
    xs_host = [synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, n_in, wl.seed + 100 * b, wl.pulses,
                                pitch=pitch) for b in range(n_batches)]
    xs = [torch.from_numpy(x).to(dev) for x in xs_host]
    outs = plan.alloc_outputs()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # the device's measured integer add rate (roofline context; outside the timed region)
    int_peak_tadd = sps.sps_measure_int_add_rate() / 1e12

    # ---- timed region: K steps of the brute-force path
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        pipe_ms, held = time_pipelined(torch, plan, xs, args.steps, args.warmup, args.streams)
        times = time_path(torch, plan, xs, outs, args.steps, args.warmup, None, flush)
    barrier(world)
    dedisp_ms = [a for a, _ in times]
    snr_ms = [b for _, b in times]
    step_ms = [a + b for a, b in times]
    total_s = max_over_ranks(pipe_ms / 1e3, world, dev)
    seq_s = max_over_ranks(sum(step_ms) / 1e3, world, dev)
    samples = wl.dm_trial_samples
    value = world * samples * args.steps / total_s
    ms_per_step = 1e3 * total_s / args.steps

    # ---- roofline of the dominant kernel (brute-force de-dispersion)
    adds = float(wl.dms.size) * wl.n_t * wl.channels
    dd_ms = statistics.mean(dedisp_ms)
    peak_tadd = N_SM * INT32_LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    achieved = adds / (dd_ms * 1e-3) / 1e12
    presum = plan.config.brute.presum
    kernel = "presum_pass_kernel" if presum else "u8_pass_kernel"
    src = "dedisperse_presum.cu" if presum else "dedisperse_u8.cu"
    summary = f"profiles/presum{1 << presum}_pass_brute_apertif_2048dm.md" if presum else \
        "profiles/u8_pass_brute_apertif_2048dm.md"
    traffic = profiled_traffic("paper_1811_04165_gb300/csrc/" + src, summary) if args.dms == 2048 else None
    roofline = {"bound": "alu", "kernel": kernel + " (brute force, incl. its pre-pass)", "achieved": achieved,
                "peak": peak_tadd,
                "unit": "Tadd/s", "frac": achieved / peak_tadd, "traffic": traffic,
                "algorithmic_bytes_per_launch": wl.channels * pitch + 4 * wl.dm_trial_samples,
                "algorithmic_adds_per_launch": adds, "ms_per_launch": dd_ms,
                "peak_derivation": "152 SMs x 128 INT32 lanes/clk x 2070 MHz",
                "peak_measured": int_peak_tadd, "frac_of_measured": achieved / int_peak_tadd,
                "peak_measured_how": "sps_measure_int_add_rate: independent add chains on the ALU and FMA pipes",
                "kernel_own_bound": {
                    2: "shared-memory data path: shared loads on 71 % of the pass's cycles (94 % of the quad "
                       "layout's algorithmic wavefronts) plus 15.5 % stage fills by bulk copies; the pass executes a "
                       "quarter of the brute-force adds (ncu, " + summary + ")",
                    1: "shared-memory data path (pairs: half the brute-force adds; no committed ncu capture)",
                    0: "instruction issue and the shared-memory data path: 75 % issue-active, 1.33 instructions "
                       "per add, L1/shared 68 % (ncu, " + summary + ")"}[presum]}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": workload_config(wl, "brute", args.streams),
            "kernels_ms": {"dedisperse": dd_ms, "snr_detect": statistics.mean(snr_ms)},
            "kernel_config": plan.config.as_dict(),
            "sequential_ms_per_step": 1e3 * seq_s / args.steps,
            "sequential_step_ms": {"median": statistics.median(step_ms),
                                   "p10": float(np.percentile(step_ms, 10)),
                                   "p90": float(np.percentile(step_ms, 90))},
            "real_time_beams": 1024.0 / ms_per_step, "gpu_launches": launches_per_step(plan) * args.steps,
            "roofline": roofline, "clocks": clk.summary()}

    # ---- the other kernels against their own rooflines (the HBM peak from the
    # driver's measured copy bandwidth when present)
    hbm_gbs, hbm_src = measured_hbm_gbs()
    snr_ms_mean = statistics.mean(snr_ms)
    snr_bytes = 4.0 * wl.dm_trial_samples + wl.widths.size * wl.dms.size * 16.0
    # the pass's own bound, the shared-memory data path: the bytes its layout
    # must read from shared memory (a 16-bit lane per unit of 2^presum channels,
    # a byte per channel for single channels) per DM-trial sample
    units = wl.channels / (1 << presum) if presum else wl.channels
    shared_bytes = float(wl.dm_trial_samples) * units * (2 if presum else 1)
    shared_peak = N_SM * 128 * SM_MAX_MHZ * 1e6 / 1e12  # TB/s: 128 B per clock per SM
    line["kernel_rooflines"] = {"dedisperse_shared": {
        "bound": "shared", "algorithmic_shared_bytes_per_launch": shared_bytes, "ms_per_launch": dd_ms,
        "achieved_tbs": shared_bytes / (dd_ms * 1e-3) / 1e12, "peak_tbs": shared_peak,
        "frac": shared_bytes / (dd_ms * 1e-3) / 1e12 / shared_peak,
        "peak_derivation": "152 SMs x 128 B/clk x 2070 MHz", "note": "time of the whole call, pre-pass included"},
        "snr_detect": {
        "bound": "hbm", "algorithmic_bytes_per_launch": snr_bytes, "ms_per_launch": snr_ms_mean,
        "achieved_gbs": snr_bytes / (snr_ms_mean * 1e-3) / 1e9, "peak_gbs": hbm_gbs, "peak_source": hbm_src,
        "frac": snr_bytes / (snr_ms_mean * 1e-3) / 1e9 / hbm_gbs,
        "note": "the exact 64-bit moments alone take about 0.032 ms at full occupancy "
                "(profiles/snr_pow2_kernel_apertif_2048dm.md)"}}

    # ---- the two-step subband path on the same batch
    if not args.no_subband and args.dms == 2048:
        wls = synth.apertif_beam(seed=2 + rank, subband=True)
        ps = sps.Plan.from_workload(wls)
        ws = ps.workspace()
        outs_s = ps.alloc_outputs()
        ts = time_path(torch, ps, xs, outs_s, args.steps, args.warmup, ws, flush)
        sub_ms = statistics.mean(a + b for a, b in ts)
        line["subband"] = {"value": samples / (sub_ms * 1e-3), "unit": UNIT, "ms_per_step": sub_ms,
                           "dedisperse_ms": statistics.mean(a for a, _ in ts),
                           "snr_detect_ms": statistics.mean(b for _, b in ts),
                           "subbands": 32, "coarse_dms": 64}
        # the same path streamed like the headline (batches on the headline's streams in turn);
        # each stream's last batch must equal a search of its input on its own
        sub_pipe_ms, held_s = time_pipelined(torch, ps, xs, args.steps, args.warmup, args.streams)
        same = True
        for _, o, xi in held_s:
            r = ps.search(xs[xi])
            same = same and all(torch.equal(o[k], r[k]) for k in ("D", "snr", "peak_t", "peak_val", "best"))
        torch.cuda.synchronize()
        line["subband"]["pipelined"] = {"value": samples * args.steps / (sub_pipe_ms * 1e-3), "unit": UNIT,
                                        "ms_per_step": sub_pipe_ms / args.steps, "outputs_equal_own_search": same,
                                        "how": f"batches on {args.streams} streams in turn, as the headline"}
        # roofline of the two steps: the slower of their algorithmic bytes over HBM
        # (x in, Y written and read, D out) and their adds at the derived ALU peak
        n_1 = ps.step1_samples
        y_bytes = 2.0 * wls.coarse_dms.size * 32 * n_1
        sb_bytes = wls.channels * ps.pitch + 2 * y_bytes + 4.0 * wl.dm_trial_samples
        sb_adds = float(wls.coarse_dms.size) * wls.channels * n_1 + float(wls.dms.size) * 32 * wls.n_t
        t_roof = max(sb_bytes / (hbm_gbs * 1e9), sb_adds / (peak_tadd * 1e12))
        sb_ms = line["subband"]["dedisperse_ms"]
        line["kernel_rooflines"]["subband_dedisperse"] = {
            "bound": "alu" if sb_adds / (peak_tadd * 1e12) > sb_bytes / (hbm_gbs * 1e9) else "hbm",
            "algorithmic_bytes_per_launch": sb_bytes, "algorithmic_adds_per_launch": sb_adds,
            "roofline_ms": 1e3 * t_roof, "ms_per_launch": sb_ms, "frac": 1e3 * t_roof / sb_ms}
        # the two steps against their own bound, the shared-memory data path: step one
        # reads one staged byte per channel-sample add (four samples per 32-bit load),
        # step two two bytes per (trial, subband, sample) (uint16 subband series)
        sb_shared = float(wls.coarse_dms.size) * wls.channels * n_1 + 2.0 * wls.dms.size * 32 * wls.n_t
        line["kernel_rooflines"]["subband_shared"] = {
            "bound": "shared", "algorithmic_shared_bytes_per_launch": sb_shared, "ms_per_launch": sb_ms,
            "achieved_tbs": sb_shared / (sb_ms * 1e-3) / 1e12, "peak_tbs": shared_peak,
            "frac": sb_shared / (sb_ms * 1e-3) / 1e12 / shared_peak,
            "peak_derivation": "152 SMs x 128 B/clk x 2070 MHz",
            "note": "time of the three launches (shifted copies, step one, step two)"}

    # ---- the batched-beam, serving and tuning workloads (rank 0 of a single-GPU run)
    if world == 1 and args.dms == 2048:
        if not args.no_batched:
            line["batched"] = leg_batched(torch, dev)
        if not args.no_serving:
            line["serving"] = leg_serving(torch, dev)
        if not args.no_tuning:
            line["tuning"] = leg_tuning(torch, dev)

    # ---- end to end through the host entry point
    if args.no_e2e:
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    xh = [torch.from_numpy(x).pin_memory() for x in xs_host]
    shp = (plan.n_widths, plan.n_dms)
    hs = torch.empty(shp, dtype=torch.float64).pin_memory()
    ht = torch.empty(shp, dtype=torch.int32).pin_memory()
    hv = torch.empty(shp, dtype=torch.int32).pin_memory()
    hb = torch.empty(4, dtype=torch.int32).pin_memory()
    xd = torch.empty((wl.channels, pitch), dtype=torch.uint8, device=dev)
    e2e_t = []
    for s in range(args.warmup + args.steps):
        flush.fill_(s & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sps.sps_search_host(plan, xh[s % n_batches], xd, outs["D"], outs["snr"], outs["peak_t"], outs["peak_val"],
                            outs["best"], hs, ht, hv, hb)
        if s >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
    e2e_seq = max_over_ranks(sum(e2e_t), world, dev)
    e2e_total = max_over_ranks(e2e_pipelined(torch, plan, xh, args.steps, args.warmup, dev, args.e2e_threads),
                               world, dev)
    line["e2e"] = {"value": world * samples * args.steps / e2e_total, "unit": UNIT,
                   "h2d_bytes_per_step": wl.channels * pitch,
                   "d2h_bytes_per_step": int(hs.numel() * 8 + ht.numel() * 4 + hv.numel() * 4 + 16),
                   "ms_per_step": 1e3 * e2e_total / args.steps,
                   "how": f"sps_search_host on {args.e2e_threads} host threads taking steps in turn (own stream and "
                          "buffers each); every step copies its pinned batch in and its S/N tables and detection out",
                   "sequential_ms_per_step": 1e3 * e2e_seq / args.steps}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1); its
    # whole-batch run is on the input of the pipelined run's last batch, whose
    # outputs are then checked against it
    parity_ok = True
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _, held_out, held_b = max(held, key=lambda h: h[0])
        rate, dt, rows = cpu_oracle_rate(wl, xs_host[held_b])
        threads = host_threads()
        rate_all, dt_all, tables = cpu_oracle_all_cores(wl, xs_host[held_b], threads)
        line["parity"] = dict(check_outputs(wl, xs_host[held_b], held_out, tables), batch=held_b,
                              what="the last timed batch of the pipelined run against the oracle")
        parity_ok = line["parity"]["ok"]
        line["cpu_baseline"] = {"value": rate_all, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"the whole batch ({wl.dms.size} DM trials), dedispersion + S/N, DM rows "
                                          f"split over {threads} threads: {dt_all:.1f} s",
                                "single_thread": {"value": rate, "unit": UNIT, "cores": 1,
                                                  "sample": f"{rows} of {wl.dms.size} DM trials, full batch, "
                                                            f"{dt:.1f} s"},
                                "cpu": cpu_model()}
        tiny_rate, tiny_s = cpu_oracle_tiny()
        line["cpu_baseline"]["tiny_single_thread"] = {
            "value": tiny_rate, "unit": UNIT, "cores": 1,
            "sample": f"the tiny 64-channel search (32 DM trials x 4096 samples, 4 widths), {1e3 * tiny_s:.1f} ms"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if not parity_ok:
        sys.exit("bench: the timed run's outputs differ from the oracle")
    if not line.get("subband", {}).get("pipelined", {}).get("outputs_equal_own_search", True):
        sys.exit("bench: the streamed two-step path's outputs differ from a search of the same input")


if __name__ == "__main__":
    main()
