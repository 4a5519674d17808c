"""Real-time serving study on the GPU: streaming beams through `sps_server_*`
against plain per-beam processing (Sec. 1: each beam's 1.024 s of data must be
searched within 1.024 s).

    python -m paper_1811_04165_gb300.serve_study [--duration 8] [--out FILE]

Beams alternate 1536 and 384 channels (1250-1550 MHz, 81.92 us, 12500-sample
batches), DM trials uniform in 1024..4096 (multiples of 32) with steps of
0.1-0.3, widths 1..64.  Each beam's batches arrive as a Poisson process of mean
interval `period` (1.024 s in real time), each delivered with a uniform jitter
of +-50 ms; a batch's latency is its completion time (GPU timeline, host
clock) minus its arrival.  Two servers: `served` dispatches up to 8 batches at
once (each beam in order), `per_beam` one batch at a time in arrival order.
Beyond the real-time runs (12-96 beams), the arrival period is compressed with
96 beams admitted, which emulates 96 x 1.024 s / period beams; the largest
emulated count whose p99 latency stays within its period is the real-time beam
capacity.  Inputs are host-pinned noise (latency does not depend on values).
"""
import argparse
import json
import sys
import time

import numpy as np

from . import Plan, Server, synth

DEADLINE_S = 1.024
JITTER_S = 0.050


def serve_beams(n, seed=5):
    rng = np.random.Generator(np.random.PCG64(seed + 31337))
    out = []
    for b in range(n):
        ch = 1536 if b % 2 == 0 else 384
        n_dm = int(rng.integers(32, 129)) * 32
        step = round(float(rng.uniform(0.1, 0.3)), 2)
        out.append(synth.Workload(f"serve{b}-{ch}ch-{n_dm}dm-step{step}", ch, 1250.0, 1550.0, 81.92e-6, 12500,
                                  synth.dm_grid(n_dm, step), np.array([1, 2, 4, 8, 16, 32, 64], np.int32),
                                  seed=seed * 1000 + b))
    return out


def arrivals(n_beams, period, duration, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    ev = []
    for b in range(n_beams):
        t = float(rng.exponential(period))
        while t < duration:
            ev.append((max(0.0, t + float(rng.uniform(-JITTER_S, JITTER_S)) * period / DEADLINE_S), b))
            t += float(rng.exponential(period))
    ev.sort()
    return ev


def run(plans, host_x, period, duration, inflight, seed, budget):
    import torch
    srv = Server(budget, max_inflight=inflight)
    ids = [srv.add_beam(p) for p in plans]
    snr = [torch.empty((p.n_widths, p.n_dms), dtype=torch.float64).pin_memory() for p in plans]
    best = [torch.empty(4, dtype=torch.int32).pin_memory() for _ in plans]
    # warm-up: one batch per beam, drained
    for b, p in enumerate(plans):
        srv.submit(ids[b], host_x[p.channels], snr[b], best[b], tag=b)
    while srv.pending():
        srv.poll()
    ev = arrivals(len(plans), period, duration, seed)
    t0 = Server.clock() + 0.2
    arrive, done = {}, {}
    for k, (t, b) in enumerate(ev):
        due = t0 + t
        while Server.clock() < due:
            for c in srv.poll():
                done[c.tag] = c.done_s
        tag = 1_000_000 + k
        arrive[tag] = due
        srv.submit(ids[b], host_x[plans[b].channels], snr[b], best[b], tag=tag)
    while srv.pending():
        for c in srv.poll():
            done[c.tag] = c.done_s
    for c in srv.poll():
        done[c.tag] = c.done_s
    lat = np.array([done[t] - arrive[t] for t in arrive])
    span = max(done.values()) - t0
    return {"batches": int(lat.size), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "max_s": float(lat.max()), "over_period": float(np.mean(lat > period)),
            "dm_trial_samples_per_s": float(sum(plans[b].n_dms * plans[b].n_samples for _, b in ev) / span)}


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--duration", type=float, default=8.0, help="seconds of arrivals per run (real-time runs)")
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    budget = int(a.budget_gb * 2 ** 30)
    wls = serve_beams(96)
    plans = [Plan.from_workload(wl) for wl in wls]
    rng = np.random.Generator(np.random.PCG64(1))
    host_x = {ch: torch.from_numpy(np.clip(np.rint(128 + 16 * rng.standard_normal((ch, 12500))), 0, 255)
                                   .astype(np.uint8)).pin_memory() for ch in (384, 1536)}
    res = {"real_time": {}, "compressed": {}}
    for n in (12, 24, 48, 96):
        for mode, inflight in (("served", 8), ("per_beam", 1)):
            res["real_time"][f"{n}/{mode}"] = run(plans[:n], host_x, DEADLINE_S, a.duration, inflight, seed=n,
                                                  budget=budget)
    capacity = {}
    for period in (0.256, 0.128, 0.112, 0.096, 0.085, 0.075, 0.064, 0.032):
        emulated = int(round(96 * DEADLINE_S / period))
        for mode, inflight in (("served", 8), ("per_beam", 1)):
            r = run(plans, host_x, period, a.duration * period / DEADLINE_S * 4, inflight, seed=emulated,
                    budget=budget)
            r["period_s"] = period
            r["emulated_beams"] = emulated
            res["compressed"][f"{emulated}/{mode}"] = r
            if r["p99_s"] <= period:
                capacity[mode] = max(capacity.get(mode, 0), emulated)
    res["real_time_beam_capacity"] = capacity
    text = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")
    print(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
