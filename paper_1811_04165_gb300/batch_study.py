"""Batched beams on the GPU: 40 beams in one CUDA-graph launch against plain
per-beam launches.

    python -m paper_1811_04165_gb300.batch_study [--beams 40] [--tune-evals 60] [--out FILE]

The beams (``synth.batch_beams``): 1.024 s batches of 12500 samples, alternately
1536 and 384 channels over 1250-1550 MHz, 512-4096 DM trials with steps of
0.1-0.5, the first 1-7 boxcar widths of 1..64, two pulses each.  Kernel tiles
per channel count come from a live GA run (`sps_tune`, full gene space, Sec. 4)
on the beam of that shape with the most DM trials, under a workspace bound;
beams whose tables do not fit the tuned tiles keep their defaults.  Timing:
CUDA events around whole batches, inputs larger than L2.  Every beam's batched
outputs are checked equal to its own search.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

from . import SPACE_FULL, TUNE_GA, Batch, Plan, SpsError, batch_workspace_bytes, search_desc, sps_tune, synth


def _inputs(plans, wls):
    import torch
    xs = []
    for p, wl in zip(plans, wls):
        x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, p.input_samples, wl.seed, wl.pulses,
                             pitch=p.pitch)
        xs.append(torch.from_numpy(x).cuda())
    return xs


def _time(fn, n, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


# GA-tuned configurations per channel count for the batched-beam mix, written
# by `--save-tuned` on a GB300 (applied where a beam's tables fit them).
TUNED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned", "gb300_batch_beams_configs.json")


def apply_tuned(plans, path=TUNED):
    """Put each plan on the stored tuned configuration of its channel count
    where that configuration fits it; returns how many plans took one."""
    from . import DedispConfig, KernelConfig, SnrConfig
    with open(path) as f:
        cfgs = json.load(f)["configs"]
    n = 0
    for p in plans:
        c = cfgs.get(str(p.channels))
        if c is None:
            continue
        k = KernelConfig()
        for name in ("brute", "step1", "step2"):
            setattr(k, name, DedispConfig(*c[name]))
        k.snr = SnrConfig(*c["snr"])
        try:
            p.config = k
            n += 1
        except SpsError:
            pass
    return n


def tune_shapes(plans, wls, xs, evals, ws_limit):
    """GA-tuned configuration per channel count, applied where it fits."""
    import torch
    out = {}
    for ch in sorted({wl.channels for wl in wls}):
        idx = [b for b, wl in enumerate(wls) if wl.channels == ch]
        rep = max(idx, key=lambda b: wls[b].dms.size)
        p = plans[rep]
        ws = torch.empty(ws_limit, dtype=torch.uint8, device="cuda")
        t0 = time.perf_counter()
        best, res, trace = sps_tune(p, xs[rep], which=SPACE_FULL, workspace=ws,
                                    desc=search_desc(algorithm=TUNE_GA, max_evaluations=evals, seed=ch), reps=1)
        del ws
        cfg = p.config
        applied = 0
        for b in idx:
            try:
                plans[b].config = cfg
                applied += 1
            except SpsError:
                pass
        out[str(ch)] = {"tuned_on": wls[rep].name, "evaluations": res.evaluations, "best_ms": res.best_fitness,
                        "seconds": time.perf_counter() - t0, "config": cfg.as_dict(), "applied_to": applied,
                        "beams": len(idx)}
    return out


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--beams", type=int, default=40)
    ap.add_argument("--tune-evals", type=int, default=60, help="0 keeps the default configurations")
    ap.add_argument("--ws-limit-gb", type=float, default=1.0, help="workspace bound per beam while tuning")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--batch-ws-gb", type=float, default=48.0, help="largest batch workspace to allocate")
    ap.add_argument("--out", default=None)
    ap.add_argument("--save-tuned", default=None, metavar="FILE",
                    help="write the tuned configuration per channel count (JSON) for later batches")
    a = ap.parse_args(argv)
    wls = synth.batch_beams(a.beams)
    t0 = time.perf_counter()
    plans = [Plan.from_workload(wl) for wl in wls]
    t_plan = time.perf_counter() - t0
    xs = _inputs(plans, wls)
    res = {"beams": len(wls), "channels": sorted({wl.channels for wl in wls}),
           "dm_trial_samples": int(sum(wl.dm_trial_samples for wl in wls)), "plan_s": t_plan}
    ws_limit = int(a.ws_limit_gb * 2 ** 30)
    if a.tune_evals:
        res["tuning"] = tune_shapes(plans, wls, xs, a.tune_evals, ws_limit)
        if a.save_tuned:
            import torch
            with open(a.save_tuned, "w") as f:
                json.dump({"how": "python -m paper_1811_04165_gb300.batch_study (live GA, full space, "
                                  f"{a.tune_evals} evaluations per channel count)",
                           "gpu": torch.cuda.get_device_name(), "workload": "batched beams (synth.batch_beams)",
                           "configs": {ch: r["config"] for ch, r in res["tuning"].items()}}, f, indent=1)
    # plain per-beam launches on one stream, one workspace sized for the largest beam
    res["workspace_gb_per_beam_max"] = max(batch_workspace_bytes([p], 1) for p in plans) / 2 ** 30
    ws = torch.empty(max(batch_workspace_bytes([p], 1) for p in plans), dtype=torch.uint8, device="cuda")
    outs = [p.alloc_outputs() for p in plans]

    def per_beam():
        for p, x, o in zip(plans, xs, outs):
            p.search(x, out=o, workspace=ws)

    t_beam = _time(per_beam, a.reps)
    ref = [{k: v.clone() for k, v in o.items()} for o in outs]
    del ws
    samples = res["dm_trial_samples"]
    res["per_beam"] = {"ms_per_batch": t_beam, "dm_trial_samples_per_s": samples / (t_beam * 1e-3)}
    res["batched"] = {}
    for branches in (1, 4, 8, 16):
        need = batch_workspace_bytes(plans, branches)
        if need > a.batch_ws_gb * 2 ** 30:
            res["batched"][str(branches)] = {"skipped": f"workspace {need / 2 ** 30:.1f} GB over the bound"}
            continue
        batch = Batch(plans, xs, branches=branches)
        t = _time(batch.launch, a.reps)
        exact = all(torch.equal(o[k], r[k]) for o, r in zip(batch.outs, ref) for k in ("D", "snr", "peak_t",
                                                                                        "peak_val", "best"))
        res["batched"][str(branches)] = {"ms_per_batch": t, "dm_trial_samples_per_s": samples / (t * 1e-3),
                                         "speedup_vs_per_beam": t_beam / t, "exact": exact,
                                         "workspace_gb": batch.workspace.numel() / 2 ** 30,
                                         "real_time_beams": len(wls) * 1024.0 / t}
        del batch
        torch.cuda.empty_cache()
    text = json.dumps(res, indent=1, default=lambda v: v.item() if hasattr(v, "item") else str(v))
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")
    print(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
