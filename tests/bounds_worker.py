"""Runs the de-dispersion paths on the bounds-checked build of the library and
prints one JSON line: per case, the plan's status word (the bounds bit is set
when a pass would have read outside a shared-memory stage) and whether the
result equals the oracle.  Started by tests/test_gpu_bounds.py in a process of
its own with SPS_BUILD=checked, so that this process loads libsps_checked.so."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import paper_1811_04165_gb300 as sps  # noqa: E402
from paper_1811_04165_gb300 import _lib, synth  # noqa: E402
from tests import oracle_rows  # noqa: E402

# the brute-force configurations of the ragged parity test: single channels, pairs, quads
CONFIGS = [
    (1, 4, 1, 1, 2, 0), (1, 8, 2, 2, 6, 0), (2, 4, 4, 2, 16, 0), (2, 16, 2, 1, 32, 0), (4, 4, 2, 2, 10, 0),
    (4, 8, 4, 2, 16, 0), (4, 16, 8, 1, 16, 0), (8, 4, 2, 4, 8, 0), (8, 8, 1, 8, 6, 0), (1, 32, 16, 1, 4, 0),
    (1, 4, 1, 1, 2, 1), (1, 8, 2, 2, 6, 1), (2, 4, 4, 2, 16, 1), (2, 32, 2, 1, 8, 1), (4, 16, 8, 1, 8, 1),
    (8, 4, 2, 4, 8, 1), (8, 8, 4, 2, 4, 1), (1, 32, 16, 1, 4, 1),
    (1, 4, 1, 1, 2, 2), (1, 8, 2, 2, 8, 2), (2, 4, 4, 2, 16, 2), (2, 32, 2, 1, 8, 2), (4, 16, 8, 1, 4, 2),
    (8, 4, 2, 4, 8, 2), (8, 8, 4, 2, 4, 2), (1, 32, 16, 1, 4, 2),
]


def main():
    assert _lib.lib_path().endswith("libsps_checked.so"), _lib.lib_path()
    res = {}

    # ragged shapes: 37 channels, 29 DM trials, 1003 samples, every kernel configuration above
    for cfg in CONFIGS:
        dms = synth.dm_grid(29, 0.31 if cfg[5] else 3.1)
        p = sps.Plan(37, 1300.0, 1500.0, 65.536e-6, 1003, dms, [1, 3, 8, 50])
        c = p.config
        c.brute = sps.DedispConfig(*cfg)
        p.config = c
        x = synth.filterbank(37, 1300.0, 1500.0, 65.536e-6, p.input_samples, 99, pitch=p.pitch + 32)
        D = torch.full((29, 1003), -7, dtype=torch.int32, device="cuda")
        sps.sps_dedisperse(p, torch.from_numpy(x).cuda(), D)
        torch.cuda.synchronize()
        want = oracle.dedisperse(x, oracle.delay_table(1300.0, 1500.0, 37, 65.536e-6, dms), 1003)
        res["ragged" + ",".join(map(str, cfg))] = {"status": p.status(), "ok": bool(np.array_equal(D.cpu().numpy(), want))}

    # the beam, brute force on each kernel (single channels, pairs, quads), every row
    wl = synth.apertif_beam()
    delays = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    for presum in (0, 1, 2):
        p = sps.Plan.from_workload(wl, mode=sps.MODE_BRUTE)
        c = p.config
        c.brute.presum = presum
        p.config = c
        x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, p.input_samples, wl.seed, wl.pulses,
                             pitch=p.pitch)
        out = p.search(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        want = oracle_rows.dedisperse(x, delays, wl.n_t)
        res[f"beam_presum{presum}"] = {"status": p.status(), "ok": bool(np.array_equal(out["D"].cpu().numpy(), want))}

    # the beam's two-step path (32 subbands): step one on single channels, step two
    wls = synth.apertif_beam(subband=True)
    p = sps.Plan.from_workload(wls)
    x = synth.filterbank(wls.channels, wls.f_lo, wls.f_hi, wls.t_samp, p.input_samples, wls.seed, wls.pulses,
                         pitch=p.pitch)
    out = p.search(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    d1, d2 = oracle.subband_tables(wls.f_lo, wls.f_hi, wls.channels, wls.t_samp, wls.n_subbands, wls.coarse_dms,
                                   wls.dms)
    n_1, _ = oracle.subband_lengths(wls.n_t, d1, d2)
    Y = oracle_rows.subband_step1(x, d1, wls.n_subbands, n_1)
    Do = oracle_rows.subband_step2(Y, d2, oracle.coarse_index(wls.dms.size, wls.coarse_dms.size), wls.n_t)
    res["beam_subband32"] = {"status": p.status(), "ok": bool(np.array_equal(out["D"].cpu().numpy(), Do))}

    # batched beams: pre-summed beams share one pass launch (the work-list kernel)
    wlb = synth.batch_beams(4, seed=9, n_t=2000, channels=(96, 48), dm_trials=(64, 256), dm_steps=(0.1, 0.2),
                            max_widths=4)
    plans = [sps.Plan.from_workload(w) for w in wlb]
    xs = []
    for pb, w in zip(plans, wlb):
        c = pb.config
        c.brute = sps.DedispConfig(4, 16, 8, 1, 8, 2)
        pb.config = c
        xs.append(torch.from_numpy(synth.filterbank(w.channels, w.f_lo, w.f_hi, w.t_samp, pb.input_samples, w.seed,
                                                    w.pulses, pitch=pb.pitch)).cuda())
    batch = sps.Batch(plans, xs, branches=2)
    batch.launch()
    torch.cuda.synchronize()
    for b, (pb, w, xb, o) in enumerate(zip(plans, wlb, xs, batch.outs)):
        want = oracle.dedisperse(xb.cpu().numpy(), oracle.delay_table(w.f_lo, w.f_hi, w.channels, w.t_samp, w.dms),
                                 w.n_t)
        res[f"batch{b}"] = {"status": pb.status(), "ok": bool(np.array_equal(o["D"].cpu().numpy(), want))}
    print("RESULT " + json.dumps(res))


if __name__ == "__main__":
    main()
