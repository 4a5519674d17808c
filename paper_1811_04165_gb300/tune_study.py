"""Auto-tuning study on the GPU (Sec. 4 and Sec. 5; the analogue of Figs. 3-5).

    python -m paper_1811_04165_gb300.tune_study [--seeds 50] [--budget 500] [--beam-evals 200] [--out FILE]

1. The tiny 64-channel search in two-step subband mode, reduced joint space of
   5000 points (step one warps_dm x chunk, step two dms_per_thread x warps_dm x
   chunk, S/N threads): every point is timed live (exhaustive search), giving
   the exact optimum and a fitness table.
2. On that table, the library's GA (population 32, tournament pools of 20 %,
   uniform crossover p_cross 0.8, mutation 0.1) and pure random search run with
   equal budgets of distinct evaluations over many seeds: best-of-run relative
   to the optimum, the share of runs within 5 %, and the spread (coefficient
   of variation) of the best fitness over runs.
3. Sweeps of p_mut, p_cross, population, crossover kind and budget on the same
   table (Fig. 3), a histogram of the GA's best over seeds (Fig. 5), and the
   convergence diagnostic of Sec. 5 (Fig. 4): per gene, the coefficient of
   variation c_v = sigma / mu of the parameter over a run's 20 end
   configurations, averaged over 30 GA and 30 random-search runs.
4. One live GA run on the tiny plan, and one on the 1536-channel Apertif beam's
   full brute-force gene space (7 genes), against the library's default
   configuration.

Everything runs through the C ABI (`sps_tune`, `sps_optimize`); fitness is the
median over three trials of the mean time of back-to-back searches.
"""
import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

from . import (CROSS_ONE_POINT, CROSS_UNIFORM, SPACE_FULL, SPACE_REDUCED, TUNE_EXHAUSTIVE, TUNE_GA, TUNE_RANDOM,
               Plan, search_desc, sps_optimize, sps_tune, sps_tune_config, sps_tune_space, synth)


def tiny_subband():
    """The tiny search (64 ch, 4096 samples, 32 DMs 0..62) in subband mode: 8
    subbands, 4 coarse DMs (0, 16, 32, 48)."""
    wl = synth.tiny_brute()
    wl.n_subbands = 8
    wl.coarse_dms = wl.dms[::8].copy()
    wl.name = "tiny-64ch-4096s-32dm-subband8"
    return wl


def _input(plan, wl):
    import torch
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, plan.input_samples, wl.seed, wl.pulses,
                         pitch=plan.pitch)
    return torch.from_numpy(x).cuda()


def _runs(nv, ko, table, algorithm, seeds, budget, valid=None, **kw):
    best = []
    for s in seeds:
        _, res, _ = sps_optimize(nv, ko, table.__getitem__, valid,
                                 search_desc(algorithm=algorithm, max_evaluations=budget, seed=s, **kw))
        best.append(res.best_fitness)
    return best


GENE_NAMES = {0: ("dms_per_thread", "samples_per_thread", "warps_dm", "warps_time", "chunk", "presum"),
              1: ("dms_per_thread", "samples_per_thread", "warps_dm", "warps_time", "chunk")}


def gene_cv(end_configurations, values):
    """Sec. 5: per gene, sigma / mu of the parameter values over the end
    configurations (population standard deviation); None for a zero mean."""
    out = []
    for g, vals in enumerate(values):
        v = [float(vals[p[g]]) for p in end_configurations]
        mu = statistics.fmean(v)
        out.append(None if mu == 0 else statistics.pstdev(v) / mu)
    return out


def _cv_study(nv, ko, table, values, names, seeds, budget, population=20):
    """Averaged per-gene c_v of GA and random search (genes with one value left out)."""
    res_all = {}
    for name, alg in (("ga", TUNE_GA), ("random", TUNE_RANDOM)):
        per_run = []
        for s in seeds:
            _, res, _ = sps_optimize(nv, ko, table.__getitem__, None,
                                     search_desc(algorithm=alg, max_evaluations=budget, seed=s,
                                                 population=population))
            per_run.append(gene_cv(res.final_population, values))
        res_all[name] = {names[g]: statistics.fmean(r[g] for r in per_run if r[g] is not None)
                         for g in range(len(values)) if len(values[g]) > 1}
    return res_all


def _summary(best, opt):
    r = [b / opt for b in best]
    mean = statistics.fmean(best)
    return {"runs": len(r), "mean_ratio": statistics.fmean(r), "median_ratio": statistics.median(r),
            "worst_ratio": max(r), "within_5pct": sum(x <= 1.05 for x in r) / len(r),
            "cv": statistics.pstdev(best) / mean if mean > 0 else 0.0}


def study_table(seeds, budget, reps):
    import torch
    wl = tiny_subband()
    plan = Plan.from_workload(wl)
    x = _input(plan, wl)
    nv, ko, values = sps_tune_space(plan, SPACE_REDUCED)
    t0 = time.perf_counter()
    _, res, trace = sps_tune(plan, x, which=SPACE_REDUCED, desc=search_desc(algorithm=TUNE_EXHAUSTIVE), reps=reps)
    torch.cuda.synchronize()
    t_exh = time.perf_counter() - t0
    table = {pt: f for pt, f in trace}
    finite = [f for f in table.values() if np.isfinite(f)]
    opt = min(finite)
    out = {"workload": wl.name, "space": "reduced", "points": int(np.prod(nv)), "valid": len(finite),
           "exhaustive_s": t_exh, "optimum_ms": opt, "median_ms": statistics.median(finite),
           "worst_ms": max(finite), "budget": budget}
    seeds = list(seeds)
    ga = _runs(nv, ko, table, TUNE_GA, seeds, budget)
    rnd = _runs(nv, ko, table, TUNE_RANDOM, seeds, budget)
    out["ga"] = _summary(ga, opt)
    out["random"] = _summary(rnd, opt)
    # Fig. 5 analogue: histogram of the GA's best relative to the optimum
    edges = [1.0, 1.01, 1.02, 1.05, 1.1, 1.2, 1.5, float("inf")]
    h = np.histogram([b / opt for b in ga], bins=edges)[0]
    out["ga_histogram"] = {f"[{edges[i]:.2f},{edges[i + 1]:.2f})": int(h[i]) for i in range(len(h))}
    # Fig. 4 analogue: per-gene c_v over 20 end configurations, 30 runs each
    kernel_names = ("step1", "step2", "snr")
    names, field = [], {}
    for g, k in enumerate(ko):
        j = field.get(k, 0)
        field[k] = j + 1
        names.append(f"{kernel_names[k]}.threads" if k == 2 else f"{kernel_names[k]}.{GENE_NAMES[k][j]}")
    out["gene_cv"] = _cv_study(nv, ko, table, values, names, list(range(30)), budget)
    # Fig. 3 analogue: sweeps on the same table, 20 seeds each
    sw = seeds[:20]
    sweeps = {}
    for p in (0.05, 0.1, 0.2, 0.4):
        sweeps[f"p_mut={p}"] = _summary(_runs(nv, ko, table, TUNE_GA, sw, budget, p_mut=p), opt)["mean_ratio"]
    for p in (0.5, 0.8, 1.0):
        sweeps[f"p_cross={p}"] = _summary(_runs(nv, ko, table, TUNE_GA, sw, budget, p_cross=p), opt)["mean_ratio"]
    for n in (16, 32, 64):
        sweeps[f"population={n}"] = _summary(_runs(nv, ko, table, TUNE_GA, sw, budget, population=n),
                                             opt)["mean_ratio"]
    for name, c in (("uniform", CROSS_UNIFORM), ("one_point", CROSS_ONE_POINT)):
        sweeps[f"crossover={name}"] = _summary(_runs(nv, ko, table, TUNE_GA, sw, budget, crossover=c),
                                               opt)["mean_ratio"]
    for b in (100, 250, 500, 1000):
        sweeps[f"budget={b}/ga"] = _summary(_runs(nv, ko, table, TUNE_GA, sw, b), opt)["mean_ratio"]
        sweeps[f"budget={b}/random"] = _summary(_runs(nv, ko, table, TUNE_RANDOM, sw, b), opt)["mean_ratio"]
    out["sweeps_mean_ratio"] = sweeps
    # one live GA run with the same budget: its configuration's table time vs the optimum
    best, res, tr = sps_tune(plan, x, which=SPACE_REDUCED,
                             desc=search_desc(algorithm=TUNE_GA, max_evaluations=budget, seed=seeds[0]), reps=reps)
    out["live_ga"] = {"evaluations": res.evaluations, "best_ms_live": res.best_fitness,
                      "best_ms_in_table": table[tuple(best)], "ratio_in_table": table[tuple(best)] / opt}
    return out


def study_beam(evals, reps, seed):
    import torch
    wl = synth.apertif_beam()
    plan = Plan.from_workload(wl)
    x = _input(plan, wl)
    default = plan.config
    out_buf = plan.alloc_outputs()
    ws = plan.workspace()

    def time_cfg(n=20):
        for _ in range(3):
            plan.search(x, out=out_buf, workspace=ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            plan.search(x, out=out_buf, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    t_default = time_cfg()
    nv, ko, _ = sps_tune_space(plan, SPACE_FULL)
    t0 = time.perf_counter()
    best, res, trace = sps_tune(plan, x, which=SPACE_FULL, out=out_buf, workspace=ws,
                                desc=search_desc(algorithm=TUNE_GA, max_evaluations=evals, seed=seed), reps=reps)
    t_ga = time.perf_counter() - t0
    cfg = sps_tune_config(plan, SPACE_FULL, best)
    t_best = time_cfg()
    plan.config = default
    return {"workload": wl.name, "space": "full brute-force (7 genes)", "points": int(np.prod(nv)),
            "evaluations": res.evaluations, "finite": int(sum(bool(np.isfinite(f)) for _, f in trace)), "ga_s": t_ga,
            "default_config": default.as_dict(), "default_ms": t_default, "ga_config": cfg.as_dict(),
            "ga_ms": t_best, "speedup": t_default / t_best}


def study_beam_table(seeds, budget_frac, reps, table_out=None):
    """The bench's workload (the Apertif beam, brute force) over its reduced
    joint space: every valid point timed live (exhaustive search), then GA and
    random search on that table at `budget_frac` of its valid points over
    `seeds`, and the library's default configuration placed in the table."""
    import torch
    wl = synth.apertif_beam()
    plan = Plan.from_workload(wl)
    x = _input(plan, wl)
    default = plan.config
    nv, ko, values = sps_tune_space(plan, SPACE_REDUCED)
    t0 = time.perf_counter()
    _, res, trace = sps_tune(plan, x, which=SPACE_REDUCED, desc=search_desc(algorithm=TUNE_EXHAUSTIVE), reps=reps)
    torch.cuda.synchronize()
    t_exh = time.perf_counter() - t0
    plan.config = default
    table = {tuple(int(v) for v in pt): float(f) for pt, f in trace}
    finite = {pt: f for pt, f in table.items() if np.isfinite(f)}
    opt_pt = min(finite, key=finite.get)
    opt = finite[opt_pt]
    # the default configuration's point in the space (None if it lies outside)
    default_pt = None
    for pt in finite:
        if sps_tune_config(plan, SPACE_REDUCED, pt).as_dict() == default.as_dict():
            default_pt = pt
            break
    budget = max(1, int(budget_frac * len(finite)))
    seeds = list(seeds)
    # the searches see the plan's boundary conditions: the points the exhaustive search visited
    valid = table.__contains__
    ga = _runs(nv, ko, table, TUNE_GA, seeds, budget, valid)
    rnd = _runs(nv, ko, table, TUNE_RANDOM, seeds, budget, valid)
    ga0 = _runs(nv, ko, table, TUNE_GA, seeds, budget, valid, renew=0)
    out = {"workload": wl.name, "space": "reduced brute force", "genes": [list(map(int, v)) for v in values],
           "points": int(np.prod(nv)), "valid": len(finite), "exhaustive_s": t_exh, "reps": reps,
           "optimum_ms": opt, "optimum_config": sps_tune_config(plan, SPACE_REDUCED, opt_pt).as_dict(),
           "median_ms": statistics.median(finite.values()), "worst_ms": max(finite.values()), "budget": budget,
           "default_ms": finite.get(default_pt) if default_pt is not None else None,
           "default_ratio": finite[default_pt] / opt if default_pt is not None else None,
           "ga": _summary(ga, opt), "random": _summary(rnd, opt), "ga_without_renewal": _summary(ga0, opt)}
    if table_out:
        with open(table_out, "w") as f:
            json.dump({"how": "python -m paper_1811_04165_gb300.tune_study --beam-table (sps_tune, exhaustive "
                              f"search of the reduced space, reps={reps}, median of three trials per point)",
                       "gpu": torch.cuda.get_device_name(), "workload": wl.name, "n_values": [int(v) for v in nv],
                       "kernel_of": [int(k) for k in ko], "values": out["genes"],
                       "default_point": list(default_pt) if default_pt is not None else None,
                       "points": [[list(pt), (f if np.isfinite(f) else None)] for pt, f in table.items()]}, f)
    return out


def study_subband_joint(subbands=(16, 32, 64), evals=300, reps=2, seed=1):
    """The beam's two-step path with the subband count as one more gene (the
    joint space of step one, step two and S/N genes times S): the library GA
    (sps_optimize) over it with live fitness -- the median over three trials of
    the mean time of `reps` searches -- against random search at the same
    budget.  Each S is its own plan (its own delay tables, and so its own
    exact result); points a plan rejects are invalid."""
    import torch
    plans = {}
    for S in subbands:
        wl = synth.apertif_beam(subband=True)
        wl.n_subbands = S
        plans[S] = Plan.from_workload(wl)
    pitch = max(p.pitch for p in plans.values())
    wl = synth.apertif_beam()
    x = torch.from_numpy(synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, pitch, wl.seed, wl.pulses,
                                          pitch=pitch)).cuda()
    nv0, ko0, values0 = sps_tune_space(plans[subbands[0]], SPACE_REDUCED)
    nv = [len(subbands)] + [int(v) for v in nv0]
    ko = [0] + [int(k) + 1 for k in ko0]
    outs = {S: p.alloc_outputs() for S, p in plans.items()}
    wss = {S: p.workspace() for S, p in plans.items()}
    defaults = {S: p.config for S, p in plans.items()}

    def config_of(pt):
        S = subbands[pt[0]]
        return S, sps_tune_config(plans[S], SPACE_REDUCED, list(pt[1:]))

    def valid(pt):
        try:
            config_of(pt)
            return True
        except Exception:
            return False

    def fitness(pt):
        S, cfg = config_of(pt)
        p = plans[S]
        p.config = cfg
        o, ws = outs[S], wss[S]
        p.search(x, out=o, workspace=ws)
        trials = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                p.search(x, out=o, workspace=ws)
            e1.record()
            torch.cuda.synchronize()
            trials.append(e0.elapsed_time(e1) / reps)
        return sorted(trials)[1]

    res = {"workload": "apertif-1536ch-12500s-2048dm two-step", "subbands": list(subbands),
           "genes": ["subbands"] + [f"gene{g}" for g in range(len(nv0))], "points": int(np.prod(nv)),
           "budget": evals}
    for name, alg in (("ga", TUNE_GA), ("random", TUNE_RANDOM)):
        t0 = time.perf_counter()
        best, r, trace = sps_optimize(nv, ko, fitness, valid,
                                      search_desc(algorithm=alg, max_evaluations=evals, seed=seed))
        S, cfg = config_of(best)
        by_s = {}
        for pt, f in trace:
            if np.isfinite(f):
                by_s.setdefault(subbands[pt[0]], []).append(f)
        res[name] = {"best_ms": r.best_fitness, "subbands": S, "config": cfg.as_dict(), "evaluations": r.evaluations,
                     "seconds": time.perf_counter() - t0,
                     "best_ms_per_subbands": {str(k): min(v) for k, v in by_s.items()}}
    for S, p in plans.items():
        p.config = defaults[S]
    res["default_ms"] = {str(S): fitness([i] + list(_point_of(plans[S], defaults[S], values0)))
                         for i, S in enumerate(subbands)
                         if _point_of(plans[S], defaults[S], values0) is not None}
    return res


def _point_of(plan, cfg, values):
    """The reduced-space point of a configuration, or None if it lies outside."""
    for pt in np.ndindex(*[len(v) for v in values]):
        try:
            if sps_tune_config(plan, SPACE_REDUCED, list(pt)).as_dict() == cfg.as_dict():
                return pt
        except Exception:
            continue
    return None


# The committed table of the beam's reduced brute-force space (written by
# `--beam-table`): every valid point's live fitness on a GB300.
BEAM_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned", "gb300_apertif_brute_reduced.json")


def load_table(path):
    """A fitness table written by study_beam_table: {n_values, kernel_of,
    values, default_point, table {point: ms (inf for a failed run)}, optimum_point,
    optimum_ms, ...}; points outside `table` break the plan's boundary conditions."""
    with open(path) as f:
        rec = json.load(f)
    table = {tuple(p): (float("inf") if v is None else float(v)) for p, v in rec["points"]}
    finite = {p: v for p, v in table.items() if np.isfinite(v)}
    opt = min(finite, key=finite.get)
    rec["table"] = table
    rec["optimum_point"] = list(opt)
    rec["optimum_ms"] = finite[opt]
    rec["valid"] = len(table)
    return rec


def replay(rec, seeds, budget_frac=0.1):
    """GA and random search on a stored table at `budget_frac` of its valid
    points: best-of-run relative to the table's optimum, and the default
    configuration's ratio."""
    table, nv, ko = rec["table"], rec["n_values"], rec["kernel_of"]
    budget = max(1, int(budget_frac * len(table)))
    valid = table.__contains__
    opt = rec["optimum_ms"]
    seeds = list(seeds)
    out = {"table": os.path.basename(rec.get("path", "")) or "stored", "gpu": rec.get("gpu"),
           "workload": rec.get("workload"), "valid_points": len(table), "budget": budget,
           "optimum_ms": opt, "ga": _summary(_runs(nv, ko, table, TUNE_GA, seeds, budget, valid), opt),
           "random": _summary(_runs(nv, ko, table, TUNE_RANDOM, seeds, budget, valid), opt)}
    dp = rec.get("default_point")
    out["default_ratio"] = table[tuple(dp)] / opt if dp is not None and tuple(dp) in table else None
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--seeds", type=int, default=50)
    ap.add_argument("--budget", type=int, default=500, help="distinct evaluations per search (10 % of 5000)")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--beam-evals", type=int, default=200, help="0 skips the live run on the beam")
    ap.add_argument("--out", default=None)
    ap.add_argument("--beam-table", default=None, metavar="FILE",
                    help="only the beam's reduced-space study; writes its fitness table to FILE")
    ap.add_argument("--subband-joint", type=int, default=0, metavar="EVALS",
                    help="only the two-step joint study with the subband count as a gene, EVALS per search")
    a = ap.parse_args(argv)
    if a.subband_joint:
        res = {"subband_joint": study_subband_joint(evals=a.subband_joint, reps=a.reps)}
        text = json.dumps(res, indent=1, default=lambda v: v.item() if hasattr(v, "item") else str(v))
        if a.out:
            with open(a.out, "w") as f:
                f.write(text + "\n")
        print(text)
        return 0
    if a.beam_table:
        res = {"apertif_beam_table": study_beam_table(range(a.seeds), 0.1, a.reps, a.beam_table)}
        text = json.dumps(res, indent=1, default=lambda v: v.item() if hasattr(v, "item") else str(v))
        if a.out:
            with open(a.out, "w") as f:
                f.write(text + "\n")
        print(text)
        return 0
    res = {"tiny_subband": study_table(range(a.seeds), a.budget, a.reps)}
    if a.beam_evals:
        res["apertif_beam"] = study_beam(a.beam_evals, a.reps, seed=1)
    text = json.dumps(res, indent=1, default=lambda v: v.item() if hasattr(v, "item") else str(v))
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")
    print(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
