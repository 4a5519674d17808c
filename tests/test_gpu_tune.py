"""Live auto-tuning on the GPU through the C ABI: the plan's gene space, the
mapping of points to kernel configurations, and GA / random / exhaustive
search with measured kernel time as fitness (Sec. 3.2, Sec. 4).  Every tuned
configuration must give the same (exact) results."""
import numpy as np
import pytest

from oracle import ga
from paper_1811_04165_gb300 import synth

pytestmark = pytest.mark.gpu


def tiny_subband():
    """The tiny 64-channel search run through the paper's two-step pipeline:
    8 subbands, 4 coarse DMs (0, 16, 32, 48) for the 32 trials."""
    wl = synth.tiny_brute()
    wl.n_subbands = 8
    wl.coarse_dms = wl.dms[::8].copy()
    wl.name = "tiny-64ch-4096s-32dm-subband8"
    return wl


def _setup(lib, wl):
    import torch
    p = lib.Plan.from_workload(wl)
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, p.input_samples, wl.seed, wl.pulses,
                         pitch=p.pitch)
    return p, torch.from_numpy(x).cuda()


def test_reduced_space_has_5000_valid_points(lib):
    p, _ = _setup(lib, tiny_subband())
    nv, ko, vals = lib.sps_tune_space(p, lib.SPACE_REDUCED)
    assert int(np.prod(nv)) == 5000 and list(ko) == sorted(ko)
    valid = 0
    for pt in np.ndindex(*nv):
        try:
            lib.sps_tune_config(p, lib.SPACE_REDUCED, pt)
            valid += 1
        except lib.SpsError:
            pass
    assert valid == 5000


def test_full_space_configs_map_and_validate(lib):
    p, _ = _setup(lib, synth.apertif_beam())
    nv, ko, vals = lib.sps_tune_space(p, lib.SPACE_FULL)
    assert len(nv) == 7 and list(ko) == [0, 0, 0, 0, 0, 0, 1]
    c = lib.sps_tune_config(p, lib.SPACE_FULL, [2, 2, 3, 0, 3, 1, 3])
    assert c.brute.as_tuple() == (4, 16, 8, 1, 16, 1) and c.snr.threads == 256
    with pytest.raises(lib.SpsError):  # 16 x 16 warps: too many threads
        lib.sps_tune_config(p, lib.SPACE_FULL, [0, 0, 4, 4, 0, 0, 0])


def test_live_ga_tuning_keeps_results_exact(lib):
    import torch
    wl = tiny_subband()
    p, x = _setup(lib, wl)
    want = p.search(x)
    torch.cuda.synchronize()
    ref = {k: v.clone() for k, v in want.items()}
    desc = lib.search_desc(algorithm=lib.TUNE_GA, population=8, max_evaluations=24, seed=3)
    best, res, trace = lib.sps_tune(p, x, which=lib.SPACE_FULL, desc=desc, reps=2)
    assert res.evaluations == len(trace) <= 24 and np.isfinite(res.best_fitness)
    assert res.best_fitness == min(f for _, f in trace)
    # the plan now runs the best configuration; results are unchanged
    cfg = lib.sps_tune_config(p, lib.SPACE_FULL, best)
    assert p.config.as_dict() == cfg.as_dict()
    got = p.search(x)
    torch.cuda.synchronize()
    for k in ("D", "peak_t", "peak_val", "best"):
        assert torch.equal(got[k], ref[k]), k
    assert torch.allclose(got["snr"], ref["snr"], rtol=1e-12, atol=0)


def test_exhaustive_reduced_space_and_ga_on_its_table(lib):
    """Config 3 in miniature: exhaustive search of the reduced 5000-point joint
    space with live timings, then GA and pure random search replayed on the
    measured table with equal budgets (10 % of the evaluations)."""
    wl = tiny_subband()
    p, x = _setup(lib, wl)
    desc = lib.search_desc(algorithm=lib.TUNE_EXHAUSTIVE)
    best, res, trace = lib.sps_tune(p, x, which=lib.SPACE_REDUCED, desc=desc, reps=2)
    assert res.evaluations == 5000 == len(trace)
    table = {pt: f for pt, f in trace}
    opt = min(table.values())
    assert res.best_fitness == opt and np.isfinite(opt)
    nv, ko, _ = lib.sps_tune_space(p, lib.SPACE_REDUCED)
    space = ga.Space(list(nv), list(ko))
    ga_best = [ga.genetic(space, table.__getitem__, n_pop=32, max_evaluations=500, seed=s).best_fitness
               for s in range(10)]
    rnd_best = [ga.random_search(space, table.__getitem__, max_evaluations=500, seed=s).best_fitness
                for s in range(10)]
    assert min(ga_best) >= opt and min(rnd_best) >= opt
    # the library's engine on the same table agrees with the oracle
    b, r, _ = lib.sps_optimize(nv, ko, table.__getitem__, None,
                               lib.search_desc(population=32, max_evaluations=500, seed=0))
    assert r.best_fitness == ga_best[0]


def test_live_tuning_log_resume_and_saved_config(lib, tmp_path):
    """A live GA writes its JSON-lines log; re-run with the log as known
    evaluations it replays them unmeasured (identical fitness values) and goes
    on; the tuned configuration saved as JSON loads into a plan of the same
    shape and is refused for another shape."""
    import json
    wl = tiny_subband()
    p, x = _setup(lib, wl)
    log1 = tmp_path / "live.jsonl"
    b1, r1, t1 = lib.sps_tune(p, x, which=lib.SPACE_REDUCED, reps=1, log=str(log1),
                              desc=lib.search_desc(max_evaluations=12, seed=3))
    known = lib.read_tuning_log(str(log1))
    assert known == t1 and r1.evaluations == len(t1)
    closing = json.loads(log1.read_text().splitlines()[-1])
    assert tuple(closing["best"]) == b1
    assert closing["config"] == {k: list(v) for k, v in p.config.as_dict().items()}
    b2, r2, t2 = lib.sps_tune(p, x, which=lib.SPACE_REDUCED, reps=1,
                              desc=lib.search_desc(max_evaluations=24, seed=3, known=known))
    assert t2[:len(known)] == known  # replayed from the log, not measured again
    assert r2.evaluations >= r1.evaluations and r2.best_fitness <= r1.best_fitness
    out = p.search(x)  # the plan is left on the best configuration and stays exact
    D = out["D"].cpu().numpy()
    xh = x.cpu().numpy()
    import oracle
    d1, d2 = oracle.subband_tables(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, 8, wl.coarse_dms, wl.dms)
    n_1, _ = oracle.subband_lengths(wl.n_t, d1, d2)
    want = oracle.subband_step2(oracle.subband_step1(xh, d1, 8, n_1), d2,
                                oracle.coarse_index(wl.dms.size, wl.coarse_dms.size), wl.n_t)
    assert np.array_equal(D, want)
    cfg = tmp_path / "tuned.json"
    p.save_config(str(cfg))
    q, _ = _setup(lib, tiny_subband())
    q.load_config(str(cfg))
    assert q.config.as_dict() == p.config.as_dict()
    other_wl = tiny_subband()
    other_wl.n_t = 2048
    other, _ = _setup(lib, other_wl)
    with pytest.raises(ValueError):
        other.load_config(str(cfg))


def test_live_ga_on_the_beam_within_five_percent_of_its_table_optimum(lib):
    """Live GA on the benchmark workload's reduced space at 10 % of its valid
    points: its configuration, re-timed, is within 5 % of the committed
    exhaustive table's optimum re-timed in the same run, and gives the same
    results."""
    import torch
    from paper_1811_04165_gb300 import tune_study
    wl = synth.apertif_beam()
    p, x = _setup(lib, wl)
    rec = tune_study.load_table(tune_study.BEAM_TABLE)
    assert [int(v) for v in lib.sps_tune_space(p, lib.SPACE_REDUCED)[0]] == rec["n_values"]
    want = {k: v.clone() for k, v in p.search(x).items()}
    out, ws = p.alloc_outputs(), p.workspace()

    def timed():
        for _ in range(3):
            p.search(x, out=out, workspace=ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            p.search(x, out=out, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 20

    best, res, _ = lib.sps_tune(p, x, which=lib.SPACE_REDUCED, reps=2,
                                desc=lib.search_desc(max_evaluations=int(0.1 * rec["valid"]), seed=1))
    assert res.evaluations <= int(0.1 * rec["valid"])
    t_ga = timed()
    for k in ("D", "snr", "peak_t", "peak_val", "best"):
        assert torch.equal(out[k], want[k]), k
    p.config = lib.sps_tune_config(p, lib.SPACE_REDUCED, rec["optimum_point"])
    t_opt = timed()
    assert t_ga <= 1.05 * t_opt, (t_ga, t_opt, best)
