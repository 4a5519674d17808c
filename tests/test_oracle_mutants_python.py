"""The pins of the oracle's Python parts must catch plausible mistakes: each
case plants one slip in a function of oracle/ga.py (the tuner) or of the
oracle's downsampling and zapping (monkeypatched for the test only) and runs
the pins that cover it; at least one must fail.  (The C part's mutants are in
test_oracle_mutants.py.)"""
import math

import pytest

from oracle import ga
from tests import test_tuner as tuner_tests


def _cv_sample_sigma(end_configurations, values):
    out = []
    for g in range(len(values)):
        v = [values[g][p[g]] for p in end_configurations]
        mu = sum(v) / len(v)
        out.append(None if mu == 0 else math.sqrt(sum((a - mu) ** 2 for a in v) / (len(v) - 1)) / mu)
    return out


def _cv_over_indices(end_configurations, values):  # the value index instead of the parameter value
    return _real_cv(end_configurations, [list(range(len(v))) for v in values])


def _random_first_draws(space, fitness, max_evaluations=500, seed=1, max_draws=None, n_pop=32):
    r = _real_random(space, fitness, max_evaluations, seed, max_draws, n_pop)
    r.final_population = [p for p, _ in r.trace[:n_pop]]
    return r


def _ga_initial_population(space, fitness, **kw):
    r = _real_genetic(space, fitness, **kw)
    r.final_population = [p for p, _ in r.trace[:kw.get("n_pop", 32)]]
    return r


_real_random, _real_genetic, _real_cv = ga.random_search, ga.genetic, ga.coefficients_of_variation


def _ga_no_renewal(space, fitness, **kw):  # renewal tries ignored
    kw["renew"] = 0
    return _real_genetic(space, fitness, **kw)


def _planted(fn, old, new):
    """A copy of an oracle function with one slip planted in its source."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, old
    ns = dict(vars(ga))
    exec(compile(src.replace(old, new), f"<planted {fn.__name__}>", "exec"), ns)
    return ns[fn.__name__]


# renewal that checks the cache but not the generation's earlier offspring
_ga_renewal_against_the_cache_only = _planted(ga.genetic, " or child in offspring[:j]", "")


@pytest.mark.parametrize("name,attr,wrong,pins", [
    ("c_v with the sample sigma", "coefficients_of_variation", _cv_sample_sigma,
     ["test_coefficients_of_variation_pins"]),
    ("c_v over value indices", "coefficients_of_variation", _cv_over_indices,
     ["test_coefficients_of_variation_pins"]),
    ("random search's first draws as its end configurations", "random_search", _random_first_draws,
     ["test_end_configurations_are_the_last_population"]),
    ("the GA's initial population as its end configurations", "genetic", _ga_initial_population,
     ["test_end_configurations_are_the_last_population"]),
    ("a GA without renewal", "genetic", _ga_no_renewal, ["test_renewal_keeps_a_converged_population_exploring"]),
    ("renewal that checks the cache but not the generation's other offspring", "genetic",
     _ga_renewal_against_the_cache_only, ["test_renewal_keeps_a_converged_population_exploring"]),
])
def test_a_pin_fails(monkeypatch, name, attr, wrong, pins):
    monkeypatch.setattr(ga, attr, wrong)
    failed = False
    for pin in pins:
        fn = getattr(tuner_tests, pin)
        args = [2] if pin == "test_end_configurations_are_the_last_population" else []
        try:
            fn(*args)
        except AssertionError:
            failed = True
    assert failed, f"no pin caught: {name}"


# ----------------------------------------------------------------------------- the variants' oracle functions
import numpy as np  # noqa: E402

import oracle  # noqa: E402
from tests import test_oracle_pins as pins  # noqa: E402

_real_decimate, _real_snr_decimated, _real_zap = oracle.decimate, oracle.snr_decimated, oracle.zap_channels


def _decimate_keeps_tail(D, f):  # a trailing partial window counted as a sample
    D = np.asarray(D)
    n = -(-D.shape[1] // f)
    P = np.zeros((D.shape[0], n * f), np.int64)
    P[:, :D.shape[1]] = D
    return P.reshape(D.shape[0], n, f).sum(axis=2)


def _decimate_shifted(D, f):  # windows starting one sample late
    D = np.asarray(D)
    n = (D.shape[1] - 1) // f
    return D[:, 1:1 + n * f].astype(np.int64).reshape(D.shape[0], n, f).sum(axis=2)


def _snr_decimated_peak_in_output_samples(D, factors):  # peak_t left in downsampled samples
    s, pt, pv = _real_snr_decimated(D, factors)
    return s, pt // np.array([int(f) for f in factors])[:, None], pv


def _zap_keeps_first_flag(x, zap):  # the first zapped channel survives
    z = np.asarray(zap).astype(bool).copy()
    first = np.flatnonzero(z)
    if first.size:
        z[first[0]] = False
    return _real_zap(x, z)


def _run_pin(name, params):
    fn = getattr(pins, name)
    for p in params:
        try:
            fn(*p)
        except AssertionError:
            return True
    return False


@pytest.mark.parametrize("attr,wrong,pin,params", [
    ("decimate", _decimate_keeps_tail, "test_decimated_series_is_the_boxcar_at_stride_f", [(3,), (7,), (10,)]),
    ("decimate", _decimate_shifted, "test_decimated_series_is_the_boxcar_at_stride_f", [(2,), (3,)]),
    ("snr_decimated", _snr_decimated_peak_in_output_samples, "test_decimated_snr_single_spike_closed_form",
     [(4, 13), (10, 99)]),
    ("zap_channels", _zap_keeps_first_flag, "test_zapping_is_linear_in_the_channel_set", [()]),
])
def test_variant_pin_fails(monkeypatch, attr, wrong, pin, params):
    monkeypatch.setattr(oracle, attr, wrong)
    assert _run_pin(pin, params), f"no pin caught the {attr} slip"


# ----------------------------------------------------------------------------- the two-step path's index helpers
_real_coarse_index, _real_subband_lengths = oracle.coarse_index, oracle.subband_lengths


def _coarse_index_modulo(n_dms, n_coarse):  # trials dealt round-robin to the coarse DMs
    return (np.arange(n_dms) % n_coarse).astype(np.int32)


def _coarse_index_nearest(n_dms, n_coarse):  # the nearest block start instead of the one below
    per = n_dms // n_coarse
    return np.minimum(np.rint(np.arange(n_dms) / per), n_coarse - 1).astype(np.int32)


def _coarse_index_off_by_one(n_dms, n_coarse):  # blocks shifted by one trial
    per = n_dms // n_coarse
    return np.minimum((np.arange(n_dms) + 1) // per, n_coarse - 1).astype(np.int32)


def _lengths_swapped(n_t, d1, d2):  # step one's spread taken for step two's
    n_1 = n_t + int(d1.max())
    return n_1, n_1 + int(d2.max())


def _lengths_step1_spread_twice(n_t, d1, d2):  # N_in from step two's spread again
    n_1 = n_t + int(d2.max())
    return n_1, n_1 + int(d2.max())


def _lengths_one_short(n_t, d1, d2):  # the last sample of step two's reads dropped
    n_1 = n_t + int(d2.max()) - 1
    return n_1, n_1 + int(d1.max())


@pytest.mark.parametrize("attr,wrong,pins_to_run", [
    ("coarse_index", _coarse_index_modulo, ["test_coarse_index_hand_example", "test_coarse_index_apertif_grid"]),
    ("coarse_index", _coarse_index_nearest, ["test_coarse_index_hand_example", "test_coarse_index_apertif_grid"]),
    ("coarse_index", _coarse_index_off_by_one, ["test_coarse_index_hand_example", "test_coarse_index_apertif_grid"]),
    ("subband_lengths", _lengths_swapped, ["test_subband_lengths_hand_example", "test_subband_apertif_lengths"]),
    ("subband_lengths", _lengths_step1_spread_twice,
     ["test_subband_lengths_hand_example", "test_subband_apertif_lengths"]),
    ("subband_lengths", _lengths_one_short, ["test_subband_lengths_hand_example", "test_subband_apertif_lengths"]),
])
def test_subband_helper_pin_fails(monkeypatch, attr, wrong, pins_to_run):
    monkeypatch.setattr(oracle, attr, wrong)
    caught = [name for name in pins_to_run if _run_pin(name, [()])]
    assert caught, f"no pin caught the {attr} slip"
