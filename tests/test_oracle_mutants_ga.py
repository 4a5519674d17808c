"""The tuner oracle's pins must catch plausible mistakes: each case plants one
slip in oracle/ga.py's functions (monkeypatched for the test only) and runs the
pins that cover it; at least one must fail."""
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


@pytest.mark.parametrize("name,attr,wrong,pins", [
    ("c_v with the sample sigma", "coefficients_of_variation", _cv_sample_sigma,
     ["test_coefficients_of_variation_pins"]),
    ("c_v over value indices", "coefficients_of_variation", _cv_over_indices,
     ["test_coefficients_of_variation_pins"]),
    ("random search's first draws as its end configurations", "random_search", _random_first_draws,
     ["test_end_configurations_are_the_last_population"]),
    ("the GA's initial population as its end configurations", "genetic", _ga_initial_population,
     ["test_end_configurations_are_the_last_population"]),
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
