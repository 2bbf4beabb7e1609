"""Regression fixtures of the oracle (``tests/golden``, written by
``tests/golden/make_golden.py`` from the oracle only; the paper prints no
worked numerical example for the pressure solve).  A mismatch means the
oracle's arithmetic changed: regenerate only with a commit that names the
passage justifying the change."""
import importlib.util
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
mk = importlib.util.module_from_spec(spec)
spec.loader.exec_module(mk)


def _stored(name):
    return np.loadtxt(os.path.join(HERE, name + ".txt"), comments="#")


@pytest.mark.parametrize("name", list(mk.CASES))
def test_metric_matches_fixture(name):
    want = _stored(name)
    got = mk.metric_rows(mk.CASES[name])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_solution_matches_fixture():
    name, d, st = mk.SOLVE
    want = _stored(name)
    got = mk.solution(d, st)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
