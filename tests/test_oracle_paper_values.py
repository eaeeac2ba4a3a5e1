"""Pins of the oracle to values the paper prints (tests/golden/paper_values.txt,
each with its citation): the electron transport cutoff, by its behaviour: an
electron just below it deposits its energy where it starts, one just above
it takes CSDA steps."""
import os

import pytest

from oracle import oracle as O
from paper_1503_01725_b300 import workloads as W


def paper_values():
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, value, unit, *cite = line.split()
                assert unit == "MeV" and cite, line
                vals[name] = float(value)
    return vals


def test_electron_cutoff_is_the_papers():
    cut = paper_values()["electron_cutoff"]
    ph = W.water_phantom(16, 16, 16, 0.5)
    for E in (cut * (1 - 1e-6), cut * 0.5):
        path, dep = O.electron_path(ph, E, seed=1, ms_off=1)
        assert path == 0.0 and dep == pytest.approx(E, rel=1e-12)
    path, dep = O.electron_path(ph, cut * (1 + 1e-3), seed=1, ms_off=1)
    assert path > 0.0 and dep == pytest.approx(cut * (1 + 1e-3), rel=1e-9)
