"""The synthetic input recipes against the values the paper prints (tests/golden)."""
import itertools
import json
import os

import numpy as np

from paper_1402_4089_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_sweep_grid_matches_table1():
    g = _load("table1_sweep_grid.json")
    pr, rd = g["printed"], g["reading"]
    # the reading changes only the repeated N value
    assert pr["K"] and pr["p"] and len(pr["N"]) == len(rd["N"])
    assert [a for a, b in zip(pr["N"], rd["N"]) if a != b] == [1000]
    assert len(set(rd["N"])) == len(rd["N"])
    shapes = synthetic.sweep_shapes()
    want = {(n, p, k) for n, k, p in itertools.product(rd["N"], pr["K"], pr["p"])}
    assert set(shapes) == want and len(shapes) == len(want)
    assert len(shapes) == pr["combinations"]


def test_sweep_values_have_the_printed_variance():
    g = _load("table1_sweep_grid.json")
    var = g["reading"]["X_and_B_variance"]
    X, y, B = synthetic.sweep_problem(4000, 50, 5)
    assert abs(X.var() / var - 1.0) < 0.05
    nz = B[B != 0]
    assert abs(nz.var() / var - 1.0) < 0.2
