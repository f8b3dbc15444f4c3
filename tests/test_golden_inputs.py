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


def test_mnist_shaped_recipe():
    X, y, B, spec = synthetic.make_workload("mnist_shaped", n=3000)
    assert X.shape == (3000, 785) and X.dtype == np.float32 and spec["K"] == 10
    assert np.all(X[:, 0] == 1.0)
    px = X[:, 1:]
    k = np.rint(px * 255.0)
    assert np.all((k >= 0) & (k <= 255)) and np.allclose(px, (k / 255.0).astype(np.float32), rtol=0, atol=0)
    assert abs((px > 0).mean() - 0.19) < 0.01
    assert y.min() >= 0 and y.max() < 10 and len(np.unique(y)) == 10
    assert spec["prior"] == ("cauchy", 1.0) and spec["burn_in"] == 100 and spec["L"] == 100


def test_annealing_schedule_matches_oracle():
    from oracle import hmc as ohmc
    from paper_1402_4089_gb300 import hmc
    for t0, r, n in ((1.0e3, 0.9, 100), (50.0, 0.7, 20), (1.0, 0.5, 5)):
        assert np.array_equal(hmc.annealing_temperatures(n, t0, r), ohmc.annealing_temperatures(n, t0, r))
    t = hmc.annealing_temperatures(100)
    assert t[0] == 900.0 and t[-1] == 1.0 and np.all(np.diff(t) <= 0)
