"""The throughput report's ESS estimator (package, vectorised over coordinates)
against the oracle's one-chain-at-a-time Geyer estimator and the AR(1) closed
form N (1 - rho) / (1 + rho)."""
import numpy as np

from oracle import ess as oess
from paper_1402_4089_gb300 import diagnostics


def _ar1(rng, n, rho, shape):
    x = np.empty((n,) + shape)
    x[0] = rng.standard_normal(shape)
    z = rng.standard_normal((n,) + shape) * np.sqrt(1 - rho * rho)
    for t in range(1, n):
        x[t] = rho * x[t - 1] + z[t]
    return x


def test_matches_oracle_per_coordinate():
    rng = np.random.default_rng(5)
    rhos = np.array([0.0, 0.3, 0.6, 0.9])
    x = np.stack([_ar1(rng, 2000, r, (2,)) for r in rhos], axis=2)   # [N, chains=2, coords=4]
    got = diagnostics.ess(x)
    for j in range(len(rhos)):
        want = oess.ess_chains(x[:, :, j].T)
        assert abs(got[j] - want) <= 1e-9 * want, (j, got[j], want)


def test_ar1_closed_form():
    rng = np.random.default_rng(6)
    rho, n = 0.8, 200000
    x = _ar1(rng, n, rho, (1,))
    want = n * (1 - rho) / (1 + rho)
    assert abs(diagnostics.ess(x)[0] - want) / want < 0.05


def test_constant_coordinate_counts_as_independent():
    x = np.zeros((100, 3))
    x[:, 1] = np.random.default_rng(7).standard_normal(100)
    e = diagnostics.ess(x)
    assert e.shape == (3,) and np.all(np.isfinite(e))
