"""Posterior accuracy of the reduced-precision paths: GPU chains (FP32 X on CUDA
cores, BF16 X on tensor cores) against FP64 oracle chains on the original X, on
the plain workload's problem (n=1000 p=50 K=3, Gaussian prior sd 10, L=20,
eps=0.01).  Criterion per coordinate: |m_gpu - m_oracle| <= 3 sqrt(MCSE_gpu^2 +
MCSE_oracle^2), MCSE = sd / sqrt(ESS) (Geyer initial monotone sequence, chains
pooled); at most 1 % of coordinates may exceed it and none may exceed 5.
The two sides use different seeds, so the two posteriors are sampled
independently.
"""
import numpy as np
import pytest

from oracle import ess as oess
from oracle import hmc as ohmc
from paper_1402_4089_gb300 import hmc, synthetic

pytestmark = pytest.mark.gpu

ITERS, BURN, L, EPS = 1200, 200, 20, 0.01


def _means_and_mcse(draws):
    """draws (N, chains, K-1, p) -> per-coordinate pooled mean and MCSE."""
    n, c = draws.shape[:2]
    flat = draws.reshape(n, c, -1)
    m = flat.mean(axis=(0, 1))
    se = np.empty(flat.shape[2])
    for j in range(flat.shape[2]):
        se[j], _ = oess.mcse_mean(flat[:, :, j].T)
    return m, se


@pytest.fixture(scope="module")
def oracle_posterior():
    X, y, _, spec = synthetic.make_workload("plain_fp64")
    ref = ohmc.sample(X, y, 3, "gaussian", 10.0, 4, L, EPS, ITERS, 11)
    return X, y, _means_and_mcse(ref["samples"][BURN:])


@pytest.mark.parametrize("storage,engine", [("f32", 1), ("bf16", 2), ("bf16", 3)])
def test_posterior_means_within_three_mcse(cuda, oracle_posterior, storage, engine):
    import torch
    X, y, (m_o, se_o) = oracle_posterior
    chains = 32
    with hmc.create(X.astype(np.float32), y, 3, "gaussian", 10.0, x_storage=storage, max_chains=chains,
                    engine=engine) as h:
        draws = torch.empty((ITERS, chains, 2, X.shape[1]), dtype=torch.float32, device=cuda)
        stats = h.sample(chains, L, EPS, ITERS, 12345, beta0=torch.zeros((chains, 2, X.shape[1]), device=cuda),
                         samples=draws)
        torch.cuda.synchronize()
        d = draws.cpu().numpy().astype(np.float64)[BURN:]
    assert sum(s["diverged"] for s in stats) == 0
    m_g, se_g = _means_and_mcse(d)
    z = np.abs(m_g - m_o) / np.sqrt(se_g ** 2 + se_o ** 2)
    assert np.mean(z > 3.0) <= 0.01 and z.max() <= 5.0, (storage, float(z.max()), float(np.mean(z > 3.0)))
