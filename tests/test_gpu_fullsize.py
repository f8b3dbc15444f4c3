"""Parity at the full sizes of the timed workloads, in the launch configuration
the library chooses for them (the one the bench runs unless its autotuner finds a
faster tile), against the FP64 oracle evaluated on the same stored X values.

* precision workload, n=50000 p=10000 K=20, 4 chains in one tensor-core launch,
  X stored in BF16 and in per-column-scaled FP8 (codes and scales bit-exact
  against the oracle's quantisation);
* batched workload's shared problem, n=20000 p=2000 K=10, 64 chains (the chains
  run in groups that fit TMEM, several launches per call).

Tolerance: the BF16 bar of the tensor-core engine (coefficients and residual
are BF16 MMA operands, FP32 accumulation): gradient relative error <= 1e-2 per
chain, log K relative error <= 1e-3.  The oracle is plain numpy FP64 (a BLAS
matmul per contraction), a few seconds per chain at these sizes.
"""
import numpy as np
import pytest

from oracle import model, quant
from paper_1402_4089_gb300 import hmc, synthetic

pytestmark = pytest.mark.gpu

TOL_G, TOL_L = 1e-2, 1e-3


def _errs(Xq, y, beta, lp, g, kind, scale, chains):
    out = []
    for c in chains:
        lk_o = model.log_kernel(Xq, y, beta[c].astype(np.float64), kind, scale)
        g_o = model.grad_log_kernel(Xq, y, beta[c].astype(np.float64), kind, scale)
        out.append((c, abs(lp[c] - lk_o) / max(1.0, abs(lk_o)),
                    float(np.linalg.norm(g[c].astype(np.float64) - g_o) / np.linalg.norm(g_o))))
    return out


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_precision_workload_full_size(cuda, storage):
    import torch
    X, y, btrue, spec = synthetic.make_workload("precision")
    K, chains = spec["K"], spec["chains"]
    kind, scale = spec["prior"]
    rng = np.random.default_rng(21)
    beta = (0.01 * rng.standard_normal((chains, K - 1, X.shape[1]))).astype(np.float32)
    with hmc.create(X, y, K, kind, scale, x_storage=storage, max_chains=chains) as h:
        d = h.describe()
        assert d["engine"] == "tcgen05" and d["problems"][0]["group_chains"] == chains, d
        bits, scales = h.get_x()
        lp, g = h.logpost_grad(torch.from_numpy(beta).to(cuda))
        torch.cuda.synchronize()
        lp, g = lp.cpu().numpy(), g.cpu().numpy()
    if storage == "fp8":
        c_o, s_o = quant.fp8_quantize(X)
        assert np.array_equal(scales, s_o) and np.array_equal(bits, c_o)
        Xq = quant.fp8_dequantize(bits, scales)
    else:
        assert np.array_equal(bits, quant.bf16_bits(X))
        Xq = quant.bf16_decode(bits).astype(np.float64)
    del X
    for c, el, eg in _errs(Xq, y, beta, lp, g, kind, scale, range(chains)):
        assert el <= TOL_L and eg <= TOL_G, (storage, c, el, eg)


def test_batched_workload_64_chains_full_size(cuda):
    import torch
    X, y, btrue, spec = synthetic.make_workload("batched")
    K, chains = spec["K"], spec["chains"]
    kind, scale = spec["prior"]
    rng = np.random.default_rng(22)
    beta = (0.05 * rng.standard_normal((chains, K - 1, X.shape[1]))).astype(np.float32)
    with hmc.create(X, y, K, kind, scale, x_storage="bf16", max_chains=chains) as h:
        assert h.describe()["engine"] == "tcgen05"
        bits, _ = h.get_x()
        lp, g = h.logpost_grad(torch.from_numpy(beta).to(cuda))
        torch.cuda.synchronize()
        lp, g = lp.cpu().numpy(), g.cpu().numpy()
    Xq = quant.bf16_decode(bits).astype(np.float64)
    # every chain group, first and last chains sampled plus a seeded spread
    picks = sorted(set([0, 1, chains - 2, chains - 1] + list(rng.choice(chains, 8, replace=False))))
    for c, el, eg in _errs(Xq, y, beta, lp, g, kind, scale, picks):
        assert el <= TOL_L and eg <= TOL_G, (c, el, eg)
