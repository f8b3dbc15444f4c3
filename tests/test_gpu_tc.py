"""Tensor-core engine (tcgen05, BF16 or per-column-scaled FP8 X) against the
FP64 oracle on the same stored values (FP8: the dequantised codes x_q s_j).

The MMA operands are BF16: the coefficients enter as two BF16 terms (hi + lo,
about 16 bits), the residual R = Y - P as one BF16 term (relative rounding
error <= 2^-9 per entry), accumulation is FP32 in TMEM.  The gradient's
arithmetic error against the oracle on the stored X is therefore dominated by
the rounding of R: about 2^-9 / sqrt(3) ~ 1.1e-3 relative for independent
roundings, so the gate is 3e-3 (relative norm and element-wise), log K 1e-4.
The total error against the original X (BF16 storage adds a 2^-9 relative
rounding of every x_ij) is held to the BF16 bar of 1e-2."""
import numpy as np
import pytest

from oracle import model, quant
from paper_1402_4089_gb300 import hmc, synthetic
from parity_util import grad_errs, lk_err

pytestmark = pytest.mark.gpu

TOL_G, TOL_L = 3e-3, 1e-4
TOL_TOTAL_BF16 = 1e-2


def _run(cuda, n, p, K, chains, seed, bscale=0.05, tile=None, prior=("gaussian", 10.0), storage="bf16"):
    import torch
    X, y, _ = synthetic.make_problem(n, p, K, seed=seed)
    rng = np.random.default_rng(seed + 1)
    beta = (bscale * rng.standard_normal((chains, K - 1, p))).astype(np.float32)
    with hmc.create(X, y, K, prior[0], prior[1], x_storage=storage, max_chains=chains, engine=2, tile=tile) as h:
        d = h.describe()
        assert d["engine"] == "tcgen05"
        bits, scales = h.get_x()
        if storage == "fp8":
            # stored codes and scales are exactly the oracle's quantisation of X
            c_o, s_o = quant.fp8_quantize(X)
            assert np.array_equal(scales, s_o) and np.array_equal(bits, c_o)
            Xq = quant.fp8_dequantize(bits, scales).astype(np.float64)
        else:
            Xq = quant.bf16_decode(bits).astype(np.float64)
        lp, g = h.logpost_grad(torch.from_numpy(beta).to(cuda))
        torch.cuda.synchronize()
        lp, g = lp.cpu().numpy(), g.cpu().numpy()
    errs = []
    for c in range(chains):
        lk_o = model.log_kernel(Xq, y, beta[c], prior[0], prior[1])
        g_o = model.grad_log_kernel(Xq, y, beta[c], prior[0], prior[1])
        g_t = model.grad_log_kernel(X.astype(np.float64), y, beta[c], prior[0], prior[1])   # original X
        errs.append((lk_err(lp[c], lk_o),) + grad_errs(g[c], g_o) + (max(grad_errs(g[c], g_t)),))
    return d, errs


@pytest.mark.parametrize("n,p,K,chains,S", [(1000, 700, 6, 2, 0), (333, 129, 3, 1, 1), (2049, 1000, 20, 4, 0),
                                            (128, 64, 2, 3, 2), (5000, 2000, 10, 7, 4), (130, 4100, 5, 1, 16)])
def test_tc_matches_oracle(cuda, n, p, K, chains, S):
    d, errs = _run(cuda, n, p, K, chains, seed=n + p, tile=(S, 0, 0, 0))
    for c, (el, eg, ee, et) in enumerate(errs):
        assert el <= TOL_L and eg <= TOL_G and ee <= TOL_G, (d["problems"][0], c, el, eg, ee)
        assert et <= TOL_TOTAL_BF16, (d["problems"][0], c, "total error vs original X", et)


def test_tc_deterministic(cuda):
    import torch
    X, y, _ = synthetic.make_problem(3000, 1500, 8, seed=3)
    beta = torch.from_numpy((0.05 * np.random.default_rng(4).standard_normal((3, 7, 1500))).astype(np.float32)).to(cuda)
    with hmc.create(X, y, 8, "gaussian", 10.0, x_storage="bf16", max_chains=3, engine=2) as h:
        a = [t.cpu().numpy() for t in h.logpost_grad(beta)]
        b = [t.cpu().numpy() for t in h.logpost_grad(beta)]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("n,p,K,chains,S", [(1000, 700, 6, 2, 0), (333, 129, 3, 1, 1), (2049, 1000, 20, 4, 0),
                                            (5000, 2000, 10, 7, 4)])
def test_tc_fp8_matches_oracle(cuda, n, p, K, chains, S):
    d, errs = _run(cuda, n, p, K, chains, seed=n + 3 * p, tile=(S, 0, 0, 0), storage="fp8")
    for c, (el, eg, ee, et) in enumerate(errs):
        assert el <= TOL_L and eg <= TOL_G and ee <= TOL_G, (d["problems"][0], c, el, eg, ee)
        # total error of E4M3 storage (3 mantissa bits) against the original X: reported, aim <= 3e-2
        print(f"fp8 total error n={n} p={p} K={K} chain {c}: {et:.3e}")
        assert et <= 0.1, et


def test_tc_fp8_deterministic(cuda):
    import torch
    X, y, _ = synthetic.make_problem(3000, 1500, 8, seed=13)
    beta = torch.from_numpy((0.05 * np.random.default_rng(14).standard_normal((3, 7, 1500))).astype(np.float32)).to(cuda)
    with hmc.create(X, y, 8, "gaussian", 10.0, x_storage="fp8", max_chains=3, engine=2) as h:
        a = [t.cpu().numpy() for t in h.logpost_grad(beta)]
        b = [t.cpu().numpy() for t in h.logpost_grad(beta)]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_tc_batch_of_uneven_problems_one_launch(cuda, storage):
    """Independent problems of different n, p, K in one tensor-core launch."""
    import torch
    shapes = [(900, 130, 3), (2049, 700, 12), (300, 64, 2), (5000, 1500, 20)]
    probs = [synthetic.make_problem(n, p, K, seed=31, sub=i) for i, (n, p, K) in enumerate(shapes)]
    chains = 2
    rng = np.random.default_rng(32)
    betas = [(0.05 * rng.standard_normal((chains, K - 1, p))).astype(np.float32) for (n, p, K) in shapes]
    flat = torch.from_numpy(np.concatenate([b.ravel() for b in betas])).to(cuda)
    with hmc.create_batch([pr[0] for pr in probs], [pr[1] for pr in probs], [s[2] for s in shapes],
                          "gaussian", 10.0, x_storage=storage, max_chains=chains) as h:
        d = h.describe()
        assert d["engine"] == "tcgen05" and d["batched_launch"] is True, d
        xs = [h.get_x(b) for b in range(len(shapes))]
        h.set_timing(True)
        lp, g = h.logpost_grad(flat, chains=chains)
        torch.cuda.synchronize()
        _, launches = h.fused_kernel_time()
        assert launches == 1
        lp, g = lp.cpu().numpy(), g.cpu().numpy()
    off = 0
    for b, ((X, y, _), (n, p, K)) in enumerate(zip(probs, shapes)):
        bits, scales = xs[b]
        Xq = (quant.fp8_dequantize(bits, scales) if storage == "fp8" else quant.bf16_decode(bits)).astype(np.float64)
        gb = g[off:off + chains * (K - 1) * p].reshape(chains, K - 1, p)
        off += chains * (K - 1) * p
        for c in range(chains):
            lk_o = model.log_kernel(Xq, y, betas[b][c], "gaussian", 10.0)
            g_o = model.grad_log_kernel(Xq, y, betas[b][c], "gaussian", 10.0)
            assert lk_err(lp[b * chains + c], lk_o) <= TOL_L, (b, c)
            assert max(grad_errs(gb[c], g_o)) <= TOL_G, (b, c, grad_errs(gb[c], g_o))


def test_tc_chain_groups_are_even(cuda):
    """16 chains where one launch holds at most 14 (p = 5000, K = 10): two launches
    of 8 chains each (a 14 + 2 split would stream X a second time for 2 chains)."""
    import torch
    n, p, K, chains = 1500, 5000, 10, 16
    X, y, _ = synthetic.make_problem(n, p, K, seed=41)
    rng = np.random.default_rng(42)
    beta = (0.05 * rng.standard_normal((chains, K - 1, p))).astype(np.float32)
    with hmc.create(X, y, K, "gaussian", 10.0, x_storage="bf16", max_chains=chains, engine=2) as h:
        d = h.describe()["problems"][0]
        assert d["group_chains"] == 8, d
        bits, _ = h.get_x()
        h.set_timing(True)
        lp, g = h.logpost_grad(torch.from_numpy(beta).to(cuda))
        torch.cuda.synchronize()
        _, launches = h.fused_kernel_time()
        assert launches == 2
        lp, g = lp.cpu().numpy(), g.cpu().numpy()
    Xq = quant.bf16_decode(bits).astype(np.float64)
    for c in (0, 7, 8, 15):
        lk_o = model.log_kernel(Xq, y, beta[c], "gaussian", 10.0)
        g_o = model.grad_log_kernel(Xq, y, beta[c], "gaussian", 10.0)
        assert lk_err(lp[c], lk_o) <= TOL_L and max(grad_errs(g[c], g_o)) <= TOL_G, (c, grad_errs(g[c], g_o))
