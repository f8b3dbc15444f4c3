"""Parity at the full sizes of the timed workloads, in the launch configuration
the library chooses for them (the one the bench runs unless its autotuner finds a
faster tile), against the FP64 oracle evaluated on the same stored X values.

* precision workload, n=50000 p=10000 K=20, 4 chains, X stored in BF16 and in
  per-column-scaled FP8 (codes and scales bit-exact against the oracle's
  quantisation), on the default two-pass engine and on the fused engine (all
  chains in one launch);
* batched workload's shared problem, n=20000 p=2000 K=10, 64 chains;
* batched workload's 32 uneven problems (n ~ U[500, 20000], p ~ U[100, 4000],
  K ~ U{3..20}) in one handle, one fused launch per gradient;
* autodiff workload, n=100000 p=20000 K=10, 8 chains, X in BF16 (4 GB): the
  gradient at states the GPU chains reached, against the oracle on the stored X
  (evaluated in row blocks, FP64) and against central finite differences of the
  oracle's log K on 64 coordinates drawn with a Philox generator.

Gates: arithmetic error (against the oracle on the stored X) 3e-3 relative in
norm and element-wise per chain, log K 1e-4 (the tensor-core bound: BF16
residual operand); total error against the original X: 1e-2 for BF16 storage;
FP8 storage's total error is reported (E4M3 keeps 3 mantissa bits).
"""
import numpy as np
import pytest

from oracle import model, quant
from paper_1402_4089_gb300 import hmc, synthetic
from parity_util import grad_errs, lk_err

pytestmark = pytest.mark.gpu

TOL_G, TOL_L = 3e-3, 1e-4
TOL_TOTAL_BF16 = 1e-2


def _errs(Xq, y, beta, lp, g, kind, scale, chains, X=None):
    out = []
    for c in chains:
        b = beta[c].astype(np.float64)
        lk_o = model.log_kernel(Xq, y, b, kind, scale)
        g_o = model.grad_log_kernel(Xq, y, b, kind, scale)
        tot = max(grad_errs(g[c], model.grad_log_kernel(X, y, b, kind, scale))) if X is not None else None
        out.append((c, lk_err(lp[c], lk_o)) + grad_errs(g[c], g_o) + (tot,))
    return out


@pytest.mark.parametrize("storage,engine", [("bf16", 0), ("fp8", 0), ("bf16", 2), ("fp8", 2)])
def test_precision_workload_full_size(cuda, storage, engine):
    import torch
    X, y, btrue, spec = synthetic.make_workload("precision")
    K, chains = spec["K"], spec["chains"]
    kind, scale = spec["prior"]
    rng = np.random.default_rng(21)
    beta = (0.01 * rng.standard_normal((chains, K - 1, X.shape[1]))).astype(np.float32)
    with hmc.create(X, y, K, kind, scale, x_storage=storage, max_chains=chains, engine=engine) as h:
        d = h.describe()
        # a single problem defaults to the two-pass engine (BF16 and FP8)
        assert d["engine"] == ("tcgen05_2pass" if engine == 0 else "tcgen05"), d
        assert d["problems"][0]["group_chains"] == chains, d
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
    X64 = X.astype(np.float64)
    del X, bits
    for c, el, eg, ee, et in _errs(Xq, y, beta, lp, g, kind, scale, range(chains), X=X64):
        assert el <= TOL_L and eg <= TOL_G and ee <= TOL_G, (storage, c, el, eg, ee)
        if storage == "bf16":
            assert et <= TOL_TOTAL_BF16, (c, "total error", et)
        else:
            print(f"precision workload, FP8 storage, chain {c}: total gradient error vs original X {et:.3e}")
            assert et <= 0.1, et


def test_batched_workload_64_chains_full_size(cuda):
    import torch
    X, y, btrue, spec = synthetic.make_workload("batched")
    K, chains = spec["K"], spec["chains"]
    kind, scale = spec["prior"]
    rng = np.random.default_rng(22)
    beta = (0.05 * rng.standard_normal((chains, K - 1, X.shape[1]))).astype(np.float32)
    with hmc.create(X, y, K, kind, scale, x_storage="bf16", max_chains=chains) as h:
        # 64 chains do not fit one fused launch: the two-pass engine takes them all at once
        assert h.describe()["engine"] == "tcgen05_2pass"
        bits, _ = h.get_x()
        lp, g = h.logpost_grad(torch.from_numpy(beta).to(cuda))
        torch.cuda.synchronize()
        lp, g = lp.cpu().numpy(), g.cpu().numpy()
    Xq = quant.bf16_decode(bits).astype(np.float64)
    # every chain group, first and last chains sampled plus a seeded spread
    picks = sorted(set([0, 1, chains - 2, chains - 1] + list(rng.choice(chains, 8, replace=False))))
    for c, el, eg, ee, et in _errs(Xq, y, beta, lp, g, kind, scale, picks, X=X.astype(np.float64)):
        assert el <= TOL_L and eg <= TOL_G and ee <= TOL_G, (c, el, eg, ee)
        assert et <= TOL_TOTAL_BF16, (c, "total error", et)


def test_batched_uneven_32_problems_full_size(cuda):
    import torch
    spec = synthetic.WORKLOADS["batched"]
    kind, scale = spec["prior"]
    shapes = synthetic.batched_shapes()
    probs = [synthetic.make_problem(n, p, K, seed=0, sub=100 + i) for i, (n, p, K) in enumerate(shapes)]
    rng = np.random.default_rng(23)
    betas = [(0.05 * rng.standard_normal((1, K - 1, p))).astype(np.float32) for (n, p, K) in shapes]
    with hmc.create_batch([pr[0] for pr in probs], [pr[1] for pr in probs], [K for (_, _, K) in shapes], kind, scale,
                          x_storage="bf16", max_chains=1) as h:
        d = h.describe()
        assert d["engine"] == "tcgen05" and d["batched_launch"] is True, d
        h.set_timing(True)
        lp, g = h.logpost_grad(torch.from_numpy(np.concatenate([b.ravel() for b in betas])).to(cuda), chains=1)
        torch.cuda.synchronize()
        assert h.fused_kernel_time()[1] == 1            # every problem in one launch
        bits = [h.get_x(b)[0] for b in range(len(shapes))]
        lp, g = lp.cpu().numpy(), g.cpu().numpy()
    off = 0
    for b, ((X, y, _), (n, p, K)) in enumerate(zip(probs, shapes)):
        Xq = quant.bf16_decode(bits[b]).astype(np.float64)
        gb = g[off:off + (K - 1) * p].reshape(1, K - 1, p)
        off += (K - 1) * p
        (_, el, eg, ee, et), = _errs(Xq, y, betas[b], lp[b:b + 1], gb, kind, scale, [0], X=X.astype(np.float64))
        assert el <= TOL_L and eg <= TOL_G and ee <= TOL_G, (b, (n, p, K), el, eg, ee)
        assert et <= TOL_TOTAL_BF16, (b, "total error", et)


@pytest.mark.parametrize("engine", [0, 2])
def test_autodiff_workload_full_size(cuda, engine):
    """Default engine (two-pass: the fused engine fits 3 of the 8 chains per
    launch here) and the fused engine (three launches of 3, 3 and 2 chains)."""
    import torch
    X, y, btrue, spec = synthetic.make_workload("autodiff")
    n, p, K, chains = spec["n"], spec["p"], spec["K"], spec["chains"]
    kind, scale = spec["prior"]
    rng = np.random.default_rng(24)
    b0 = (0.01 * rng.standard_normal((chains, K - 1, p))).astype(np.float32)
    with hmc.create(X, y, K, kind, scale, x_storage="bf16", max_chains=chains, engine=engine) as h:
        del X
        assert h.describe()["engine"] == ("tcgen05" if engine == 2 else "tcgen05_2pass")
        h.sample(chains, 5, spec["eps"], 2, 7, beta0=torch.from_numpy(b0).to(cuda))      # states the chains reach
        beta = torch.empty((chains, K - 1, p), dtype=torch.float32, device=cuda)
        h.get_state(chains, beta=beta)
        lp, g = h.logpost_grad(beta)
        torch.cuda.synchronize()
        beta, lp, g = beta.cpu().numpy(), lp.cpu().numpy(), g.cpu().numpy()
        bits, _ = h.get_x()
    blocks = ((quant.bf16_decode(bits[a:a + 10000]), y[a:a + 10000]) for a in range(0, n, 10000))
    lk_o, g_o, Z = model.log_kernel_and_grad_by_rows(blocks, list(beta), kind, scale)
    for c in range(chains):
        el = lk_err(lp[c], lk_o[c])
        eg, ee = grad_errs(g[c], g_o[c])
        assert el <= TOL_L and eg <= TOL_G and ee <= TOL_G, (c, el, eg, ee)
    # central differences of the oracle's log K on 64 Philox-drawn coordinates: moving
    # beta_kj by +-h moves the logits of class k by +-h x_.j
    pick = np.random.Generator(np.random.Philox(key=2014)).integers(0, [chains, K - 1, p], size=(64, 3))
    h_fd = 1e-3
    for c, k, j in pick:
        xj = quant.bf16_decode(np.ascontiguousarray(bits[:, j])).astype(np.float64)
        fd = 0.0
        for sgn in (1.0, -1.0):
            Zs = Z[c].copy()
            Zs[:, k] += sgn * h_fd * xj
            bk = beta[c, k, j] + sgn * h_fd
            fd += sgn * (model.log_likelihood_of_logits(Zs, y) + float(model.prior_terms(bk, kind, scale)))
        fd /= 2 * h_fd
        assert abs(g[c, k, j] - fd) <= TOL_G * np.abs(g_o[c]).max() + 1e-6 * abs(fd), (c, k, j, g[c, k, j], fd)
