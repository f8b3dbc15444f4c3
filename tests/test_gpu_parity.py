"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (gradient: ||g - g_ref|| / ||g_ref|| over all coordinates of a
chain and, against the same bound, the element-wise max |g - g_ref| /
max |g_ref|; log K: |d| / max(1, |log K_ref|)):
* FP64 state and X: 1e-11 (rounding-order differences only);
* FP32 arithmetic (FP32, BF16 and FP8 storage, each compared with the oracle
  run on the same stored values): 1e-5;
* BF16 storage against the oracle on the original FP32 X: 1e-2.
Byte work (the stored BF16 / FP8 codes and FP8 column scales) is bit-exact.
"""
import os

import numpy as np
import pytest

from oracle import hmc as ohmc
from oracle import model, quant
from paper_1402_4089_gb300 import hmc, synthetic
from parity_util import assert_grad, lk_err

pytestmark = pytest.mark.gpu


def oracle_lpg(X, y, beta, kind, scale):
    lk = np.array([model.log_kernel(X, y, b, kind, scale) for b in beta])
    g = np.stack([model.grad_log_kernel(X, y, b, kind, scale) for b in beta])
    return lk, g


def gpu_lpg(h, beta, dev):
    import torch
    bt = torch.from_numpy(np.ascontiguousarray(beta)).to(dev)
    lp, g = h.logpost_grad(bt)
    torch.cuda.synchronize()
    return lp.cpu().numpy(), g.cpu().numpy()


def check(h, X, y, beta, kind, scale, dev, tol_g, tol_l, Xref=None):
    lp, g = gpu_lpg(h, beta, dev)
    lk_o, g_o = oracle_lpg(X if Xref is None else Xref, y, beta, kind, scale)
    for c in range(beta.shape[0]):
        assert lk_err(lp[c], lk_o[c]) <= tol_l, (c, lp[c], lk_o[c])
        assert_grad(g[c], g_o[c], tol_g, c)
    return lp, g


def test_fp64_plain_workload(cuda):
    X, y, _, spec = synthetic.make_workload("plain_fp64")
    rng = np.random.default_rng(0)
    beta = 0.3 * rng.standard_normal((3, 2, 50))
    with hmc.create(X, y, 3, "gaussian", 10.0, x_storage="f64", state="f64", max_chains=3) as h:
        check(h, X, y, beta, "gaussian", 10.0, cuda, 1e-11, 1e-11)


@pytest.mark.parametrize("S,NS", [(1, 3), (2, 2), (4, 6), (8, 2), (16, 4), (1, 5)])
def test_fp32_tiles_ragged(cuda, S, NS):
    X, y, _ = synthetic.make_problem(1013, 300, 4, seed=5)
    rng = np.random.default_rng(S * 100 + NS)
    beta = (0.2 * rng.standard_normal((2, 3, 300))).astype(np.float32)
    with hmc.create(X, y, 4, "gaussian", 1.0, max_chains=2, tile=(S, 0, 0, NS)) as h:
        d = h.describe()["problems"][0]
        assert (d["S"], d["BM"], d["NSTAGE"]) == (S, 16, NS)          # 1013 rows: 63 tiles of 16 + 5
        check(h, X, y, beta, "gaussian", 1.0, cuda, 1e-5, 1e-5)


def test_fp32_highdim_full_size(cuda):
    X, y, btrue, spec = synthetic.make_workload("highdim_fp32")
    rng = np.random.default_rng(1)
    beta = (btrue + 0.01 * rng.standard_normal(btrue.shape)).astype(np.float32)[None]
    with hmc.create(X, y, 10, "gaussian", 1.0) as h:
        check(h, X, y, beta, "gaussian", 1.0, cuda, 1e-5, 1e-5)


def test_bf16_storage_bits_and_error(cuda):
    X, y, btrue = synthetic.make_problem(3000, 700, 6, seed=7)
    rng = np.random.default_rng(2)
    beta = (0.05 * rng.standard_normal((2, 5, 700))).astype(np.float32)
    with hmc.create(X, y, 6, "gaussian", 10.0, x_storage="bf16", max_chains=2, engine=1) as h:
        bits, _ = h.get_x()
        assert np.array_equal(bits, quant.bf16_bits(X))
        Xq = quant.bf16_decode(bits).astype(np.float64)
        check(h, Xq, y, beta, "gaussian", 10.0, cuda, 1e-5, 1e-5)          # arithmetic error
        check(h, X, y, beta, "gaussian", 10.0, cuda, 1e-2, 1e-2)           # total error vs original X


def test_fp8_storage_bits_and_error(cuda):
    X, y, _ = synthetic.make_problem(2000, 513, 5, seed=8)
    X[:, 7] = 0.0
    rng = np.random.default_rng(3)
    beta = (0.05 * rng.standard_normal((1, 4, 513))).astype(np.float32)
    with hmc.create(X, y, 5, "gaussian", 10.0, x_storage="fp8", engine=1) as h:   # CUDA cores, FP32 arithmetic
        codes, scales = h.get_x()
        c_o, s_o = quant.fp8_quantize(X)
        assert np.array_equal(scales, s_o)
        assert np.array_equal(codes, c_o)
        Xq = quant.fp8_dequantize(codes, scales)
        check(h, Xq, y, beta, "gaussian", 10.0, cuda, 1e-5, 1e-5)


@pytest.mark.parametrize("n,p,K,chains", [(0, 40, 3, 2), (1, 5, 2, 1), (37, 1, 2, 3), (100, 33, 21, 1),
                                          (65, 64, 3, 4)])
def test_edge_shapes(cuda, n, p, K, chains):
    rng = np.random.default_rng(n + p + K)
    X = rng.standard_normal((n, p)).astype(np.float32)
    y = rng.integers(0, K, size=n).astype(np.int32)
    if n > 3:
        y[:3] = K - 1
    beta = (0.3 * rng.standard_normal((chains, K - 1, p))).astype(np.float32)
    with hmc.create(X, y, K, "cauchy", 1.0, max_chains=chains) as h:
        check(h, X, y, beta, "cauchy", 1.0, cuda, 1e-5, 1e-5)


def test_cauchy_fp64(cuda):
    X, y, _ = synthetic.make_problem(500, 70, 4, seed=9, dtype=np.float64)
    beta = 0.5 * np.random.default_rng(4).standard_normal((1, 3, 70))
    with hmc.create(X, y, 4, "cauchy", 1.0, x_storage="f64", state="f64") as h:
        check(h, X, y, beta, "cauchy", 1.0, cuda, 1e-11, 1e-11)


def test_bitwise_determinism(cuda):
    X, y, _ = synthetic.make_problem(4000, 1000, 10, seed=10)
    beta = (0.05 * np.random.default_rng(5).standard_normal((1, 9, 1000))).astype(np.float32)
    with hmc.create(X, y, 10, "gaussian", 1.0, tile=(4, 0, 0, 0)) as h:
        a = gpu_lpg(h, beta, cuda)
        b = gpu_lpg(h, beta, cuda)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_host_buffers_match_device(cuda):
    X, y, _ = synthetic.make_problem(800, 90, 3, seed=11)
    beta = (0.1 * np.random.default_rng(6).standard_normal((2, 2, 90))).astype(np.float32)
    with hmc.create(X, y, 3, "gaussian", 1.0, max_chains=2) as h:
        lp_h, g_h = h.logpost_grad(beta)            # numpy in, numpy out
        lp_d, g_d = gpu_lpg(h, beta, cuda)
        assert np.array_equal(lp_h, lp_d) and np.array_equal(g_h, g_d)


def test_batch_of_uneven_problems(cuda):
    shapes = [(900, 130, 3), (50, 400, 7), (1500, 64, 2)]
    probs = [synthetic.make_problem(n, p, K, seed=12, sub=i) for i, (n, p, K) in enumerate(shapes)]
    chains = 2
    rng = np.random.default_rng(7)
    betas = [(0.1 * rng.standard_normal((chains, K - 1, p))).astype(np.float32) for (n, p, K) in shapes]
    flat = np.concatenate([b.ravel() for b in betas])
    with hmc.create_batch([pr[0] for pr in probs], [pr[1] for pr in probs], [s[2] for s in shapes],
                          "gaussian", 5.0, max_chains=chains) as h:
        assert h.chain_size == sum((K - 1) * p for (n, p, K) in shapes)
        assert h.describe()["batched_launch"] is True
        lp, g = h.logpost_grad(flat, chains=chains)
        off = 0
        for b, ((X, y, _), (n, p, K)) in enumerate(zip(probs, shapes)):
            lk_o, g_o = oracle_lpg(X, y, betas[b], "gaussian", 5.0)
            gb = g[off:off + chains * (K - 1) * p].reshape(chains, K - 1, p)
            off += chains * (K - 1) * p
            for c in range(chains):
                assert lk_err(lp[b * chains + c], lk_o[c]) <= 1e-5
                assert_grad(gb[c], g_o[c], 1e-5, (b, c))


def test_leapfrog_fp64_matches_oracle_and_reverses(cuda):
    import torch
    X, y, _, spec = synthetic.make_workload("plain_fp64")
    rng = np.random.default_rng(8)
    b0 = 0.05 * rng.standard_normal((1, 2, 50))
    e0 = rng.standard_normal((1, 2, 50))
    with hmc.create(X, y, 3, "gaussian", 10.0, x_storage="f64", state="f64") as h:
        bt = torch.from_numpy(b0.copy()).to(cuda)
        et = torch.from_numpy(e0.copy()).to(cuda)
        gt = torch.empty_like(bt)
        lp = torch.empty(1, dtype=torch.float64, device=cuda)
        h.leapfrog(bt, et, spec["L"], spec["eps"], grad=None, logpost=lp)
        torch.cuda.synchronize()
        b1, e1, lk1, g1 = ohmc.leapfrog(X, y, b0[0], e0[0], spec["eps"], spec["L"], "gaussian", 10.0)
        assert np.max(np.abs(bt.cpu().numpy()[0] - b1)) <= 1e-11
        assert np.max(np.abs(et.cpu().numpy()[0] - e1)) <= 1e-10
        assert lk_err(lp.item(), lk1) <= 1e-11
        # reversibility on the device: negate eta, run L steps back
        et.neg_()
        h.leapfrog(bt, et, spec["L"], spec["eps"], grad=None)
        torch.cuda.synchronize()
        assert np.max(np.abs(bt.cpu().numpy() - b0)) <= 1e-12
        assert np.max(np.abs(-et.cpu().numpy() - e0)) <= 1e-12


def test_sample_fp64_matches_oracle(cuda):
    import torch
    X, y, _, spec = synthetic.make_workload("plain_fp64")
    iters, chains, seed = 25, 2, 1234
    with hmc.create(X, y, 3, "gaussian", 10.0, x_storage="f64", state="f64", max_chains=chains) as h:
        samples = torch.empty((iters, chains, 2, 50), dtype=torch.float64, device=cuda)
        b0 = torch.zeros((chains, 2, 50), dtype=torch.float64, device=cuda)
        stats = h.sample(chains, spec["L"], spec["eps"], iters, seed, beta0=b0, samples=samples)
        ref = ohmc.sample(X, y, 3, "gaussian", 10.0, chains, spec["L"], spec["eps"], iters, seed)
        s = samples.cpu().numpy()
        assert np.max(np.abs(s - ref["samples"])) <= 1e-9
        for c in range(chains):
            assert stats[c]["accepted"] == int(ref["accept"][:, c].sum())
            assert stats[c]["iterations"] == iters
            assert lk_err(stats[c]["logpost"], ref["logk"][-1, c]) <= 1e-10
            assert abs(stats[c]["sum_abs_dH"] - np.abs(ref["dH"][:, c]).sum()) <= 1e-8 * max(1, np.abs(ref["dH"][:, c]).sum())
        # continuing (beta0=None) uses the next iteration indices
        more = torch.empty((5, chains, 2, 50), dtype=torch.float64, device=cuda)
        h.sample(chains, spec["L"], spec["eps"], 5, seed, samples=more)
        ref2 = ohmc.sample(X, y, 3, "gaussian", 10.0, chains, spec["L"], spec["eps"], 5, seed,
                           beta0=ref["beta"], iter0=iters)
        assert np.max(np.abs(more.cpu().numpy() - ref2["samples"])) <= 1e-9


def test_sample_tempered_fp64_matches_oracle(cuda):
    import torch
    X, y, _, _ = synthetic.make_workload("plain_fp64", n=300, p=20)
    iters = 12
    temps = ohmc.annealing_temperatures(iters, t0=50.0, r=0.7)
    with hmc.create(X, y, 3, "cauchy", 1.0, x_storage="f64", state="f64") as h:
        samples = torch.empty((iters, 1, 2, 20), dtype=torch.float64, device=cuda)
        h.sample(1, 10, 0.05, iters, 77, beta0=torch.zeros((1, 2, 20), dtype=torch.float64, device=cuda),
                 samples=samples, temps=temps)
        ref = ohmc.sample(X, y, 3, "cauchy", 1.0, 1, 10, 0.05, iters, 77, temps=temps)
        assert np.max(np.abs(samples.cpu().numpy() - ref["samples"])) <= 1e-9


def test_sample_fp32_reduced_highdim(cuda):
    import torch
    X, y, _, spec = synthetic.make_workload("highdim_fp32", n=2000, p=500)
    iters, L, eps, seed = 8, 20, 2e-3, 5
    with hmc.create(X, y, 10, "gaussian", 1.0) as h:
        samples = torch.empty((iters, 1, 9, 500), dtype=torch.float32, device=cuda)
        stats = h.sample(1, L, eps, iters, seed, beta0=torch.zeros((1, 9, 500), device=cuda), samples=samples)
        ref = ohmc.sample(X, y, 10, "gaussian", 1.0, 1, L, eps, iters, seed)
        s = samples.cpu().numpy().astype(np.float64)
        # FP32 trajectories: same accept decisions away from ties, states within FP32 error.
        # A GPU proposal was accepted iff the sample moved (a proposal never lands on the
        # old state exactly).
        margin = np.abs(ref["dH"][:, 0]) > 1e-3
        assert stats[0]["iterations"] == iters
        scale = np.max(np.abs(ref["samples"])) + 1e-12
        assert np.max(np.abs(s - ref["samples"])) <= 1e-3 * scale
        prev = np.concatenate([np.zeros((1,) + s.shape[1:]), s[:-1]])
        gpu_acc = np.any(s[:, 0] != prev[:, 0], axis=(1, 2))
        assert margin.sum() >= 1
        assert np.array_equal(gpu_acc[margin], ref["accept"][margin, 0]), (gpu_acc, ref["accept"][:, 0], ref["dH"][:, 0])
        assert stats[0]["accepted"] == int(gpu_acc.sum())


def test_timeout_is_reported_and_handle_recovers(cuda):
    X, y, _ = synthetic.make_problem(600, 256, 3, seed=13)
    beta = (0.1 * np.random.default_rng(9).standard_normal((1, 2, 256))).astype(np.float32)
    os.environ["HMC_FAULT"] = "timeout"
    try:
        h = hmc.create(X, y, 3, "gaussian", 1.0, spin_limit=2000, tile=(2, 0, 0, 0))
    finally:
        del os.environ["HMC_FAULT"]
    with h:
        with pytest.raises(hmc.HmcError) as ei:
            h.logpost_grad(beta)
        assert ei.value.status == hmc.ETIMEOUT
        lp, g = h.logpost_grad(beta)          # the handle and the context stay usable
        lk_o, g_o = oracle_lpg(X, y, beta, "gaussian", 1.0)
        assert lk_err(lp[0], lk_o[0]) <= 1e-5
        assert_grad(g[0], g_o[0], 1e-5)


def test_batch_sampling_matches_oracle(cuda):
    """Two problems in one handle, one fused launch per leapfrog step; the
    chains of problem b draw with chain word (b << 32) + c."""
    import torch
    shapes = [(400, 30, 3), (250, 45, 4)]
    probs = [synthetic.make_problem(n, p, K, seed=31, sub=i, dtype=np.float64) for i, (n, p, K) in enumerate(shapes)]
    chains, iters, L, eps, seed = 2, 6, 8, 0.02, 99
    with hmc.create_batch([pr[0] for pr in probs], [pr[1] for pr in probs], [s[2] for s in shapes], "cauchy", 1.0,
                          x_storage="f64", state="f64", max_chains=chains) as h:
        assert h.describe()["batched_launch"] is True
        size = chains * h.chain_size
        samples = torch.empty((iters, size), dtype=torch.float64, device=cuda)
        b0 = torch.zeros(size, dtype=torch.float64, device=cuda)
        h.sample(chains, L, eps, iters, seed, beta0=b0, samples=samples)
        s = samples.cpu().numpy()
        off = 0
        for b, ((X, y, _), (n, p, K)) in enumerate(zip(probs, shapes)):
            blk = chains * (K - 1) * p
            ref = ohmc.sample(X, y, K, "cauchy", 1.0, chains, L, eps, iters, seed, chain0=b << 32)
            got = s[:, off:off + blk].reshape(iters, chains, K - 1, p)
            assert np.max(np.abs(got - ref["samples"])) <= 1e-9
            off += blk
