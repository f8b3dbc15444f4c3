"""The two-pass tensor-core engine (opts.engine = 3, BF16 or per-column-scaled
FP8 X): pass A forms the logits, softmax and residual of every (row tile, chain
group), pass B the partial gradients X^T R; against the FP64 oracle on the
stored X (FP8: codes and scales bit-exact against the oracle's quantisation,
the codes widened to BF16 in shared memory, the scales folded into the
coefficients and the gradient).

Same operand precision as the fused tensor-core engine (two-term BF16
coefficients, BF16 residual, FP32 accumulation), so the same gates: gradient
3e-3 relative in norm and element-wise, log K 1e-4."""
import os

import numpy as np
import pytest

from oracle import model, quant
from paper_1402_4089_gb300 import hmc, synthetic
from parity_util import grad_errs, lk_err

pytestmark = pytest.mark.gpu

TOL_G, TOL_L = 3e-3, 1e-4


def _run(cuda, n, p, K, chains, seed, layout="free", prior=("gaussian", 10.0), bscale=0.05, U=0, storage="bf16"):
    import torch
    X, y, _ = synthetic.make_problem(n, p, K, seed=seed)
    rows = K - 1 if layout == "free" else K
    beta = (bscale * np.random.default_rng(seed + 1).standard_normal((chains, rows, p))).astype(np.float32)
    with hmc.create(X, y, K, prior[0], prior[1], x_storage=storage, max_chains=chains, engine=3, layout=layout,
                    tile=(U, 0, 0, 0)) as h:
        d = h.describe()
        assert d["engine"] == "tcgen05_2pass", d
        bits, scales = h.get_x()
        lp, g = h.logpost_grad(torch.from_numpy(beta).to(cuda))
        torch.cuda.synchronize()
        lp, g = lp.cpu().numpy(), g.cpu().numpy()
    if storage == "fp8":
        c_o, s_o = quant.fp8_quantize(X)
        assert np.array_equal(scales, s_o) and np.array_equal(bits, c_o)
        Xq = quant.fp8_dequantize(bits, scales).astype(np.float64)
    else:
        Xq = quant.bf16_decode(bits).astype(np.float64)
    for c in range(chains):
        lk_o = model.log_kernel_layout(Xq, y, beta[c], prior[0], prior[1], layout)
        g_o = model.grad_log_kernel_layout(Xq, y, beta[c], prior[0], prior[1], layout)
        el = lk_err(lp[c], lk_o)
        eg, ee = grad_errs(g[c], g_o)
        assert el <= TOL_L and eg <= TOL_G and ee <= TOL_G, (d["problems"][0], c, el, eg, ee)
    return d


@pytest.mark.parametrize("n,p,K,chains", [(1000, 700, 6, 2), (333, 129, 3, 1), (2049, 1000, 20, 4), (128, 64, 2, 3),
                                          (5000, 2000, 10, 7), (130, 4100, 5, 1), (257, 300, 33, 1)])
def test_tc2_matches_oracle(cuda, n, p, K, chains):
    _run(cuda, n, p, K, chains, seed=n + 7 * p)


@pytest.mark.parametrize("n,p,K,chains,U", [(700, 300, 2, 40, 0), (600, 200, 33, 8, 0), (900, 250, 17, 5, 0),
                                            (500 * 128 + 77, 300, 11, 6, 3)])
def test_tc2_epilogue_chain_layouts(cuda, n, p, K, chains, U):
    """Chain layouts of the softmax epilogue: one column per chain (K = 2, 40
    chains: a chain ends at every column), 32 columns per chain (K = 33, each
    chain over two or three 16-column blocks, 8 chains in groups), chains of
    exactly one block (K = 17), and units split over two CTAs with 60 columns
    (the other CTA's partial logits added to four blocks per tile)."""
    _run(cuda, n, p, K, chains, seed=n + 13 * K, U=U)


@pytest.mark.parametrize("U,n", [(2, 10 * 128 + 5), (3, 10 * 128 + 5), (3, 9 * 128), (4, 3 * 128 + 1)])
def test_tc2_row_tiles_per_unit(cuda, U, n):
    """Several row tiles per first-pass unit sharing each coefficient box, with a
    last unit that holds fewer tiles."""
    d = _run(cuda, n, 1000, 6, 2, seed=70 + U, U=U)
    assert d["problems"][0]["pass_a"]["tiles_per_unit"] == U


@pytest.mark.parametrize("U,n,p", [(1, 200 * 128 + 37, 512), (2, 400 * 128 + 5, 300), (3, 500 * 128, 200)])
def test_tc2_units_split_over_two_ctas(cuda, U, n, p):
    """More first-pass units than SMs: every CTA takes an even share of the
    (unit, feature box) steps, so units are split between neighbouring CTAs and
    finished by the one holding their first boxes."""
    d = _run(cuda, n, p, 4, 2, seed=80 + U, U=U)
    pa = d["problems"][0]["pass_a"]
    assert pa["tiles_per_unit"] == U and pa["grid"] < (n + 128 * U - 1) // (128 * U)


@pytest.mark.parametrize("n,p,K,chains,U", [(1000, 700, 6, 2, 0), (333, 129, 3, 1, 0), (2049, 1000, 20, 4, 0),
                                            (5000, 2000, 10, 7, 0), (10 * 128 + 5, 1000, 6, 2, 4),
                                            (200 * 128 + 37, 512, 4, 2, 1), (3000, 500, 10, 40, 0)])
def test_tc2_fp8_matches_oracle(cuda, n, p, K, chains, U):
    """FP8 X: ragged rows and features, up to four tiles per unit (the widest
    converter load), units split over two CTAs, several chain groups."""
    _run(cuda, n, p, K, chains, seed=n + 11 * p, U=U, storage="fp8")


@pytest.mark.parametrize("layout", ["masked", "unconstrained"])
def test_tc2_fp8_layouts(cuda, layout):
    _run(cuda, 1500, 400, 6, 3, seed=73, layout=layout, prior=("cauchy", 1.0), storage="fp8")


def test_tc2_many_chains_in_groups(cuda):
    d = _run(cuda, 3000, 500, 10, 64, seed=71)
    pa = d["problems"][0]["pass_a"]
    assert pa["chain_group"] < 64                      # several chain groups inside the two launches


@pytest.mark.parametrize("layout", ["masked", "unconstrained"])
def test_tc2_layouts(cuda, layout):
    _run(cuda, 1500, 400, 6, 3, seed=72, layout=layout, prior=("cauchy", 1.0))


def test_tc2_deterministic_and_one_launch_pair(cuda):
    import torch
    X, y, _ = synthetic.make_problem(3000, 1500, 8, seed=73)
    beta = torch.from_numpy((0.05 * np.random.default_rng(74).standard_normal((9, 7, 1500))).astype(np.float32)).to(cuda)
    with hmc.create(X, y, 8, "gaussian", 10.0, x_storage="bf16", max_chains=9, engine=3) as h:
        h.set_timing(True)
        a = [t.cpu().numpy() for t in h.logpost_grad(beta)]
        assert h.fused_kernel_time()[1] == 1          # both passes inside one timed pair of events
        b = [t.cpu().numpy() for t in h.logpost_grad(beta)]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_tc2_sampling_follows_the_fused_engine(cuda):
    """The same chains on both tensor-core engines: identical momenta and accept
    draws, gradients equal to rounding, so the samples agree closely."""
    import torch
    X, y, _ = synthetic.make_problem(2000, 300, 5, seed=75)
    out = []
    for engine in (2, 3):
        with hmc.create(X, y, 5, "gaussian", 10.0, x_storage="bf16", max_chains=2, engine=engine) as h:
            s = torch.empty((6, 2, 4, 300), dtype=torch.float32, device=cuda)
            st = h.sample(2, 10, 0.005, 6, 9, beta0=torch.zeros((2, 4, 300), device=cuda), samples=s)
            out.append((s.cpu().numpy(), [x["accepted"] for x in st]))
    assert out[0][1] == out[1][1]
    scale = np.abs(out[0][0]).max()
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-3 * scale


def test_tc2_timeout_is_reported_and_handle_recovers(cuda):
    import torch
    X, y, _ = synthetic.make_problem(600, 256, 3, seed=76)
    beta = torch.from_numpy((0.1 * np.random.default_rng(77).standard_normal((1, 2, 256))).astype(np.float32)).to(cuda)
    os.environ["HMC_FAULT"] = "timeout"
    try:
        h = hmc.create(X, y, 3, "gaussian", 1.0, x_storage="bf16", engine=3)
    finally:
        del os.environ["HMC_FAULT"]
    with h:
        with pytest.raises(hmc.HmcError) as ei:
            h.logpost_grad(beta.cpu().numpy())        # host buffers: the call reads the error word
        assert ei.value.status == hmc.ETIMEOUT
        lp, g = h.logpost_grad(beta.cpu().numpy())
        bits, _ = h.get_x()
    Xq = quant.bf16_decode(bits).astype(np.float64)
    b = beta.cpu().numpy()[0].astype(np.float64)
    assert lk_err(lp[0], model.log_kernel(Xq, y, b, "gaussian", 1.0)) <= TOL_L
    assert max(grad_errs(g[0], model.grad_log_kernel(Xq, y, b, "gaussian", 1.0))) <= TOL_G


@pytest.mark.parametrize("engine", [3, 2])
def test_fp8_every_code_widened_exactly(cuda, engine):
    """Column 5 of X holds every finite E4M3 code (zeros, subnormals, both signs,
    +-448): the stored codes match the oracle's quantisation bit for bit and the
    gradient matches the oracle on the dequantised X, so every widening path
    (the field arithmetic for normal codes, the exact conversion otherwise) is
    exact."""
    import torch
    n, p, K, chains = 700, 130, 4, 2
    X, y, _ = synthetic.make_problem(n, p, K, seed=91)
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF)])
    s = np.float32(0.01)
    col = (quant.e4m3_table()[codes] * s).astype(np.float32)
    X[:, 5] = np.resize(col, n)
    rng = np.random.default_rng(92)
    beta = (0.05 * rng.standard_normal((chains, K - 1, p))).astype(np.float32)
    with hmc.create(X, y, K, "gaussian", 10.0, x_storage="fp8", max_chains=chains, engine=engine) as h:
        bits, scales = h.get_x()
        lp, g = h.logpost_grad(torch.from_numpy(beta).to(cuda))
        torch.cuda.synchronize()
        lp, g = lp.cpu().numpy(), g.cpu().numpy()
    c_o, s_o = quant.fp8_quantize(X)
    assert np.array_equal(scales, s_o) and np.array_equal(bits, c_o)
    assert set(np.unique(bits[:, 5])) == set(codes.tolist())
    Xq = quant.fp8_dequantize(bits, scales).astype(np.float64)
    for c in range(chains):
        lk_o = model.log_kernel(Xq, y, beta[c], "gaussian", 10.0)
        g_o = model.grad_log_kernel(Xq, y, beta[c], "gaussian", 10.0)
        eg, ee = grad_errs(g[c], g_o)
        assert lk_err(lp[c], lk_o) <= TOL_L and eg <= TOL_G and ee <= TOL_G, (c, eg, ee)
        # column 5 alone: its gradient entries depend on every code's value
        assert np.max(np.abs(g[c][:, 5] - g_o[:, 5])) <= TOL_G * max(np.abs(g_o[:, 5]).max(), 1e-30)


def test_tc2_sample_64_chains_follows_the_fused_engine(cuda):
    """64 chains in one launch pair (two-pass) against the fused engine, which
    needs several launches for them: same momenta and accept draws, gradients
    equal to rounding, so every chain's samples and accept counts agree."""
    import torch
    n, p, K, chains, iters = 3000, 256, 4, 64, 4
    X, y, _ = synthetic.make_problem(n, p, K, seed=93)
    out = []
    for engine in (3, 2):
        with hmc.create(X, y, K, "gaussian", 10.0, x_storage="bf16", max_chains=chains, engine=engine) as h:
            d = h.describe()
            if engine == 2:
                assert d["problems"][0]["group_chains"] < chains        # several fused launches
            s = torch.empty((iters, chains, K - 1, p), dtype=torch.float32, device=cuda)
            st = h.sample(chains, 8, 0.004, iters, 17, beta0=torch.zeros((chains, K - 1, p), device=cuda), samples=s)
            out.append((s.cpu().numpy(), [x["accepted"] for x in st]))
    assert out[0][1] == out[1][1]
    scale = np.abs(out[1][0]).max()
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-3 * scale


def test_tc2_tempered_sampling_follows_the_fused_engine(cuda):
    """Annealed iterations (Sec. 3.2 schedule through the library) on the two-pass
    engine against the fused engine: same accept decisions, close samples."""
    import torch
    X, y, _ = synthetic.make_problem(1500, 200, 5, seed=94)
    iters = 8
    temps = hmc.annealing_temperatures(iters, t0=20.0, r=0.6)
    out = []
    for engine in (3, 2):
        with hmc.create(X, y, 5, "cauchy", 1.0, x_storage="bf16", max_chains=2, engine=engine) as h:
            s = torch.empty((iters, 2, 4, 200), dtype=torch.float32, device=cuda)
            st = h.sample(2, 6, 0.01, iters, 21, beta0=torch.zeros((2, 4, 200), device=cuda), samples=s, temps=temps)
            out.append((s.cpu().numpy(), [x["accepted"] for x in st]))
    assert out[0][1] == out[1][1]
    scale = np.abs(out[1][0]).max()
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-3 * scale
