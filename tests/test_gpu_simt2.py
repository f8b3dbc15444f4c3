"""The two-pass CUDA-core engine (engine 4: row logits, softmax, residual and
row log-likelihoods in a first pass, X^T R in a second) against the FP64
oracle: the wide Table 1 shapes it exists for (FP32 X, K = 15 and 20 at
p = 20000, where the fused CUDA-core pass has no tile), both models of Figs 1-4,
FP64 X with more classes than the fused pass handles, forced small and ragged
shapes (several chain groups, one row, one feature, 64 columns per launch), the
masked layout, determinism and the leapfrog integrator.

Tolerances as in test_gpu_parity: FP32 arithmetic 1e-5, FP64 1e-11 (gradient
in norm and element-wise per chain; log K relative to max(1, |log K|))."""
import numpy as np
import pytest

from oracle import hmc as ohmc
from oracle import model
from paper_1402_4089_gb300 import hmc, synthetic
from parity_util import assert_grad, lk_err

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-11}


def _lpg(h, beta, dev):
    import torch
    lp, g = h.logpost_grad(torch.from_numpy(np.ascontiguousarray(beta)).to(dev))
    torch.cuda.synchronize()
    return lp.cpu().numpy(), g.cpu().numpy()


def _check(h, X, y, beta, kind, scale, layout, tol, dev):
    lp, g = _lpg(h, beta, dev)
    X64 = np.asarray(X, np.float64)
    for c in range(beta.shape[0]):
        b = beta[c].astype(np.float64)
        lk_o = model.log_kernel_layout(X64, y, b, kind, scale, layout)
        g_o = model.grad_log_kernel_layout(X64, y, b, kind, scale, layout)
        assert lk_err(lp[c], lk_o) <= tol, (c, lp[c], lk_o)
        if layout == "masked":
            assert np.all(g[c, -1] == 0.0)
            assert_grad(g[c, :-1], g_o[:-1], tol, c)
        else:
            assert_grad(g[c], g_o, tol, c)
    return lp, g


@pytest.mark.parametrize("layout", ["free", "unconstrained"])
@pytest.mark.parametrize("K", [15, 20])
def test_table1_wide_shapes(cuda, layout, K):
    """N = 1000, p = 20000: chosen by default, at the sweep's own inputs."""
    n, p = 1000, 20000
    X, y, B = synthetic.sweep_problem(n, p, K)
    if layout == "unconstrained":
        B = np.concatenate([B, np.zeros((1, p))])
    beta = B.astype(np.float32)[None]
    with hmc.create(X, y, K, "cauchy", 1.0, x_storage="f32", layout=layout) as h:
        d = h.describe()
        assert d["engine"] == "simt_2pass", d
        _check(h, X, y, beta, "cauchy", 1.0, layout, TOL["f32"], cuda)


def test_fp64_beyond_fused_class_bound(cuda):
    """FP64 X with K - 1 = 19 free classes (the fused FP64 pass takes at most 12)."""
    X, y, _ = synthetic.make_problem(700, 90, 20, seed=61, dtype=np.float64)
    beta = 0.2 * np.random.default_rng(62).standard_normal((2, 19, 90))
    with hmc.create(X, y, 20, "gaussian", 3.0, x_storage="f64", state="f64", max_chains=2) as h:
        assert h.describe()["engine"] == "simt_2pass"
        _check(h, X, y, beta, "gaussian", 3.0, "free", TOL["f64"], cuda)


@pytest.mark.parametrize("xs", ["f32", "f64"])
@pytest.mark.parametrize("n,p,K,chains", [(1013, 300, 4, 2), (1, 5, 2, 1), (37, 1, 2, 3), (100, 33, 21, 3),
                                          (257, 130, 65, 1), (2049, 517, 21, 5), (64, 4, 9, 8)])
def test_forced_shapes(cuda, xs, n, p, K, chains):
    """Ragged rows and features, C from 1 to 64 columns per launch, 5 chains of
    20 classes in two chain groups (3 + 2)."""
    dt = np.float64 if xs == "f64" else np.float32
    rng = np.random.default_rng(n * 7 + p + K)
    X = rng.standard_normal((n, p)).astype(dt)
    y = rng.integers(0, K, size=n).astype(np.int32)
    if n > 3:
        y[:3] = K - 1
    beta = (0.3 * rng.standard_normal((chains, K - 1, p))).astype(dt)
    with hmc.create(X, y, K, "cauchy", 1.0, x_storage=xs, state=xs, max_chains=chains, engine=4) as h:
        d = h.describe()
        assert d["engine"] == "simt_2pass"
        g = min(chains, 64 // (K - 1))
        assert d["problems"][0]["group_chains"] == -(-chains // -(-chains // g))   # even split over the launches
        _check(h, X, y, beta, "cauchy", 1.0, "free", TOL[xs], cuda)


@pytest.mark.parametrize("layout", ["masked", "unconstrained"])
def test_forced_layouts(cuda, layout):
    n, p, K, chains = 1037, 300, 5, 2
    X, y, _ = synthetic.make_problem(n, p, K, seed=63)
    beta = (0.1 * np.random.default_rng(64).standard_normal((chains, K, p))).astype(np.float32)
    if layout == "masked":
        beta[:, -1] = 5.0                          # row K of an input is ignored
    with hmc.create(X, y, K, "cauchy", 1.0, max_chains=chains, engine=4, layout=layout) as h:
        assert h.rows() == K
        _check(h, X, y, beta, "cauchy", 1.0, layout, TOL["f32"], cuda)


def test_deterministic_and_matches_fused_engine(cuda):
    """Bitwise repeatable; within FP32 rounding of the fused CUDA-core engine."""
    X, y, _ = synthetic.make_problem(4000, 1000, 10, seed=65)
    beta = (0.05 * np.random.default_rng(66).standard_normal((2, 9, 1000))).astype(np.float32)
    out = {}
    for engine in (1, 4):
        with hmc.create(X, y, 10, "gaussian", 1.0, max_chains=2, engine=engine) as h:
            a = _lpg(h, beta, cuda)
            b = _lpg(h, beta, cuda)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
            out[engine] = a
    for c in range(2):
        assert lk_err(out[4][0][c], out[1][0][c]) <= 1e-5
        assert_grad(out[4][1][c], out[1][1][c], 1e-5, c)


def test_leapfrog_fp64_matches_oracle(cuda):
    """L leapfrog steps of Eq. 5 on engine 4 (FP64) against the oracle's integrator."""
    import torch
    n, p, K, L, eps = 400, 40, 14, 6, 0.01
    X, y, _ = synthetic.make_problem(n, p, K, seed=67, dtype=np.float64)
    rng = np.random.default_rng(68)
    b0 = 0.1 * rng.standard_normal((1, K - 1, p))
    e0 = rng.standard_normal((1, K - 1, p))
    with hmc.create(X, y, K, "gaussian", 2.0, x_storage="f64", state="f64", engine=4) as h:
        beta = torch.from_numpy(b0.copy()).to(cuda)
        eta = torch.from_numpy(e0.copy()).to(cuda)
        lp = torch.empty(1, dtype=torch.float64, device=cuda)
        h.leapfrog(beta, eta, L, eps, logpost=lp)
        torch.cuda.synchronize()
        bg, eg = beta.cpu().numpy()[0], eta.cpu().numpy()[0]
    bo, eo, lko, _ = ohmc.leapfrog(X, y, b0[0], e0[0], eps, L, "gaussian", 2.0)
    assert np.max(np.abs(bg - bo)) <= 1e-11 * max(1.0, np.max(np.abs(bo)))
    assert np.max(np.abs(eg - eo)) <= 1e-10 * max(1.0, np.max(np.abs(eo)))
    assert lk_err(lp.item(), lko) <= 1e-11


@pytest.mark.parametrize("layout", ["free", "unconstrained"])
def test_sample_fp64_matches_oracle(cuda, layout):
    """HMC iterations (one captured graph each) on engine 4 in FP64: samples,
    accept decisions and log K against the oracle's sampler, two chains, then a
    continuation from the saved state."""
    import torch
    n, p, K, chains, iters, seed, L, eps = 300, 24, 6, 2, 12, 4321, 8, 0.02
    X, y, _ = synthetic.make_problem(n, p, K, seed=69, dtype=np.float64)
    rows = K - 1 if layout == "free" else K
    with hmc.create(X, y, K, "gaussian", 5.0, x_storage="f64", state="f64", max_chains=chains, engine=4,
                    layout=layout) as h:
        assert h.describe()["engine"] == "simt_2pass"
        samples = torch.empty((iters, chains, rows, p), dtype=torch.float64, device=cuda)
        b0 = torch.zeros((chains, rows, p), dtype=torch.float64, device=cuda)
        stats = h.sample(chains, L, eps, iters, seed, beta0=b0, samples=samples)
        ref = ohmc.sample(X, y, K, "gaussian", 5.0, chains, L, eps, iters, seed, layout=layout)
        assert np.max(np.abs(samples.cpu().numpy() - ref["samples"])) <= 1e-9
        for c in range(chains):
            assert stats[c]["accepted"] == int(ref["accept"][:, c].sum())
            assert lk_err(stats[c]["logpost"], ref["logk"][-1, c]) <= 1e-10
        more = torch.empty((4, chains, rows, p), dtype=torch.float64, device=cuda)
        h.sample(chains, L, eps, 4, seed, samples=more)
        ref2 = ohmc.sample(X, y, K, "gaussian", 5.0, chains, L, eps, 4, seed, beta0=ref["beta"], iter0=iters,
                           layout=layout)
        assert np.max(np.abs(more.cpu().numpy() - ref2["samples"])) <= 1e-9


def test_sample_fp32_wide_default_engine(cuda):
    """The default engine for a wide FP32 problem (engine 4) samples within FP32
    rounding of the fused CUDA-core engine over a few iterations: same accept
    decisions where |dH| is not near the threshold, samples close."""
    import torch
    n, p, K, chains, iters, seed = 2000, 2100, 8, 3, 4, 99      # C = 21 columns: the default is engine 4
    X, y, _ = synthetic.make_problem(n, p, K, seed=70)
    out = {}
    for engine in (0, 1):
        with hmc.create(X, y, K, "gaussian", 1.0, max_chains=chains, engine=engine) as h:
            out[engine] = [h.describe()["engine"]]
            s = torch.empty((iters, chains, K - 1, p), dtype=torch.float32, device=cuda)
            st = h.sample(chains, 5, 0.002, iters, seed, beta0=torch.zeros((chains, K - 1, p), device=cuda), samples=s)
            out[engine] += [s.cpu().numpy(), [x["accepted"] for x in st]]
    assert out[0][0] == "simt_2pass" and out[1][0] == "simt"
    assert out[0][2] == out[1][2]
    scale = max(1e-6, np.abs(out[1][1]).max())
    assert np.max(np.abs(out[0][1] - out[1][1])) <= 1e-4 * scale


def test_tempered_sampling_fp32_follows_the_fused_engine(cuda):
    """Annealed iterations on engine 4 (FP32) against the fused CUDA-core engine."""
    import torch
    n, p, K, iters = 1200, 150, 6, 8
    X, y, _ = synthetic.make_problem(n, p, K, seed=95)
    temps = hmc.annealing_temperatures(iters, t0=20.0, r=0.6)
    out = []
    for engine in (4, 1):
        with hmc.create(X, y, K, "gaussian", 2.0, max_chains=2, engine=engine) as h:
            s = torch.empty((iters, 2, K - 1, p), dtype=torch.float32, device=cuda)
            st = h.sample(2, 6, 0.01, iters, 23, beta0=torch.zeros((2, K - 1, p), device=cuda), samples=s, temps=temps)
            out.append((s.cpu().numpy(), [x["accepted"] for x in st]))
    assert out[0][1] == out[1][1]
    scale = max(1e-6, np.abs(out[1][0]).max())
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-4 * scale
