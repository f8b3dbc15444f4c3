"""The coefficient layouts of the Appendix on the GPU against the oracle:
HMC_LAYOUT_MASKED (K rows per chain, row K held at zero by the mask M) and
HMC_LAYOUT_UNCONSTRAINED (K free rows, identifiability not enforced), on the
CUDA-core engine (FP64 and FP32) and the tensor-core engine (BF16 X), plus the
sampler in both layouts.  Tolerances as in test_gpu_parity / test_gpu_tc."""
import numpy as np
import pytest

from oracle import hmc as ohmc
from oracle import model, quant
from paper_1402_4089_gb300 import hmc, synthetic
from parity_util import assert_grad, lk_err

pytestmark = pytest.mark.gpu


def _lpg(h, beta, dev):
    import torch
    lp, g = h.logpost_grad(torch.from_numpy(np.ascontiguousarray(beta)).to(dev))
    torch.cuda.synchronize()
    return lp.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("layout", ["masked", "unconstrained"])
@pytest.mark.parametrize("xs,engine,tol_g,tol_l", [("f64", 1, 1e-11, 1e-11), ("f32", 1, 1e-5, 1e-5),
                                                    ("bf16", 2, 3e-3, 1e-4)])
def test_layout_logpost_grad(cuda, layout, xs, engine, tol_g, tol_l):
    n, p, K, chains = 1037, 300, 5, 2
    X, y, _ = synthetic.make_problem(n, p, K, seed=51, dtype=np.float64 if xs == "f64" else np.float32)
    rng = np.random.default_rng(52)
    dt = np.float64 if xs == "f64" else np.float32
    beta = (0.1 * rng.standard_normal((chains, K, p))).astype(dt)
    if layout == "masked":
        beta[:, -1] = 5.0                          # row K of an input is ignored
    with hmc.create(X, y, K, "cauchy", 1.0, x_storage=xs, state="f64" if xs == "f64" else "f32",
                    max_chains=chains, engine=engine, layout=layout) as h:
        assert h.chain_size == K * p and h.rows() == K
        assert h.describe()["engine"] == ("tcgen05" if engine == 2 else "simt")
        lp, g = _lpg(h, beta, cuda)
        bits, _ = h.get_x()
    Xq = quant.bf16_decode(bits).astype(np.float64) if xs == "bf16" else np.asarray(X, np.float64)
    for c in range(chains):
        lk_o = model.log_kernel_layout(Xq, y, beta[c], "cauchy", 1.0, layout)
        g_o = model.grad_log_kernel_layout(Xq, y, beta[c], "cauchy", 1.0, layout)
        assert lk_err(lp[c], lk_o) <= tol_l, (c, lp[c], lk_o)
        if layout == "masked":
            assert np.all(g[c, -1] == 0.0)
            assert_grad(g[c, :-1], g_o[:-1], tol_g, c)
        else:
            assert_grad(g[c], g_o, tol_g, c)


def test_masked_chains_equal_free_chains_bitwise(cuda):
    import torch
    n, p, K, chains, iters = 500, 64, 4, 2, 5
    X, y, _ = synthetic.make_problem(n, p, K, seed=53)
    out = {}
    for layout in ("free", "masked"):
        rows = K - 1 if layout == "free" else K
        with hmc.create(X, y, K, "gaussian", 5.0, max_chains=chains, layout=layout) as h:
            s = torch.empty((iters, chains, rows, p), dtype=torch.float32, device=cuda)
            st = h.sample(chains, 8, 0.02, iters, 3, beta0=torch.zeros((chains, rows, p), device=cuda), samples=s)
            out[layout] = (s.cpu().numpy(), [x["accepted"] for x in st])
    assert np.array_equal(out["masked"][0][:, :, :-1], out["free"][0])
    assert np.all(out["masked"][0][:, :, -1] == 0.0)
    assert out["masked"][1] == out["free"][1]


def test_unconstrained_sampling_fp64_matches_oracle(cuda):
    import torch
    X, y, _ = synthetic.make_problem(300, 20, 3, seed=54, dtype=np.float64)
    chains, iters, L, eps, seed = 2, 10, 10, 0.03, 55
    with hmc.create(X, y, 3, "gaussian", 3.0, x_storage="f64", state="f64", max_chains=chains,
                    layout="unconstrained") as h:
        s = torch.empty((iters, chains, 3, 20), dtype=torch.float64, device=cuda)
        stats = h.sample(chains, L, eps, iters, seed, beta0=torch.zeros((chains, 3, 20), dtype=torch.float64,
                                                                          device=cuda), samples=s)
    ref = ohmc.sample(X, y, 3, "gaussian", 3.0, chains, L, eps, iters, seed, layout="unconstrained")
    assert np.max(np.abs(s.cpu().numpy() - ref["samples"])) <= 1e-9
    for c in range(chains):
        assert stats[c]["accepted"] == int(ref["accept"][:, c].sum())
