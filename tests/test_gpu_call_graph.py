"""Repeated hmc_logpost_grad / hmc_leapfrog calls on the same device buffers
are captured as a CUDA graph on the second call and replayed afterwards: the
graph bakes the buffers' addresses, never their contents.  These tests change
the contents between calls (and the buffers, chains, L and eps now and then) and
check every call against the FP64 oracle (1e-11) or, for the reduced-precision
engines, against the first, uncaptured call bit for bit."""
import numpy as np
import pytest

from oracle import hmc as ohmc
from oracle import model
from paper_1402_4089_gb300 import hmc, synthetic
from parity_util import assert_grad, lk_err

pytestmark = pytest.mark.gpu


def test_logpost_grad_replays_follow_buffer_contents(cuda):
    import torch
    n, p, K, chains = 600, 70, 5, 2
    X, y, _ = synthetic.make_problem(n, p, K, seed=71, dtype=np.float64)
    rng = np.random.default_rng(72)
    with hmc.create(X, y, K, "cauchy", 1.0, x_storage="f64", state="f64", max_chains=chains) as h:
        beta = torch.zeros((chains, K - 1, p), dtype=torch.float64, device=cuda)
        g = torch.empty_like(beta)
        lp = torch.empty(chains, dtype=torch.float64, device=cuda)
        g2 = torch.empty_like(beta)
        for it in range(7):
            b = 0.2 * rng.standard_normal((chains, K - 1, p))
            beta.copy_(torch.from_numpy(b))
            out = g2 if it == 4 else g                 # call 5 uses another gradient buffer
            h.logpost_grad(beta, logpost=lp, grad=out)
            torch.cuda.synchronize()
            gc, lc = out.cpu().numpy(), lp.cpu().numpy()
            for c in range(chains):
                assert lk_err(lc[c], model.log_kernel(X, y, b[c], "cauchy", 1.0)) <= 1e-11, (it, c)
                assert_grad(gc[c], model.grad_log_kernel(X, y, b[c], "cauchy", 1.0), 1e-11, (it, c))
        # fewer chains than the captured call: a new key, still correct
        b = 0.2 * rng.standard_normal((1, K - 1, p))
        one = torch.from_numpy(b).to(cuda)
        lp1, g1 = h.logpost_grad(one)
        torch.cuda.synchronize()
        assert_grad(g1.cpu().numpy()[0], model.grad_log_kernel(X, y, b[0], "cauchy", 1.0), 1e-11, "one chain")


def test_leapfrog_replays_continue_the_trajectory(cuda):
    import torch
    n, p, K, L, eps = 400, 30, 4, 5, 0.02
    X, y, _ = synthetic.make_problem(n, p, K, seed=73, dtype=np.float64)
    rng = np.random.default_rng(74)
    b0 = 0.1 * rng.standard_normal((1, K - 1, p))
    e0 = rng.standard_normal((1, K - 1, p))
    with hmc.create(X, y, K, "gaussian", 2.0, x_storage="f64", state="f64") as h:
        beta = torch.from_numpy(b0.copy()).to(cuda)
        eta = torch.from_numpy(e0.copy()).to(cuda)
        g = torch.empty_like(beta)
        lp = torch.empty(1, dtype=torch.float64, device=cuda)
        h.logpost_grad(beta, logpost=lp, grad=g)       # the input gradient of the first call
        bo, eo = b0[0], e0[0]
        for it in range(6):
            step = eps if it != 3 else 0.5 * eps        # call 4 changes eps: a new graph
            h.leapfrog(beta, eta, L, step, grad=g, logpost=lp)
            torch.cuda.synchronize()
            bo, eo, lko, go = ohmc.leapfrog(X, y, bo, eo, step, L, "gaussian", 2.0)
            assert np.max(np.abs(beta.cpu().numpy()[0] - bo)) <= 1e-11, it
            assert np.max(np.abs(eta.cpu().numpy()[0] - eo)) <= 1e-10, it
            assert lk_err(lp.item(), lko) <= 1e-11, it
            assert_grad(g.cpu().numpy()[0], go, 1e-10, it)


@pytest.mark.parametrize("storage,engine", [("bf16", 3), ("bf16", 2), ("f32", 4), ("f32", 1)])
def test_replays_bitwise_equal_first_call(cuda, storage, engine):
    import torch
    n, p, K, chains = 3000, 640, 6, 3
    X, y, _ = synthetic.make_problem(n, p, K, seed=75)
    beta = (0.05 * np.random.default_rng(76).standard_normal((chains, K - 1, p))).astype(np.float32)
    with hmc.create(X, y, K, "gaussian", 1.0, x_storage=storage, max_chains=chains, engine=engine) as h:
        bt = torch.from_numpy(beta).to(cuda)
        g = torch.empty_like(bt)
        lp = torch.empty(chains, dtype=torch.float64, device=cuda)
        ref = None
        for it in range(5):
            g.zero_()
            lp.zero_()
            h.logpost_grad(bt, logpost=lp, grad=g)
            torch.cuda.synchronize()
            cur = (lp.cpu().numpy().copy(), g.cpu().numpy().copy())
            if ref is None:
                ref = cur
            assert np.array_equal(cur[0], ref[0]) and np.array_equal(cur[1], ref[1]), it
