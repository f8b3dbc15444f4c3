"""The autograd op over the fused kernel: backward equals the adjoint gradient,
which is checked against the FP64 oracle's gradient and against central finite
differences of the FP64 oracle's log K (h = 1e-4) on sampled coordinates.

Finite differences of log K along coordinate (k, j) only move logit column k
by h * x_j, so each difference is evaluated from the oracle's logits plus that
shift (the same function of beta, without recomputing X B)."""
import numpy as np
import pytest

from oracle import model, quant
from paper_1402_4089_gb300 import autograd, hmc, synthetic

pytestmark = pytest.mark.gpu


def _fd(Xq, y, beta, k, j, h, kind, scale):
    Z = model.full_logits(Xq, beta)
    out = []
    for sgn in (1.0, -1.0):
        Zs = Z.copy()
        Zs[:, k] += sgn * h * Xq[:, j]
        b = beta.copy()
        b[k, j] += sgn * h
        ll = model.log_softmax(Zs)[np.arange(len(y)), y].sum()
        out.append(ll + model.prior_terms(b, kind, scale).sum())
    return (out[0] - out[1]) / (2 * h)


@pytest.mark.parametrize("xdt,engine,tol", [("f32", 1, 1e-5), ("bf16", 2, 1e-2)])
def test_autograd_backward_is_the_adjoint(cuda, xdt, engine, tol):
    import torch
    n, p, K, chains = 6000, 1500, 10, 3
    X, y, btrue, _ = synthetic.make_workload("autodiff", n=n, p=p)
    with hmc.create(X, y, K, "gaussian", 10.0, x_storage=xdt, max_chains=chains, engine=engine) as h:
        Xq = X.astype(np.float64) if xdt == "f32" else quant.bf16_decode(h.get_x()[0]).astype(np.float64)
        rng = np.random.default_rng(3)
        b0 = (0.02 * rng.standard_normal((chains, K - 1, p))).astype(np.float32)
        beta = torch.from_numpy(b0).to(cuda).requires_grad_(True)
        lp = autograd.log_posterior(beta, h)
        w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device=cuda)
        (lp * w).sum().backward()
        gb = beta.grad.cpu().numpy().astype(np.float64)
        _, gdir = h.logpost_grad(beta.detach())
        gdir = gdir.cpu().numpy().astype(np.float64)
        for c in range(chains):
            assert np.allclose(gb[c], w[c].item() * gdir[c], rtol=0, atol=0)
            g_o = model.grad_log_kernel(Xq, y, b0[c].astype(np.float64), "gaussian", 10.0)
            assert np.linalg.norm(gdir[c] - g_o) / np.linalg.norm(g_o) <= tol
        coords = [(int(k), int(j)) for k, j in zip(rng.integers(0, K - 1, 12), rng.integers(0, p, 12))]
        g_o0 = model.grad_log_kernel(Xq, y, b0[0].astype(np.float64), "gaussian", 10.0)
        scale = np.abs(g_o0).max()
        for (k, j) in coords:
            fd = _fd(Xq, y, b0[0].astype(np.float64), k, j, 1e-4, "gaussian", 10.0)
            assert abs(fd - g_o0[k, j]) <= 1e-6 * max(1.0, abs(fd))          # the oracle against FD
            assert abs(gdir[0, k, j] - fd) <= tol * scale                        # the kernel against FD


def test_autograd_in_an_optimisation_step(cuda):
    """A few gradient-ascent steps on log K through the op raise log K."""
    import torch
    X, y, _, _ = synthetic.make_workload("plain_fp64", n=800, p=40)
    with hmc.create(X, y, 3, "gaussian", 10.0, x_storage="f64", state="f64") as h:
        beta = torch.zeros((1, 2, 40), dtype=torch.float64, device=cuda, requires_grad=True)
        opt = torch.optim.SGD([beta], lr=1e-3)
        vals = []
        for _ in range(5):
            opt.zero_grad()
            lp = autograd.log_posterior(beta, h)
            (-lp.sum()).backward()
            opt.step()
            vals.append(lp.item())
        assert all(b > a for a, b in zip(vals, vals[1:]))
