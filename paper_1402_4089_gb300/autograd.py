"""The log-posterior kernel (Eq. logkernel) as a differentiable PyTorch op.

``log_posterior(beta, handle)`` returns log K for every chain of the handle's
problem(s).  The forward pass is one call of ``hmc_logpost_grad``: the fused
kernel produces log K and its gradient (Eq. gradient) in the same pass over
X, so the backward pass only scales the stored gradient by the incoming
adjoint -- no second pass over X, no autodiff tape through the model.

    beta : tensor in the handle's beta layout, [chains][K-1][p] for one
           problem, or the flat concatenation over problems (batch handle);
           dtype of the handle's state (float32 or float64), on the GPU.
    returns : float64 tensor [nprob * chains] (index b * chains + c).

The gradient with respect to X is not produced (X is data).
"""
import torch


class LogPost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta, handle, chains):
        lp, g = handle.logpost_grad(beta.detach().contiguous(), chains=chains)
        ctx.save_for_backward(g)
        ctx.handle = handle
        ctx.chains = chains
        return lp

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        h, chains = ctx.handle, ctx.chains
        flat = g.reshape(-1)
        w = grad_out.to(g.dtype)
        pieces, off = [], 0
        for b, (_, p, K) in enumerate(h.shapes):
            size = chains * (K - 1) * p
            blk = flat[off:off + size].view(chains, (K - 1) * p)
            pieces.append((blk * w[b * chains:(b + 1) * chains].view(chains, 1)).reshape(-1))
            off += size
        return torch.cat(pieces).view_as(g), None, None


def log_posterior(beta, handle, chains=None):
    """log K of each chain (float64 [nprob * chains]); differentiable in beta."""
    if chains is None:
        chains = beta.numel() // handle.chain_size
    return LogPost.apply(beta, handle, int(chains))
