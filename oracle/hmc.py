"""Leapfrog integrator and HMC sampler, straight from Sec. 1.1 and Sec. 3.2.

Test infrastructure only (see ``oracle/__init__.py``).  FP64 throughout.

One leapfrog update (Eqs. hmc1-hmc3): a half step of eps/2 for the momentum
along grad log K, a full step of eps for the coefficients, a second half step
for the momentum at the new coefficients.  One proposal applies it L times
(Sec. 1.1: L gradient evaluations per proposal, then one log-kernel
evaluation for the accept test).  The gradient at the end of one update is
the gradient at the start of the next, so it is computed once and reused:
the values are identical to recomputing it.

Metropolis test with momentum (Eq. accept, with the kinetic energy read as
eta.eta / 2 for eta ~ N(0, I) and unit-mass dynamics):
    H = -log K(beta) + eta.eta / 2,   accept  iff  log u < (H0 - H1) / T
with T = 1 while sampling and T = T_t during annealed burn-in (Sec. 3.2:
accept with probability alpha^(1/T_t), T_t = max(1, r T_{t-1})).
A proposal whose H1 is not finite is rejected and counted as divergent.
The accept test is strict; u comes from ``philox.accept_uniform`` and is
never 0.
"""
import numpy as np

from . import model, philox


def leapfrog(X, y, beta, eta, eps, L, kind, scale, grad0=None, layout="free"):
    """Apply L leapfrog updates (Eqs. hmc1-hmc3) to (beta, eta).

    beta, eta: arrays of shape (K-1, p), or (K, p) for the "masked" and
    "unconstrained" layouts of ``model``.  Returns (beta', eta', log K(beta'),
    grad log K(beta')).
    """
    beta = np.array(beta, dtype=np.float64, copy=True)
    eta = np.array(eta, dtype=np.float64, copy=True)

    def grad(b):
        return model.grad_log_kernel_layout(X, y, b, kind, scale, layout)

    g = grad(beta) if grad0 is None else np.array(grad0, dtype=np.float64)
    for _ in range(L):
        eta = eta + (eps / 2.0) * g          # Eq. hmc1
        beta = beta + eps * eta              # theta update between hmc1 and hmc3
        g = grad(beta)
        eta = eta + (eps / 2.0) * g          # Eq. hmc3
    return beta, eta, model.log_kernel_layout(X, y, beta, kind, scale, layout), g


def hamiltonian(logk, eta):
    """H = -log K + eta.eta / 2 (Eq. accept, kinetic energy with the factor 1/2)."""
    eta = np.asarray(eta, dtype=np.float64)
    return -float(logk) + 0.5 * float(np.sum(eta * eta))


def annealing_temperatures(burn_in, t0=1.0e3, r=0.9):
    """T_t = max(1, r T_{t-1}) for burn-in iterations t = 1..burn_in, T_0 = t0 (Sec. 3.2)."""
    temps = np.empty(burn_in)
    t = float(t0)
    for i in range(burn_in):
        t = max(1.0, r * t)
        temps[i] = t
    return temps


def sample(X, y, K, kind, scale, chains, L, eps, iters, seed,
           beta0=None, iter0=0, temps=None, chain0=0, layout="free"):
    """Run `chains` independent HMC chains for `iters` iterations.

    eps   : scalar or per-iteration array of step sizes.
    beta0 : (chains, R, p) start, zeros if None (R = K-1, or K for the
            "masked" and "unconstrained" layouts).
    iter0 : RNG iteration index of the first iteration (counter word 1).
    temps : per-iteration acceptance temperatures (None -> all 1).
    chain0: RNG chain word of chain 0 (counter word 2 is chain0 + c).

    The momentum is drawn for the free coefficients only: (K-1) p normals,
    with the row of beta_K held at 0 in the masked layout (the Appendix sets
    its momentum to 0), and K p normals in the unconstrained layout.

    Returns a dict with samples (iters, chains, R, p), accept (iters, chains),
    dH = H1 - H0, logk (log K of the state kept), diverged, and the final
    state (beta, grad, logk).
    """
    X = np.asarray(X, dtype=np.float64)
    p = X.shape[1]
    km1 = K - 1 if layout == "free" else K
    nfree = K * p if layout == "unconstrained" else (K - 1) * p
    eps_t = np.broadcast_to(np.asarray(eps, dtype=np.float64), (iters,))
    temp_t = np.ones(iters) if temps is None else np.asarray(temps, dtype=np.float64)
    if beta0 is None:
        beta = np.zeros((chains, km1, p))
    else:
        beta = np.array(beta0, dtype=np.float64).reshape(chains, km1, p).copy()
    if layout == "masked":
        beta[:, -1] = 0.0
    logk = np.array([model.log_kernel_layout(X, y, beta[c], kind, scale, layout) for c in range(chains)])
    grad = np.stack([model.grad_log_kernel_layout(X, y, beta[c], kind, scale, layout) for c in range(chains)])

    out_samples = np.empty((iters, chains, km1, p))
    out_acc = np.zeros((iters, chains), dtype=bool)
    out_dh = np.empty((iters, chains))
    out_logk = np.empty((iters, chains))
    out_div = np.zeros((iters, chains), dtype=bool)
    for t in range(iters):
        it = iter0 + t
        for c in range(chains):
            eta0 = np.zeros((km1, p))
            eta0.reshape(-1)[:nfree] = philox.momentum_normals(seed, it, chain0 + c, nfree)
            h0 = hamiltonian(logk[c], eta0)
            b1, e1, lk1, g1 = leapfrog(X, y, beta[c], eta0, eps_t[t], L, kind, scale, grad0=grad[c], layout=layout)
            h1 = hamiltonian(lk1, e1)
            u = philox.accept_uniform(seed, it, chain0 + c)
            finite = np.isfinite(h1)
            acc = bool(finite and np.log(u) < (h0 - h1) / temp_t[t])
            out_div[t, c] = not finite
            out_dh[t, c] = h1 - h0
            if acc:
                beta[c], grad[c], logk[c] = b1, g1, lk1
            out_acc[t, c] = acc
            out_samples[t, c] = beta[c]
            out_logk[t, c] = logk[c]
    return dict(samples=out_samples, accept=out_acc, dH=out_dh, logk=out_logk,
                diverged=out_div, beta=beta, grad=grad, logk_final=logk)
