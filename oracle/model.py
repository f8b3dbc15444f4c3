"""Log-posterior kernel of Bayesian multinomial regression and its gradient.

Test infrastructure only (see ``oracle/__init__.py``).  FP64 throughout.

Notation of Sec. 2.1: X is n x p, labels y_i in {0..K-1} stand for the
one-hot rows of Y (classes are mutually exclusive), B = [beta_1..beta_K] is
p x K with beta_K = 0 for identifiability.  Only the p x (K-1) free block is
a parameter; it is passed as ``beta`` with shape (K-1, p) (class-major, the
layout the sampler uses), or (chains, K-1, p).

The Appendix describes two other ways to hold the coefficients, both with all
K class rows stored (shape (K, p)):
* "masked": beta_K is set to 0, the full p x K gradient of Eq. fullgrad is
  formed and multiplied elementwise by the mask M (M_jk = 1 for k != K, else
  0), which zeroes the gradient of beta_K;
* "unconstrained": identifiability is not enforced ("if the task is only
  prediction"); all K rows are free, the softmax runs over K free logits and
  the prior covers every coefficient (the setting timed in Figs 3-4).
The default layout, "free", is the p x (K-1) block above.

Priors (no normalising constants anywhere, Sec. 1.1):
* "cauchy", scale s (the paper uses the standard Cauchy, s = 1, Eq. logkernel):
  log prior = -log(1 + b^2/s^2), derivative -2b/(s^2 + b^2)
  (the paper's Appendix prints the opposite sign; the derivative is used).
* "gaussian", scale sigma (the benchmark workloads): -b^2/(2 sigma^2),
  derivative -b/sigma^2.
"""
import numpy as np

PRIORS = ("gaussian", "cauchy")


def prior_terms(beta, kind, scale):
    """Elementwise log-prior kernel of the free coefficients (Gamma of Eq. logkernelGPU)."""
    b = np.asarray(beta, dtype=np.float64)
    s = float(scale)
    if kind == "cauchy":
        return -np.log1p((b / s) ** 2)
    if kind == "gaussian":
        return -(b * b) / (2.0 * s * s)
    raise ValueError(f"unknown prior {kind!r}")


def prior_grad(beta, kind, scale):
    """Elementwise derivative of ``prior_terms`` (Gamma of Eq. fullgrad, sign per calculus)."""
    b = np.asarray(beta, dtype=np.float64)
    s = float(scale)
    if kind == "cauchy":
        return -2.0 * b / (s * s + b * b)
    if kind == "gaussian":
        return -b / (s * s)
    raise ValueError(f"unknown prior {kind!r}")


def full_logits(X, beta):
    """Z = X B with the fixed zero column of class K appended (n x K), Eq. softmax."""
    X = np.asarray(X, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    n = X.shape[0]
    Z = np.zeros((n, beta.shape[0] + 1))
    Z[:, :-1] = X @ beta.T
    return Z


def softmax(Z):
    """Row-wise generalised logit psi (Eq. softmax).  The row maximum is subtracted
    before exponentiating, which leaves every ratio unchanged."""
    Z = np.asarray(Z, dtype=np.float64)
    m = Z.max(axis=1, keepdims=True)
    E = np.exp(Z - m)
    return E / E.sum(axis=1, keepdims=True)


def log_softmax(Z):
    """log psi, computed as z - logsumexp(z) row by row."""
    Z = np.asarray(Z, dtype=np.float64)
    m = Z.max(axis=1, keepdims=True)
    lse = m + np.log(np.exp(Z - m).sum(axis=1, keepdims=True))
    return Z - lse


def log_likelihood_of_logits(Z, y):
    """sum_i log psi_{i, y_i} for given n x K logits (Eq. loglike with one-hot Y)."""
    y = np.asarray(y, dtype=np.int64)
    n = y.shape[0]
    if n == 0:
        return 0.0
    LP = log_softmax(Z)
    return float(LP[np.arange(n), y].sum())


def log_likelihood(X, y, beta):
    """l(B | X, Y) = sum_i sum_k y_ik log psi_ik (Eq. loglike); one-hot Y picks
    log psi_{i, y_i}."""
    y = np.asarray(y, dtype=np.int64)
    if y.shape[0] == 0:
        return 0.0
    return log_likelihood_of_logits(full_logits(X, beta), y)


def log_kernel(X, y, beta, kind, scale):
    """log K(B | X, Y) = log-likelihood + sum of prior terms over the free block
    (Eq. logkernel with beta_K = 0)."""
    return log_likelihood(X, y, beta) + float(prior_terms(beta, kind, scale).sum())


def residual(X, y, beta):
    """R = Y - psi(XB) restricted to the K-1 free classes (n x (K-1))."""
    y = np.asarray(y, dtype=np.int64)
    n = y.shape[0]
    P = softmax(full_logits(X, beta))
    Y = np.zeros_like(P)
    Y[np.arange(n), y] = 1.0
    return (Y - P)[:, :-1]


def grad_log_kernel(X, y, beta, kind, scale):
    """d log K / d B on the free block: X^T (Y - psi(XB)) + Gamma (Eq. gradient /
    fullgrad), returned in the (K-1, p) layout of ``beta``."""
    X = np.asarray(X, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    g = prior_grad(beta, kind, scale)
    if X.shape[0] > 0:
        g = g + (X.T @ residual(X, y, beta)).T
    return g


def log_kernel_and_grad(X, y, beta, kind, scale):
    """Both quantities at one coefficient state."""
    return log_kernel(X, y, beta, kind, scale), grad_log_kernel(X, y, beta, kind, scale)


def log_kernel_and_grad_by_rows(row_blocks, betas, kind, scale):
    """log K and its gradient for several coefficient states of one problem whose
    X is too large to hold in FP64 at once.  The likelihood and its gradient are
    sums over rows (Eqs. loglike, gradient), so ``row_blocks`` yields (X_b, y_b)
    blocks of consecutive rows, each added in order; the prior term is added
    once.  Returns (logk[c], grad[c], Z[c]) with Z the n x K logits (zero column
    of class K included) of every state."""
    betas = [np.asarray(b, dtype=np.float64) for b in betas]
    ll = [0.0] * len(betas)
    g = [np.zeros_like(b) for b in betas]
    Z = [[] for _ in betas]
    for Xb, yb in row_blocks:
        Xb = np.asarray(Xb, dtype=np.float64)
        yb = np.asarray(yb, dtype=np.int64)
        for c, b in enumerate(betas):
            Zb = full_logits(Xb, b)
            ll[c] += log_likelihood_of_logits(Zb, yb)
            P = softmax(Zb)
            Y = np.zeros_like(P)
            Y[np.arange(yb.shape[0]), yb] = 1.0
            g[c] += (Xb.T @ (Y - P)[:, :-1]).T
            Z[c].append(Zb)
    logk = [ll[c] + float(prior_terms(b, kind, scale).sum()) for c, b in enumerate(betas)]
    grad = [g[c] + prior_grad(b, kind, scale) for c, b in enumerate(betas)]
    return logk, grad, [np.concatenate(z) if z else np.zeros((0, b.shape[0] + 1)) for z, b in zip(Z, betas)]


# ---------------------------------------------------------------- K-row layouts
LAYOUTS = ("free", "masked", "unconstrained")


def all_logits(X, B):
    """Z = X B over all K class rows of B (shape (K, p)), no fixed column (n x K)."""
    X = np.asarray(X, dtype=np.float64)
    return X @ np.asarray(B, dtype=np.float64).T


def full_gradient(X, y, B, kind, scale):
    """The p x K gradient of Eq. fullgrad for all K class rows of B, returned in the
    (K, p) layout: X^T (Y - psi(X B)) + Gamma, the softmax over the K logits of B."""
    X = np.asarray(X, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    g = prior_grad(B, kind, scale)
    n = X.shape[0]
    if n > 0:
        y = np.asarray(y, dtype=np.int64)
        P = softmax(all_logits(X, B))
        Y = np.zeros_like(P)
        Y[np.arange(n), y] = 1.0
        g = g + (X.T @ (Y - P)).T
    return g


def unconstrained_log_likelihood(X, y, B):
    """Eq. loglike with all K rows of B free (no beta_K = 0)."""
    y = np.asarray(y, dtype=np.int64)
    n = y.shape[0]
    if n == 0:
        return 0.0
    LP = log_softmax(all_logits(X, B))
    return float(LP[np.arange(n), y].sum())


def mask_matrix(K, p):
    """The mask M of the Appendix in the (K, p) layout: 1 except on the row of class K."""
    M = np.ones((K, p))
    M[-1] = 0.0
    return M


def log_kernel_layout(X, y, B, kind, scale, layout):
    """log K for coefficients held in ``layout`` (see the module docstring)."""
    B = np.asarray(B, dtype=np.float64)
    if layout == "free":
        return log_kernel(X, y, B, kind, scale)
    if layout == "masked":
        Bm = B.copy()
        Bm[-1] = 0.0                               # beta_K = 0 first
        return unconstrained_log_likelihood(X, y, Bm) + float(prior_terms(Bm, kind, scale).sum())
    if layout == "unconstrained":
        return unconstrained_log_likelihood(X, y, B) + float(prior_terms(B, kind, scale).sum())
    raise ValueError(f"unknown layout {layout!r}")


def grad_log_kernel_layout(X, y, B, kind, scale, layout):
    """Gradient of log K for coefficients held in ``layout``: "masked" follows the
    Appendix (beta_K = 0, full gradient of Eq. fullgrad, times M)."""
    B = np.asarray(B, dtype=np.float64)
    if layout == "free":
        return grad_log_kernel(X, y, B, kind, scale)
    if layout == "masked":
        Bm = B.copy()
        Bm[-1] = 0.0
        return full_gradient(X, y, Bm, kind, scale) * mask_matrix(B.shape[0], B.shape[1])
    if layout == "unconstrained":
        return full_gradient(X, y, B, kind, scale)
    raise ValueError(f"unknown layout {layout!r}")
