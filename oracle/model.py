"""Log-posterior kernel of Bayesian multinomial regression and its gradient.

Test infrastructure only (see ``oracle/__init__.py``).  FP64 throughout.

Notation of Sec. 2.1: X is n x p, labels y_i in {0..K-1} stand for the
one-hot rows of Y (classes are mutually exclusive), B = [beta_1..beta_K] is
p x K with beta_K = 0 for identifiability.  Only the p x (K-1) free block is
a parameter; it is passed as ``beta`` with shape (K-1, p) (class-major, the
layout the sampler uses), or (chains, K-1, p).

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


def log_likelihood(X, y, beta):
    """l(B | X, Y) = sum_i sum_k y_ik log psi_ik (Eq. loglike); one-hot Y picks
    log psi_{i, y_i}."""
    y = np.asarray(y, dtype=np.int64)
    n = y.shape[0]
    if n == 0:
        return 0.0
    LP = log_softmax(full_logits(X, beta))
    return float(LP[np.arange(n), y].sum())


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
