"""Seeded synthetic workloads shaped like the paper's multinomial setting.

This module only draws inputs: the predictor matrix X, the true coefficients
and the class labels.  It holds none of the sampler's arithmetic (no
log-posterior, gradient, leapfrog or accept test) and is the one module that
both the CUDA path's tests and the FP64 oracle's tests take their inputs from.

All draws come from ``numpy.random.Generator(numpy.random.Philox(key=...))``,
which is platform independent.  Labels are drawn from the softmax model of
Sec. 2.1 by the Gumbel-max construction: y_i = argmax_k (z_ik + G_ik) with
z_i = (x_i^T beta_1, ..., x_i^T beta_{K-1}, 0) and G_ik iid standard Gumbel,
which has exactly the softmax class probabilities.

Workloads (sizes of the paper's high-dimensional setting, Sec. 3.1 / 3.2):

* ``plain_fp64``  n=1000,  p=50,    K=3 : X, beta iid N(0,1).
* ``highdim_fp32``n=10000, p=5000,  K=10: X iid N(0,1) except columns with
  j mod 5 == 4, which are 0.8 x_{j-1} + 0.6 z (unit variance, correlated with
  their left neighbour); beta sparse: each free entry nonzero with prob. 0.05,
  value N(0, 2^2).
* ``precision``   n=50000, p=10000, K=20: X, beta iid N(0,1).
* ``batched``     n=20000, p=2000,  K=10 (64 chains share it) plus 32 uneven
  problems n ~ U[500, 20000], p ~ U[100, 4000], K ~ U{3..20}.
* ``autodiff``    n=100000, p=20000, K=10: X, beta iid N(0,1).
* ``sweep``       the timing sweep of Sec. 3.1 (Table 1): X and B iid
  N(0, 1e-3) (variance 1e-3).
"""
import numpy as np

WORKLOADS = {
    "plain_fp64": dict(n=1000, p=50, K=3, chains=1, L=20, eps=0.01, iters=500,
                       prior=("gaussian", 10.0), xdtype="f64"),
    "highdim_fp32": dict(n=10000, p=5000, K=10, chains=1, L=100, eps=2e-3, iters=2000,
                         prior=("gaussian", 1.0), xdtype="f32"),
    "precision": dict(n=50000, p=10000, K=20, chains=4, L=50, eps=1e-3, iters=1000,
                      prior=("gaussian", 10.0), xdtype="bf16"),
    "batched": dict(n=20000, p=2000, K=10, chains=64, L=50, eps=1e-3, iters=200,
                    prior=("gaussian", 10.0), xdtype="bf16"),
    # Sec. 3.2's run shape: 60000 x 785 (784 pixel columns + intercept), K = 10,
    # L = 100, annealed burn-in of 100 iterations (T0 = 1e3, r = 0.9) at eps = 1e-4,
    # then 100 sampling iterations at eps = 7e-5, Cauchy(0, 1) prior.
    "mnist_shaped": dict(n=60000, p=785, K=10, chains=1, L=100, eps=1e-4, eps_sample=7e-5, iters=200,
                         burn_in=100, t0=1.0e3, r=0.9, prior=("cauchy", 1.0), xdtype="f32"),
    "autodiff": dict(n=100000, p=20000, K=10, chains=8, L=100, eps=1e-3, iters=500,
                     prior=("gaussian", 10.0), xdtype="bf16"),
}

_TAG_X = 1
_TAG_BETA = 2
_TAG_LABEL = 3
_TAG_SHAPES = 4


def _gen(seed, tag, sub=0):
    return np.random.Generator(np.random.Philox(key=[int(seed), (int(tag) << 32) | int(sub)]))


def draw_X(n, p, seed=0, dtype=np.float32, correlated=False, sd=1.0, sub=0):
    """n x p predictors, iid N(0, sd^2); with ``correlated`` every column with
    j mod 5 == 4 becomes 0.8 x_{j-1} + 0.6 z."""
    g = _gen(seed, _TAG_X, sub)
    X = g.standard_normal((n, p), dtype=np.float32 if dtype != np.float64 else np.float64)
    if correlated and p >= 5:
        cols = np.arange(4, p, 5)
        z = g.standard_normal((n, cols.size), dtype=X.dtype)
        X[:, cols] = X.dtype.type(0.8) * X[:, cols - 1] + X.dtype.type(0.6) * z
    if sd != 1.0:
        X *= X.dtype.type(sd)
    return X.astype(dtype, copy=False)


def draw_pixels(n, seed=0, npix=784, density=0.19, sub=0):
    """n x (1 + npix) FP32: an intercept column of ones, then pixel-like columns
    that are 0 except, with probability ``density``, a grey level k / 255 with k
    uniform on 1..255 (a synthetic stand-in with the shape and value range of
    the handwritten-digit design of Sec. 3.2; no image data is involved)."""
    g = _gen(seed, _TAG_X, sub)
    X = np.zeros((n, 1 + npix), dtype=np.float32)
    X[:, 0] = 1.0
    on = g.random((n, npix)) < density
    X[:, 1:] = np.where(on, g.integers(1, 256, size=(n, npix)).astype(np.float32) / np.float32(255.0), 0.0)
    return X


def draw_beta(p, K, seed=0, sparse=0.0, scale=1.0, sub=0):
    """True free coefficients, shape (K-1, p), FP64.  ``sparse`` > 0 keeps each
    entry with that probability (others exactly 0)."""
    g = _gen(seed, _TAG_BETA, sub)
    b = scale * g.standard_normal((K - 1, p))
    if sparse > 0.0:
        b = np.where(g.random((K - 1, p)) < sparse, b, 0.0)
    return b


def draw_labels(X, beta, seed=0, sub=0, chunk=8192):
    """Labels from the softmax model by Gumbel-max (see module docstring)."""
    g = _gen(seed, _TAG_LABEL, sub)
    n = X.shape[0]
    K = beta.shape[0] + 1
    y = np.empty(n, dtype=np.int32)
    bt = np.asarray(beta, dtype=np.float64).T
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        z = np.zeros((e - s, K))
        z[:, :-1] = np.asarray(X[s:e], dtype=np.float64) @ bt
        u = g.random((e - s, K))
        gumbel = -np.log(-np.log(np.clip(u, 1e-300, 1.0)))
        y[s:e] = np.argmax(z + gumbel, axis=1).astype(np.int32)
    return y


def make_problem(n, p, K, seed=0, dtype=np.float32, correlated=False, sparse=0.0,
                 beta_scale=1.0, x_sd=1.0, sub=0):
    """(X, y, beta_true) of one regression problem."""
    X = draw_X(n, p, seed=seed, dtype=dtype, correlated=correlated, sd=x_sd, sub=sub)
    beta = draw_beta(p, K, seed=seed, sparse=sparse, scale=beta_scale, sub=sub)
    y = draw_labels(X, beta, seed=seed, sub=sub) if n > 0 else np.zeros(0, np.int32)
    return X, y, beta


def make_workload(name, seed=0, n=None, p=None):
    """(X, y, beta_true, spec) of a named workload; n / p may be overridden to get
    a reduced-size variant of the same recipe."""
    spec = dict(WORKLOADS[name])
    if n is not None:
        spec["n"] = n
    if p is not None:
        spec["p"] = p
    nn, pp, K = spec["n"], spec["p"], spec["K"]
    if name == "plain_fp64":
        X, y, b = make_problem(nn, pp, K, seed=seed, dtype=np.float64)
    elif name == "highdim_fp32":
        X, y, b = make_problem(nn, pp, K, seed=seed, correlated=True, sparse=0.05, beta_scale=2.0)
    elif name == "mnist_shaped":
        X = draw_pixels(nn, seed=seed, npix=pp - 1)
        b = draw_beta(pp, K, seed=seed, scale=0.3)
        y = draw_labels(X, b, seed=seed)
    else:
        X, y, b = make_problem(nn, pp, K, seed=seed)
    return X, y, b, spec


def batched_shapes(count=32, seed=0):
    """Shapes (n, p, K) of the uneven problems: n ~ U[500, 20000], p ~ U[100, 4000],
    K ~ U{3..20} (integers, inclusive)."""
    g = _gen(seed, _TAG_SHAPES)
    n = g.integers(500, 20000, size=count, endpoint=True)
    p = g.integers(100, 4000, size=count, endpoint=True)
    K = g.integers(3, 20, size=count, endpoint=True)
    return [(int(a), int(b), int(c)) for a, b, c in zip(n, p, K)]


def sweep_problem(n, p, K, seed=0):
    """One problem of the timing sweep of Sec. 3.1: X and B iid N(0, 1e-3), the
    1e-3 read as the variance; y drawn from the softmax model."""
    sd = float(np.sqrt(1e-3))
    return make_problem(n, p, K, seed=seed, x_sd=sd, beta_scale=sd)


def sweep_shapes():
    """(n, p, K) of the timing sweep of Sec. 3.1 (Table 1); the repeated N value
    printed there is read as 10000 (4 x 7 x 8 = 224 combinations)."""
    Ns = [100, 1000, 5000, 10000]
    Ks = [2, 3, 4, 5, 10, 15, 20]
    ps = [10, 50, 100, 500, 1000, 5000, 10000, 20000]
    return [(nn, pp, kk) for nn in Ns for kk in Ks for pp in ps]
