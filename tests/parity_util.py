"""Error measures shared by the GPU parity tests.

Gradient: both the relative 2-norm error ||g - g_ref|| / ||g_ref|| over one
chain and the element-wise error max_jk |g - g_ref| / max(max_jk |g_ref|,
1e-30), each against the same bound, so that one wrong coefficient (a padded
tail column, the last row tile, one cluster's slice) cannot hide under the
norm of the rest.  log K: |d| / max(1, |log K_ref|).
"""
import numpy as np


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def elem(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b), initial=0.0) / max(float(np.max(np.abs(b), initial=0.0)), 1e-30))


def lk_err(a, b):
    return abs(float(a) - float(b)) / max(1.0, abs(float(b)))


def grad_errs(g, g_ref):
    """(relative norm error, element-wise error) of one chain's gradient."""
    return rel(g, g_ref), elem(g, g_ref)


def assert_grad(g, g_ref, tol, what=""):
    r, e = grad_errs(g, g_ref)
    assert r <= tol and e <= tol, (what, "norm", r, "element", e, "tol", tol)
