"""Pins of the oracle's K-row coefficient layouts (Appendix: the mask M after
Eq. fullgrad, and the variant that does not enforce identifiability).

Each checks the oracle against something other than itself: the free p x (K-1)
block (pinned in test_oracle_pins.py), central finite differences, brute
force with explicit loops and no log-sum-exp shift, and the invariants the
mathematics fixes (softmax shift invariance, class sums of Y - psi).  Two
planted mistakes show that the pins decide what they claim to.
"""
import math

import numpy as np
import pytest

from oracle import hmc, model


def _data(n=31, p=5, K=4, seed=11, bscale=0.6):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    y = rng.integers(0, K, size=n)
    B = bscale * rng.standard_normal((K, p))
    return X, y, B


# --- masked layout: the mask M reproduces the free block -----------------------

@pytest.mark.parametrize("kind,scale", [("gaussian", 2.0), ("cauchy", 1.0)])
def test_masked_equals_free_block_with_zero_row(kind, scale):
    X, y, B = _data()
    B[-1] = 3.7                       # whatever row K holds is masked away
    g = model.grad_log_kernel_layout(X, y, B, kind, scale, "masked")
    g_free = model.grad_log_kernel(X, y, B[:-1], kind, scale)
    assert np.allclose(g[:-1], g_free, rtol=1e-13, atol=1e-13)
    assert np.all(g[-1] == 0.0)
    lk = model.log_kernel_layout(X, y, B, kind, scale, "masked")
    assert abs(lk - model.log_kernel(X, y, B[:-1], kind, scale)) <= 1e-12 * max(1.0, abs(lk))


def test_mask_matrix_is_the_appendix_mask():
    M = model.mask_matrix(5, 3)
    assert M.shape == (5, 3)
    assert np.all(M[:-1] == 1.0) and np.all(M[-1] == 0.0)


def test_planted_unmasked_gradient_fails_the_masked_pin():
    X, y, B = _data()
    B[-1] = 0.0
    wrong = model.full_gradient(X, y, B, "gaussian", 2.0)        # the mask step dropped
    assert np.abs(wrong[-1]).max() > 1e-3                       # row K is not zero


# --- unconstrained layout --------------------------------------------------------

@pytest.mark.parametrize("kind,scale", [("gaussian", 10.0), ("gaussian", 1.0), ("cauchy", 1.0), ("cauchy", 2.5)])
def test_unconstrained_fd_gradient_every_coordinate(kind, scale):
    X, y, B = _data(n=60, p=7, K=3)
    g = model.grad_log_kernel_layout(X, y, B, kind, scale, "unconstrained")
    h = 1e-4
    fd = np.empty_like(B)
    for k in range(B.shape[0]):
        for j in range(B.shape[1]):
            bp = B.copy(); bp[k, j] += h
            bm = B.copy(); bm[k, j] -= h
            fd[k, j] = (model.log_kernel_layout(X, y, bp, kind, scale, "unconstrained")
                        - model.log_kernel_layout(X, y, bm, kind, scale, "unconstrained")) / (2 * h)
    assert np.linalg.norm(g - fd) / np.linalg.norm(fd) < 1e-6


def test_unconstrained_likelihood_brute_force():
    X, y, B = _data(n=23, p=4, K=5)
    Y = np.zeros((23, 5))
    Y[np.arange(23), y] = 1.0
    ll = 0.0
    for i in range(23):
        z = [sum(X[i, j] * B[k, j] for j in range(4)) for k in range(5)]
        den = sum(math.exp(zk) for zk in z)
        for k in range(5):
            ll += Y[i, k] * math.log(math.exp(z[k]) / den)
    assert abs(model.unconstrained_log_likelihood(X, y, B) - ll) < 1e-11


def test_unconstrained_likelihood_is_shift_invariant():
    # Adding the same vector c to every class row adds x_i.c to every logit of
    # row i, which the softmax cancels: the coefficients are not identifiable.
    X, y, B = _data(n=40, p=6, K=4)
    c = np.random.default_rng(5).standard_normal(6)
    a = model.unconstrained_log_likelihood(X, y, B)
    b = model.unconstrained_log_likelihood(X, y, B + c[None, :])
    assert abs(a - b) <= 1e-11 * max(1.0, abs(a))


def test_unconstrained_likelihood_gradient_sums_to_zero_over_classes():
    X, y, B = _data(n=50, p=6, K=4)
    g = model.grad_log_kernel_layout(X, y, B, "gaussian", 3.0, "unconstrained")
    lik = g - model.prior_grad(B, "gaussian", 3.0)
    assert np.abs(lik.sum(axis=0)).max() < 1e-11                 # sum_k (y_ik - psi_ik) = 0


def test_unconstrained_with_zero_last_row_is_the_free_model():
    X, y, B = _data()
    B[-1] = 0.0
    lk = model.log_kernel_layout(X, y, B, "cauchy", 1.0, "unconstrained")
    assert abs(lk - model.log_kernel(X, y, B[:-1], "cauchy", 1.0)) < 1e-12 * max(1.0, abs(lk))
    g = model.grad_log_kernel_layout(X, y, B, "cauchy", 1.0, "unconstrained")
    assert np.allclose(g[:-1], model.grad_log_kernel(X, y, B[:-1], "cauchy", 1.0), rtol=1e-13, atol=1e-13)


def test_planted_zero_logit_fails_shift_invariance():
    # Keeping the implied zero logit of class K (the free model's softmax) in
    # the unconstrained likelihood breaks the shift invariance above.
    X, y, B = _data(n=40, p=6, K=4)
    c = np.random.default_rng(6).standard_normal(6)

    def wrong(Bx):
        Z = np.hstack([X @ Bx.T, np.zeros((40, 1))])             # K free logits plus a zero one
        return float(model.log_softmax(Z)[np.arange(40), y].sum())

    assert abs(wrong(B) - wrong(B + c[None, :])) > 1e-3


# --- the sampler in the K-row layouts ---------------------------------------------

def test_masked_chains_equal_free_chains():
    X, y, B = _data(n=80, p=5, K=3, bscale=0.0)
    free = hmc.sample(X, y, 3, "gaussian", 5.0, 2, 5, 0.05, 4, 17)
    masked = hmc.sample(X, y, 3, "gaussian", 5.0, 2, 5, 0.05, 4, 17, layout="masked")
    assert masked["samples"].shape == (4, 2, 3, 5)
    assert np.array_equal(masked["samples"][:, :, :-1], free["samples"])
    assert np.all(masked["samples"][:, :, -1] == 0.0)
    assert np.array_equal(masked["accept"], free["accept"])


def test_unconstrained_leapfrog_reverses():
    X, y, B = _data(n=70, p=4, K=3)
    eta = np.random.default_rng(9).standard_normal(B.shape)
    b1, e1, _, _ = hmc.leapfrog(X, y, B, eta, 0.01, 15, "gaussian", 10.0, layout="unconstrained")
    b2, e2, _, _ = hmc.leapfrog(X, y, b1, -e1, 0.01, 15, "gaussian", 10.0, layout="unconstrained")
    assert np.abs(b2 - B).max() <= 1e-12 * max(1.0, np.abs(B).max())
    assert np.abs(-e2 - eta).max() <= 1e-12 * max(1.0, np.abs(eta).max())
