"""Pins of the oracle's posterior predictive (Sec. 3.2: the class with the
highest average softmax value over the posterior samples) against closed
forms, a textbook special case and brute force."""
import math

import numpy as np
import scipy.special

from oracle import predict


def test_zero_draws_give_uniform_probabilities_and_the_lowest_class():
    X = np.random.default_rng(0).standard_normal((7, 3))
    prob, cls = predict.predictive(X, np.zeros((4, 4, 3)))          # free layout, K = 5
    assert np.allclose(prob, 0.2, rtol=0, atol=1e-15)
    assert np.all(cls == 0)                                          # a tie keeps the lowest class


def test_two_classes_single_draw_is_the_logistic_function():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((20, 4))
    b = rng.standard_normal((1, 1, 4))
    prob, cls = predict.predictive(X, b)
    z = X @ b[0, 0]
    assert np.allclose(prob[:, 0], scipy.special.expit(z), rtol=1e-13, atol=1e-15)
    assert np.array_equal(cls, np.where(z > 0, 0, 1))


def test_mean_over_draws_by_brute_force():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((5, 3))
    D = rng.standard_normal((3, 2, 3))                               # 3 draws, K = 3 (free layout)
    prob, cls = predict.predictive(X, D)
    for i in range(5):
        want = [0.0, 0.0, 0.0]
        for d in range(3):
            z = [sum(X[i, j] * D[d, k, j] for j in range(3)) for k in range(2)] + [0.0]
            den = sum(math.exp(v) for v in z)
            for k in range(3):
                want[k] += math.exp(z[k]) / den / 3.0
        assert np.allclose(prob[i], want, rtol=1e-12, atol=1e-15)
        assert cls[i] == int(np.argmax(want))


def test_layouts_agree_and_rows_sum_to_one():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((9, 4))
    D = rng.standard_normal((2, 3, 4))
    pf, cf = predict.predictive(X, D)
    Dm = np.concatenate([D, rng.standard_normal((2, 1, 4))], axis=1)   # row K of a masked draw is ignored
    pm, cm = predict.predictive(X, Dm, "masked")
    Du = np.concatenate([D, np.zeros((2, 1, 4))], axis=1)             # unconstrained with beta_K = 0
    pu, cu = predict.predictive(X, Du, "unconstrained")
    assert np.allclose(pf, pm, rtol=1e-14) and np.allclose(pf, pu, rtol=1e-14)
    assert np.array_equal(cf, cm) and np.array_equal(cf, cu)
    assert np.allclose(pf.sum(axis=1), 1.0, atol=1e-14)


def test_unconstrained_class_permutation_permutes_probabilities():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((6, 3))
    D = rng.standard_normal((2, 4, 3))
    perm = np.array([2, 0, 3, 1])
    p0, _ = predict.predictive(X, D, "unconstrained")
    p1, _ = predict.predictive(X, D[:, perm], "unconstrained")
    assert np.allclose(p1, p0[:, perm], rtol=1e-14)
