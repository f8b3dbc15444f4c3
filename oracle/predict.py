"""Posterior predictive class probabilities (Sec. 3.2).

Test infrastructure only (see ``oracle/__init__.py``).  FP64 throughout.

The paper predicts, for each new observation, the class with the highest
average softmax value over the posterior samples.  For draws B_1..B_D (each in
one of the coefficient layouts of ``model``) and a row x_i:

    prob_ik = (1/D) sum_d psi_k(x_i B_d)          (Eq. softmax, all K classes)
    class_i = argmax_k prob_ik                    (the first, i.e. lowest, k on a tie)
"""
import numpy as np

from . import model


def draw_logits(X, draw, layout):
    """n x K logits of one draw: the free rows, plus the zero column of class K
    in the identifiable layouts ("free": (K-1, p); "masked": (K, p) with row K
    read as 0; "unconstrained": (K, p), all free)."""
    B = np.asarray(draw, dtype=np.float64)
    if layout == "free":
        return model.full_logits(X, B)
    if layout == "masked":
        return model.full_logits(X, B[:-1])
    if layout == "unconstrained":
        return model.all_logits(X, B)
    raise ValueError(f"unknown layout {layout!r}")


def predictive(X, draws, layout="free"):
    """(prob, cls): the mean softmax over the draws (shape (D, R, p)) for every
    row of X, and its argmax."""
    X = np.asarray(X, dtype=np.float64)
    draws = np.asarray(draws, dtype=np.float64)
    acc = None
    for d in range(draws.shape[0]):
        P = model.softmax(draw_logits(X, draws[d], layout))
        acc = P if acc is None else acc + P
    prob = acc / draws.shape[0]
    return prob, np.argmax(prob, axis=1).astype(np.int32)
