"""Posterior predictive (hmc_predict) against the oracle: the mean softmax over
posterior draws and its argmax (Sec. 3.2).  FP64 state: probabilities to
1e-12, classes identical.  FP32 state: probabilities to 1e-5 absolute; the
classes are identical wherever the oracle's top two probabilities differ by
more than 1e-4, and elsewhere the GPU's class is one of the near-tied ones."""
import numpy as np
import pytest

from oracle import predict as opredict
from paper_1402_4089_gb300 import hmc, synthetic

pytestmark = pytest.mark.gpu


def _check_classes(prob_o, cls, gap_tol):
    srt = np.sort(prob_o, axis=1)
    clear = (srt[:, -1] - srt[:, -2]) > gap_tol
    assert np.array_equal(cls[clear], np.argmax(prob_o, axis=1)[clear])
    near = prob_o[np.arange(len(cls)), cls] >= srt[:, -1] - gap_tol
    assert np.all(near)


@pytest.mark.parametrize("layout", ["free", "masked", "unconstrained"])
@pytest.mark.parametrize("state", ["f64", "f32"])
def test_predict_matches_oracle(cuda, layout, state):
    import torch
    n, p, K = 700, 45, 4
    dt = np.float64 if state == "f64" else np.float32
    X, y, _ = synthetic.make_problem(n, p, K, seed=61, dtype=dt)
    Xnew, _, _ = synthetic.make_problem(333, p, K, seed=62, dtype=dt)
    rows = K - 1 if layout == "free" else K
    draws = (0.4 * np.random.default_rng(63).standard_normal((37, rows, p))).astype(dt)
    with hmc.create(X, y, K, "gaussian", 2.0, x_storage=state, state=state, layout=layout) as h:
        prob, cls = h.predict(torch.from_numpy(draws).to(cuda), torch.from_numpy(Xnew).to(cuda))
        prob_h, cls_h = h.predict(draws, Xnew)              # host buffers
        prob, cls = prob.cpu().numpy(), cls.cpu().numpy()
        assert np.array_equal(prob, prob_h) and np.array_equal(cls, cls_h)
    prob_o, cls_o = opredict.predictive(Xnew, draws, layout)
    if state == "f64":
        assert np.max(np.abs(prob - prob_o)) <= 1e-12
        assert np.array_equal(cls, cls_o)
    else:
        assert np.max(np.abs(prob - prob_o)) <= 1e-5
        _check_classes(prob_o, cls, 1e-4)
    assert np.allclose(prob.sum(axis=1), 1.0, atol=1e-5)


def test_predict_edge_cases(cuda):
    X, y, _ = synthetic.make_problem(50, 6, 2, seed=64)
    with hmc.create(X, y, 2, "gaussian", 2.0) as h:
        zero = np.zeros((3, 1, 6), np.float32)
        prob, cls = h.predict(zero, X)                        # every draw 0: a tie, the lowest class
        assert np.all(prob == 0.5) and np.all(cls == 0)
        prob, cls = h.predict(zero, X[:0])                     # no rows
        assert prob.shape == (0, 2) and cls.shape == (0,)
        with pytest.raises(ValueError):
            h.predict(np.zeros(7, np.float32), X)              # not whole draws


def test_predict_after_sampling_classifies_held_out_rows(cuda):
    """Draws from hmc_sample on a separable synthetic problem predict held-out
    rows well: the sampling path and the predictive compose."""
    import torch
    n, p, K = 3000, 20, 3
    X, y, btrue = synthetic.make_problem(n, p, K, seed=65, beta_scale=2.0)
    Xh = synthetic.draw_X(1000, p, seed=65, sub=1)
    yh = synthetic.draw_labels(Xh, btrue, seed=65, sub=1)
    with hmc.create(X, y, K, "gaussian", 10.0, max_chains=2) as h:
        s = torch.empty((40, 2, K - 1, p), dtype=torch.float32, device=cuda)
        h.sample(2, 10, 0.01, 40, 5, samples=s)
        draws = s[20:].reshape(-1, K - 1, p).contiguous()
        _, cls = h.predict(draws, torch.from_numpy(Xh).to(cuda))
        prob_o, cls_o = opredict.predictive(Xh, draws.cpu().numpy().astype(np.float64))
    cls = cls.cpu().numpy()
    _check_classes(prob_o, cls, 1e-4)
    # the Bayes classifier with the true coefficients as a yardstick
    bayes = np.argmax(np.hstack([Xh.astype(np.float64) @ btrue.T, np.zeros((1000, 1))]), axis=1)
    assert np.mean(cls == yh) >= np.mean(bayes == yh) - 0.05
