"""Checkpoint and resume of the chain state (hmc_state_save / hmc_state_load):
chains resumed from a checkpoint continue exactly as if they had not stopped,
because the momentum and accept draws are numbered by the global iteration the
checkpoint carries (counter-based generator) and the cached gradient and log K
travel with the coefficients."""
import numpy as np
import pytest

from paper_1402_4089_gb300 import hmc, synthetic

pytestmark = pytest.mark.gpu


def _state(h, chains, K, p):
    beta = np.empty((chains, K - 1, p), np.float32)
    grad = np.empty_like(beta)
    lp = np.empty(chains, np.float64)
    it = h.get_state(chains, beta=beta, grad=grad, logpost=lp)
    return beta, grad, lp, it


@pytest.mark.parametrize("storage,engine", [("f32", 1), ("bf16", 2)])
def test_resume_from_checkpoint_is_bitwise(cuda, tmp_path, storage, engine):
    n, p, K, chains, L, eps, seed = 700, 130, 4, 2, 5, 0.02, 99
    X, y, _ = synthetic.make_problem(n, p, K, seed=21)
    kw = dict(x_storage=storage, max_chains=chains, engine=engine)
    with hmc.create(X, y, K, "gaussian", 10.0, **kw) as a:          # 6 iterations in one go
        a.sample(chains, L, eps, 6, seed)
        ref = _state(a, chains, K, p)
    path = str(tmp_path / "chains.ckpt")
    with hmc.create(X, y, K, "gaussian", 10.0, **kw) as b:          # 3, then a checkpoint
        b.sample(chains, L, eps, 3, seed)
        b.save_state(path)
    with hmc.create(X, y, K, "gaussian", 10.0, **kw) as c:          # a fresh handle resumes
        c.load_state(path)
        assert _state(c, chains, K, p)[3] == 3
        c.sample(chains, L, eps, 3, seed)
        got = _state(c, chains, K, p)
    assert ref[3] == got[3] == 6
    for r, g in zip(ref[:3], got[:3]):
        assert np.array_equal(r, g)


def test_checkpoint_errors(cuda, tmp_path):
    X, y, _ = synthetic.make_problem(300, 40, 3, seed=5)
    path = str(tmp_path / "c.ckpt")
    with hmc.create(X, y, 3, "gaussian", 10.0, max_chains=2) as h:
        with pytest.raises(hmc.HmcError) as e:
            h.save_state(path)                                 # no chain state yet
        assert e.value.status == hmc.EINVAL
        h.sample(2, 3, 0.01, 2, 1)
        h.save_state(path)
        with pytest.raises(hmc.HmcError) as e:
            h.load_state(str(tmp_path / "missing.ckpt"))
        assert e.value.status == hmc.EINVAL
        h.load_state(path)                                     # its own checkpoint loads
    X2, y2, _ = synthetic.make_problem(300, 41, 3, seed=5)
    with hmc.create(X2, y2, 3, "gaussian", 10.0, max_chains=2) as h2:
        with pytest.raises(hmc.HmcError) as e:
            h2.load_state(path)                                # another p
        assert e.value.status == hmc.EINVAL
    with hmc.create(X, y, 3, "gaussian", 10.0, max_chains=1) as h3:
        with pytest.raises(hmc.HmcError) as e:
            h3.load_state(path)                                # 2 chains > max_chains
        assert e.value.status == hmc.EINVAL
    with hmc.create(X.astype(np.float64), y, 3, "gaussian", 10.0, max_chains=2, x_storage="f64", state="f64") as h4:
        with pytest.raises(hmc.HmcError) as e:
            h4.load_state(path)                                # other state type
        assert e.value.status == hmc.EINVAL
    with open(path, "r+b") as f:
        f.truncate(60)
    with hmc.create(X, y, 3, "gaussian", 10.0, max_chains=2) as h5:
        with pytest.raises(hmc.HmcError) as e:
            h5.load_state(path)                                # truncated
        assert e.value.status == hmc.EINVAL


def test_checkpoint_of_another_posterior_is_rejected(cuda, tmp_path):
    """A checkpoint loads only into a handle of the same posterior: the prior,
    the storage of X and the layout are in its header, and the saved gradient and
    log K must agree with the handle's own at the saved coefficients (another X or
    other labels of the same shape do not)."""
    X, y, _ = synthetic.make_problem(300, 40, 3, seed=5)
    path = str(tmp_path / "c.ckpt")
    with hmc.create(X, y, 3, "gaussian", 10.0, max_chains=2) as h:
        h.sample(2, 3, 0.01, 2, 1)
        h.save_state(path)
    X2, y2, _ = synthetic.make_problem(300, 40, 3, seed=6)           # same shape, other data
    cases = [dict(X=X, y=y, prior=("gaussian", 5.0)), dict(X=X, y=y, prior=("cauchy", 10.0)),
             dict(X=X, y=y, prior=("gaussian", 10.0), x_storage="bf16"),
             dict(X=X, y=y, prior=("gaussian", 10.0), layout="masked"),
             dict(X=X2, y=y2, prior=("gaussian", 10.0)), dict(X=X, y=y2, prior=("gaussian", 10.0))]
    for kw in cases:
        extra = {k: v for k, v in kw.items() if k in ("x_storage", "layout")}
        with hmc.create(kw["X"], kw["y"], 3, kw["prior"][0], kw["prior"][1], max_chains=2, **extra) as h2:
            with pytest.raises(hmc.HmcError) as e:
                h2.load_state(path)
            assert e.value.status == hmc.EINVAL, kw
    with hmc.create(X, y, 3, "gaussian", 10.0, max_chains=2, tile=(2, 0, 0, 3)) as h3:
        h3.load_state(path)          # the same posterior on another tile loads (not bitwise-continuing)
