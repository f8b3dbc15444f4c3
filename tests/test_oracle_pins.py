"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with a retyped copy of itself: finite
differences, closed forms, a textbook special case (K = 2 is logistic
regression), brute force with explicit one-hot Y and no log-sum-exp shift,
invariants of the leapfrog map (reversibility, O(eps^2) energy error, the
exact linear map of a Gaussian target), sampling moments of a known
distribution, a library implementation of the same generator, and the ESS of
an AR(1) series with a known closed form.
"""
import math

import numpy as np
import pytest
import scipy.special
import scipy.stats

from oracle import ess, hmc, model, philox, quant
from paper_1402_4089_gb300 import synthetic


def _small(n=37, p=6, K=4, seed=3, bscale=0.7):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    y = rng.integers(0, K, size=n)
    beta = bscale * rng.standard_normal((K - 1, p))
    return X, y, beta


# --- P1: finite-difference gradient (Eq. gradient / fullgrad) -------------

@pytest.mark.parametrize("kind,scale", [("gaussian", 10.0), ("gaussian", 1.0), ("cauchy", 1.0), ("cauchy", 2.5)])
def test_fd_gradient_every_coordinate(kind, scale):
    X, y, _, _ = synthetic.make_workload("plain_fp64", n=200, p=12)
    rng = np.random.default_rng(1)
    beta = 0.3 * rng.standard_normal((2, 12))
    g = model.grad_log_kernel(X, y, beta, kind, scale)
    h = 1e-4
    fd = np.empty_like(beta)
    for k in range(beta.shape[0]):
        for j in range(beta.shape[1]):
            bp = beta.copy(); bp[k, j] += h
            bm = beta.copy(); bm[k, j] -= h
            fd[k, j] = (model.log_kernel(X, y, bp, kind, scale) - model.log_kernel(X, y, bm, kind, scale)) / (2 * h)
    rel = np.linalg.norm(g - fd) / np.linalg.norm(fd)
    assert rel < 1e-6, rel


def test_fd_gradient_plain_workload_full_size():
    X, y, _, spec = synthetic.make_workload("plain_fp64")
    rng = np.random.default_rng(2)
    beta = 0.1 * rng.standard_normal((spec["K"] - 1, spec["p"]))
    g = model.grad_log_kernel(X, y, beta, "gaussian", 10.0)
    h = 1e-4
    for (k, j) in [(0, 0), (1, 49), (0, 17), (1, 3)]:
        bp = beta.copy(); bp[k, j] += h
        bm = beta.copy(); bm[k, j] -= h
        fd = (model.log_kernel(X, y, bp, "gaussian", 10.0) - model.log_kernel(X, y, bm, "gaussian", 10.0)) / (2 * h)
        assert abs(g[k, j] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_paper_sign_of_prior_gradient_is_caught_by_fd(monkeypatch):
    """The Appendix prints Gamma = +2b/(1+b^2); planting that sign in the oracle
    makes the finite-difference pin fail, so the pin decides the reading."""
    X, y, beta = _small()
    orig = model.prior_grad

    def paper_sign(b, kind, scale):
        return -orig(b, kind, scale)

    monkeypatch.setattr(model, "prior_grad", paper_sign)
    g = model.grad_log_kernel(X, y, beta, "cauchy", 1.0)
    h = 1e-5
    bp = beta.copy(); bp[0, 0] += h
    bm = beta.copy(); bm[0, 0] -= h
    fd = (model.log_kernel(X, y, bp, "cauchy", 1.0) - model.log_kernel(X, y, bm, "cauchy", 1.0)) / (2 * h)
    assert abs(g[0, 0] - fd) > 1e-3


# --- P2: softmax rows (Eq. softmax) -----------------------------------------

def test_softmax_rows_sum_to_one_and_extreme_logits():
    rng = np.random.default_rng(0)
    Z = rng.standard_normal((50, 7)) * 5
    Z[0] = [800, -800, 0, 799, 1, 2, 3]
    Z[1] = [-800] * 7
    P = model.softmax(Z)
    assert np.all(np.abs(P.sum(axis=1) - 1.0) <= 1e-15 * 7)
    assert np.all((P >= 0) & (P <= 1))
    assert abs(P[0, 0] - 1.0 / (1.0 + math.exp(-1.0))) < 1e-15
    ref = scipy.special.softmax(Z[2:], axis=1)
    assert np.allclose(P[2:], ref, rtol=1e-14, atol=1e-300)


# --- brute force on tiny inputs with one-hot Y (Eqs. loglike, logkernel) ----

def test_log_kernel_brute_force_one_hot():
    X, y, beta = _small(n=9, p=3, K=3, bscale=0.5)
    n, p = X.shape
    K = beta.shape[0] + 1
    B = np.zeros((p, K))
    B[:, :K - 1] = beta.T
    Y = np.zeros((n, K))
    for i in range(n):
        Y[i, y[i]] = 1.0
    total = 0.0
    for i in range(n):
        denom = sum(math.exp(sum(X[i, j] * B[j, c] for j in range(p))) for c in range(K))
        for k in range(K):
            psi = math.exp(sum(X[i, j] * B[j, k] for j in range(p))) / denom
            total += Y[i, k] * math.log(psi)
    for k in range(K - 1):
        for j in range(p):
            total += -math.log(1.0 + beta[k, j] ** 2)
    assert abs(model.log_kernel(X, y, beta, "cauchy", 1.0) - total) < 1e-12 * max(1, abs(total))


def test_gradient_brute_force_one_hot():
    X, y, beta = _small(n=8, p=3, K=3, bscale=0.5)
    n, p = X.shape
    K = beta.shape[0] + 1
    g = np.zeros((K - 1, p))
    for k in range(K - 1):
        for j in range(p):
            acc = 0.0
            for i in range(n):
                logits = [sum(X[i, q] * (beta[c, q] if c < K - 1 else 0.0) for q in range(p)) for c in range(K)]
                e = [math.exp(v) for v in logits]
                acc += X[i, j] * ((1.0 if y[i] == k else 0.0) - e[k] / sum(e))
            g[k, j] = acc - beta[k, j] / 4.0   # Gaussian sigma = 2: d/db (-b^2/8)
    assert np.allclose(model.grad_log_kernel(X, y, beta, "gaussian", 2.0), g, rtol=1e-12, atol=1e-13)


# --- P3: closed form at beta = 0 --------------------------------------------

@pytest.mark.parametrize("K", [2, 3, 10])
def test_closed_form_at_zero(K):
    X, y, _ = _small(n=41, p=5, K=K)
    beta = np.zeros((K - 1, 5))
    assert abs(model.log_kernel(X, y, beta, "cauchy", 1.0) - (-41 * math.log(K))) < 1e-12
    Y = np.eye(K)[y][:, :K - 1]
    expect = (X.T @ (Y - 1.0 / K)).T
    assert np.allclose(model.grad_log_kernel(X, y, beta, "gaussian", 3.0), expect, atol=1e-13)


# --- P4: K = 2 is logistic regression ----------------------------------------

def test_two_classes_is_logistic_regression():
    X, y, beta = _small(n=60, p=4, K=2, bscale=1.5)
    z = X @ beta[0]
    yp = (y == 0).astype(float)                 # the free class is class 1 of 2
    ll = np.sum(yp * z - np.logaddexp(0.0, z))
    assert abs(model.log_likelihood(X, y, beta) - ll) < 1e-11
    grad = X.T @ (yp - scipy.special.expit(z))
    assert np.allclose(model.grad_log_kernel(X, y, beta, "gaussian", 1e300)[0], grad, rtol=1e-12, atol=1e-12)


# --- n = 0: prior only --------------------------------------------------------

def test_prior_only_terms():
    b = np.array([[0.0, 1.0, -2.0]])
    X = np.zeros((0, 3))
    y = np.zeros(0, dtype=np.int64)
    assert abs(model.log_kernel(X, y, b, "cauchy", 1.0) - (-(math.log(2) + math.log(5)))) < 1e-15
    assert abs(model.log_kernel(X, y, b, "gaussian", 2.0) - (-(1 + 4) / 8.0)) < 1e-15
    assert np.allclose(model.grad_log_kernel(X, y, b, "cauchy", 1.0), [[0.0, -1.0, 0.8]])


# --- P5: reversibility of the leapfrog map -----------------------------------

def test_leapfrog_reversibility_plain_workload():
    X, y, _, spec = synthetic.make_workload("plain_fp64")
    rng = np.random.default_rng(5)
    beta0 = 0.05 * rng.standard_normal((2, 50))
    eta0 = rng.standard_normal((2, 50))
    b1, e1, _, _ = hmc.leapfrog(X, y, beta0, eta0, spec["eps"], spec["L"], "gaussian", 10.0)
    b2, e2, _, _ = hmc.leapfrog(X, y, b1, -e1, spec["eps"], spec["L"], "gaussian", 10.0)
    assert np.max(np.abs(b2 - beta0)) <= 1e-12 * max(1.0, np.max(np.abs(beta0)))
    assert np.max(np.abs(-e2 - eta0)) <= 1e-12 * max(1.0, np.max(np.abs(eta0)))
    assert np.max(np.abs(b1 - beta0)) > 1e-3        # the trajectory actually moved


# --- P6: energy error is O(eps^2) --------------------------------------------

def test_energy_error_second_order():
    X, y, _, _ = synthetic.make_workload("plain_fp64")
    rng = np.random.default_rng(6)
    beta0 = 0.2 * rng.standard_normal((2, 50))
    eta0 = rng.standard_normal((2, 50))
    lk0 = model.log_kernel(X, y, beta0, "gaussian", 10.0)
    h0 = hmc.hamiltonian(lk0, eta0)
    errs = []
    for eps, L in [(0.004, 10), (0.002, 20), (0.001, 40)]:
        _, e1, lk1, _ = hmc.leapfrog(X, y, beta0, eta0, eps, L, "gaussian", 10.0)
        errs.append(abs(hmc.hamiltonian(lk1, e1) - h0))
    for a, b in zip(errs, errs[1:]):
        assert 3.0 <= a / b <= 5.0, errs


# --- P7: exact map for a Gaussian target -------------------------------------

def test_gaussian_prior_leapfrog_matrix():
    sigma, eps = 1.7, 0.3
    b0 = np.array([[0.4, -1.1, 2.0]])
    e0 = np.array([[1.0, 0.25, -0.5]])
    X = np.zeros((0, 3))
    y = np.zeros(0, dtype=np.int64)
    b1, e1, _, _ = hmc.leapfrog(X, y, b0, e0, eps, 1, "gaussian", sigma)
    a = 1.0 - eps * eps / (2 * sigma * sigma)
    M = np.array([[a, eps], [-(eps / sigma ** 2) * (1 - eps * eps / (4 * sigma * sigma)), a]])
    for j in range(3):
        expect = M @ np.array([b0[0, j], e0[0, j]])
        assert abs(b1[0, j] - expect[0]) <= 1e-15 * 4
        assert abs(e1[0, j] - expect[1]) <= 1e-15 * 4


# --- P8: prior-only chains reproduce the prior's moments ---------------------

def _prior_only_chain_stats(kinetic_half=True, kind="gaussian", iters=3000, coords=64):
    """One prior-only chain (n = 0) over `coords` independent coordinates; returns
    draws shaped (coords, iters)."""
    X = np.zeros((0, coords))
    y = np.zeros(0, dtype=np.int64)
    if kinetic_half:
        res = hmc.sample(X, y, 2, kind, 1.0, 1, 13, 0.1, iters, seed=11)
        return res["samples"][:, 0, 0, :].T
    orig = hmc.hamiltonian
    try:
        hmc.hamiltonian = lambda logk, eta: -float(logk) + float(np.sum(np.asarray(eta) ** 2))
        res = hmc.sample(X, y, 2, kind, 1.0, 1, 13, 0.1, iters, seed=11)
    finally:
        hmc.hamiltonian = orig
    return res["samples"][:, 0, 0, :].T


def _moments_ok(draws):
    d = draws[:, draws.shape[1] // 10:]
    m_se, n_ess = ess.mcse_mean(d)
    mean = d.mean()
    sq = d * d
    v_se, _ = ess.mcse_mean(sq)
    var = sq.mean()
    return abs(mean) <= 3 * m_se and abs(var - 1.0) <= 3 * v_se, (mean, m_se, var, v_se, n_ess)


def test_prior_only_gaussian_moments():
    ok, info = _moments_ok(_prior_only_chain_stats(True))
    assert ok, info


def test_literal_kinetic_energy_fails_moments():
    """Eq. accept read literally (eta.eta with no 1/2) targets the wrong
    distribution: the same moment check fails, which pins the 1/2 reading."""
    ok, info = _moments_ok(_prior_only_chain_stats(False))
    assert not ok, info


def test_prior_only_cauchy_quartiles():
    d = _prior_only_chain_stats(True, kind="cauchy")
    d = d[:, 300:].ravel()
    q1, med, q3 = np.quantile(d, [0.25, 0.5, 0.75])
    assert abs(med) < 0.1 and abs(q1 + 1.0) < 0.15 and abs(q3 - 1.0) < 0.15, (q1, med, q3)


# --- P9: ESS estimator on AR(1) ----------------------------------------------

def test_ess_ar1_closed_form():
    rho, n = 0.9, 1_000_000
    rng = np.random.default_rng(9)
    e = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = e[0] / math.sqrt(1 - rho * rho)
    for i in range(1, n):
        x[i] = rho * x[i - 1] + e[i]
    expect = n * (1 - rho) / (1 + rho)
    assert abs(ess.ess_geyer(x) - expect) / expect < 0.05


def test_ess_iid_close_to_n():
    rng = np.random.default_rng(10)
    x = rng.standard_normal(200_000)
    assert abs(ess.ess_geyer(x) / 200_000 - 1.0) < 0.05


# --- P10: Philox4x64-10 against numpy's library implementation ---------------

def test_philox_matches_numpy_library():
    for key in [(0, 0), (12345, 0), (2 ** 63 + 7, 99)]:
        for ctr in [(0, 0, 0, 0), (5, 0, 0, 0), (1, 2, 3, 4), (2 ** 64 - 2, 7, 9, 1)]:
            bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
            expect = bg.random_raw(4)                       # numpy pre-increments
            nxt = list(ctr)
            nxt[0] = (nxt[0] + 1) % 2 ** 64
            got = philox.philox4x64_10([np.uint64(v) for v in nxt], key)
            assert [int(v) for v in got] == [int(v) for v in expect]


def test_momentum_normals_are_standard_normal():
    z = philox.momentum_normals(seed=3, iteration=1, chain=2, count=200_001)
    assert z.shape == (200_001,)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3
    # prefix property: a shorter draw is a prefix of a longer one
    assert np.array_equal(philox.momentum_normals(3, 1, 2, 13), z[:13])
    u = [philox.accept_uniform(3, t, 0) for t in range(2000)]
    assert 0 < min(u) and max(u) < 1 and scipy.stats.kstest(u, "uniform").pvalue > 1e-3


# --- storage formats -----------------------------------------------------------

def test_bf16_rounding_by_hand():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, -3.5, 0.0], dtype=np.float32)
    expect = np.array([1.0, 1.0, 1.0 + 4 * 2 ** -8, 1.0 + 2 ** -7, -3.5, 0.0])
    assert np.array_equal(quant.bf16_round(vals).astype(np.float64), expect)


def test_e4m3_table_and_rounding():
    t = quant.e4m3_table()
    assert t[0x7E] == 448.0 and t[0x08] == 2.0 ** -6 and t[0x01] == 2.0 ** -9 and np.isnan(t[0x7F])
    finite = t[np.isfinite(t)]
    assert len(np.unique(finite)) == 253            # +0 and -0 collapse
    codes = quant.e4m3_encode(np.array([1.0, 1.0625, 1.1875, 500.0, -500.0, 2 ** -10, 3 * 2 ** -10, -0.0]))
    # 1.0625 is halfway between 1.0 (m=0, even) and 1.125 (m=1): ties to even -> 1.0
    # 1.1875 is halfway between 1.125 (m=1) and 1.25 (m=2): -> 1.25
    # 2^-10 is halfway between 0 and 2^-9 (m=1): -> 0; 3*2^-10 between m=1 and m=2 -> m=2
    assert list(quant.e4m3_decode(codes)) == [1.0, 1.0, 1.25, 448.0, -448.0, 0.0, 2 * 2 ** -9, 0.0]
    # signed zero: -0.0 and a negative value that rounds to zero keep the sign (code 0x80)
    z = quant.e4m3_encode(np.array([0.0, -0.0, -2 ** -11, 2 ** -11]))
    assert list(z) == [0x00, 0x80, 0x80, 0x00]
    assert np.signbit(quant.e4m3_decode(z)).tolist() == [False, True, True, False]


def test_fp8_column_scales_reconstruct():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((300, 7)).astype(np.float32)
    X[:, 3] = 0.0
    codes, s = quant.fp8_quantize(X)
    assert s[3] == 1.0
    Xq = quant.fp8_dequantize(codes, s)
    for j in range(7):
        if j == 3:
            assert np.all(Xq[:, j] == 0)
            continue
        assert np.max(np.abs(Xq[:, j])) == pytest.approx(np.max(np.abs(X[:, j])), rel=1e-6)
        # relative spacing of E4M3 normals is 2^-3: rounding error <= 2^-4 relative
        big = np.abs(X[:, j]) > 2.0 ** -6 * s[j]
        assert np.all(np.abs(Xq[big, j] - X[big, j]) <= 2 ** -4 * np.abs(X[big, j]) * (1 + 1e-6))


def _small_problem():
    rng = np.random.default_rng(77)
    X = rng.standard_normal((200, 8))
    beta_true = rng.standard_normal((2, 8))
    z = np.concatenate([X @ beta_true.T, np.zeros((200, 1))], axis=1)
    y = np.array([rng.choice(3, p=np.exp(r - r.max()) / np.exp(r - r.max()).sum()) for r in z], dtype=np.int32)
    return X, y


def test_resume_continues_the_chain():
    """Counter-based draws numbered by the global iteration (c-12): 6 iterations
    equal 3 iterations followed by 3 more started from the kept state at
    iteration index 3 -- the property a checkpoint relies on."""
    X, y = _small_problem()
    full = hmc.sample(X, y, 3, "gaussian", 10.0, 2, 5, 0.05, 6, 123)
    first = hmc.sample(X, y, 3, "gaussian", 10.0, 2, 5, 0.05, 3, 123)
    rest = hmc.sample(X, y, 3, "gaussian", 10.0, 2, 5, 0.05, 3, 123, beta0=first["beta"], iter0=3)
    assert np.array_equal(full["samples"][:3], first["samples"])
    assert np.array_equal(full["samples"][3:], rest["samples"])
    assert np.array_equal(full["accept"][3:], rest["accept"])


def test_tempered_acceptance_reading():
    """Annealed burn-in (Sec. 3.2): accept iff log u < (H0 - H1) / T.  T = 1 is the
    plain test; a huge T accepts every finite proposal; raising T never turns an
    accepted proposal into a rejected one."""
    X, y = _small_problem()
    args = (X, y, 3, "gaussian", 10.0, 4, 5, 0.4, 5, 9)
    plain = hmc.sample(*args)
    ones = hmc.sample(*args, temps=np.ones(5))
    assert np.array_equal(plain["samples"], ones["samples"]) and np.array_equal(plain["accept"], ones["accept"])
    hot = hmc.sample(*args, temps=np.full(5, 1e12))
    assert np.all(hot["accept"] | hot["diverged"])
    # first iteration: same proposal at every temperature
    warm = hmc.sample(*args, temps=np.full(5, 3.0))
    assert np.all(warm["accept"][0] >= plain["accept"][0])
    assert np.array_equal(warm["dH"][0], plain["dH"][0])


# --- row-blocked evaluation (for X too large to hold in FP64 at once) ---------

def test_row_blocks_equal_the_whole_problem():
    X, y, _ = _small(n=53, p=7, K=4)
    rng = np.random.default_rng(12)
    betas = [0.4 * rng.standard_normal((3, 7)) for _ in range(2)]
    blocks = [(X[a:a + 20], y[a:a + 20]) for a in range(0, 53, 20)]
    lk, g, Z = model.log_kernel_and_grad_by_rows(blocks, betas, "cauchy", 1.5)
    for c, b in enumerate(betas):
        assert abs(lk[c] - model.log_kernel(X, y, b, "cauchy", 1.5)) < 1e-11
        assert np.allclose(g[c], model.grad_log_kernel(X, y, b, "cauchy", 1.5), rtol=1e-12, atol=1e-12)
        assert np.allclose(Z[c], model.full_logits(X, b), rtol=0, atol=1e-13)
