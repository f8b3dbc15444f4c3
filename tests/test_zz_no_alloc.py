"""The allocation-free entry point, hmc_logpost_grad_noalloc.

It serves callers that cannot allocate device memory at call time (a
framework's pool allocator owns the GPU, or a tight loop must not pay
cudaMalloc's implicit synchronisation); its intermediates live in the
library's static device array.  Here it is called through the C ABI twice in a
row (the array keeps the first call's contents) and compared with the FP64
oracle and with hmc_logpost_grad on the same inputs, within the FP32 tolerance
of the other parity tests; n = 0 (prior only), K = 2, the widest tiles, many
row tiles at a narrow stride (where the array's room for per-cluster partial
slices can bound the clusters of the fused pass) and a label outside [0, K)
are covered.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from oracle import model
from paper_1402_4089_gb300 import hmc, synthetic
from parity_util import assert_grad, lk_err

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _fn():
    """The entry point with its argument types (set here, so the file runs alone)."""
    f = hmc.lib().hmc_logpost_grad_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                  ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    return f


def _call(cuda, X, y, beta, K, ldx, prior=("cauchy", 1.0)):
    """One call on device copies of the inputs (X zero-padded to ldx columns)."""
    import torch
    n, p = X.shape
    chains = beta.shape[0]
    Xd = torch.zeros((max(n, 1), ldx), dtype=torch.float32, device=cuda)
    if n:
        Xd[:n, :p] = torch.from_numpy(X).to(cuda)
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.int32)).to(cuda) if n else torch.zeros(1, dtype=torch.int32,
                                                                                                 device=cuda)
    bd = torch.from_numpy(beta).to(cuda)
    lp = torch.full((chains,), float("nan"), dtype=torch.float64, device=cuda)
    g = torch.full(beta.shape, float("nan"), dtype=torch.float32, device=cuda)
    st = _fn()(Xd.data_ptr(), ldx, yd.data_ptr(), n, p, K, hmc.PRIORS[prior[0]], prior[1], bd.data_ptr(), chains,
               lp.data_ptr(), g.data_ptr(), torch.cuda.current_stream(cuda).cuda_stream)
    torch.cuda.synchronize()
    return st, lp.cpu().numpy(), g.cpu().numpy()


def _check_oracle(X, y, beta, lp, g, prior, tol=TOL):
    for c in range(beta.shape[0]):
        b = beta[c].astype(np.float64)
        lk_o = model.log_kernel(X.astype(np.float64), y, b, *prior)
        assert lk_err(lp[c], lk_o) <= tol, (c, lp[c], lk_o)
        assert_grad(g[c], model.grad_log_kernel(X.astype(np.float64), y, b, *prior), tol, c)


def test_noalloc_matches_oracle_and_handle_path_twice(cuda):
    import torch
    n, p, K, chains, ldx = 3001, 700, 5, 2, 1024
    X, y, _ = synthetic.make_problem(n, p, K, seed=21)
    rng = np.random.default_rng(22)
    with hmc.create(X, y, K, "cauchy", 1.0, max_chains=chains) as h:
        for call in range(2):
            beta = (0.2 * rng.standard_normal((chains, K - 1, p))).astype(np.float32)
            st, lp, g = _call(cuda, X, y, beta, K, ldx)
            assert st == hmc.OK, hmc.lib().hmc_last_error().decode()
            _check_oracle(X, y, beta, lp, g, ("cauchy", 1.0))
            r_lp, r_g = (t.cpu().numpy() for t in h.logpost_grad(torch.from_numpy(beta).to(cuda)))
            for c in range(chains):
                assert lk_err(lp[c], r_lp[c]) <= TOL, (call, c)
                assert_grad(g[c], r_g[c], TOL, (call, c))


@pytest.mark.parametrize("n,p,K,chains,ldx", [(0, 40, 3, 2, 256), (777, 33, 2, 3, 256), (1, 5, 2, 1, 16)])
def test_noalloc_edge_shapes(cuda, n, p, K, chains, ldx):
    rng = np.random.default_rng(n + p + K)
    X = rng.standard_normal((n, p)).astype(np.float32)
    y = rng.integers(0, K, size=n).astype(np.int32)
    beta = (0.3 * rng.standard_normal((chains, K - 1, p))).astype(np.float32)
    for _ in range(2):
        st, lp, g = _call(cuda, X, y, beta, K, ldx, prior=("gaussian", 2.0))
        assert st == hmc.OK, hmc.lib().hmc_last_error().decode()
        _check_oracle(X, y, beta, lp, g, ("gaussian", 2.0))


@pytest.mark.parametrize("n,p,K,ldx", [(3000, 20000, 7, 20480), (4000, 16000, 13, 16384), (3000, 10000, 21, 10240),
                                       (20000, 1000, 21, 1024)])
def test_noalloc_wide_and_long_problems(cuda, n, p, K, ldx):
    """The widest tiles for 6, 12 and 20 columns, and many row tiles at a narrow
    stride (where the array's room for cluster slices can bound the clusters)."""
    import torch
    X, y, _ = synthetic.make_problem(n, p, K, seed=25, x_sd=0.1)
    beta = (0.05 * np.random.default_rng(26).standard_normal((1, K - 1, p))).astype(np.float32)
    st, lp, g = _call(cuda, X, y, beta, K, ldx, prior=("gaussian", 1.0))
    assert st == hmc.OK, hmc.lib().hmc_last_error().decode()
    _check_oracle(X, y, beta, lp, g, ("gaussian", 1.0))
    with hmc.create(X, y, K, "gaussian", 1.0) as h:
        r_lp, r_g = (t.cpu().numpy() for t in h.logpost_grad(torch.from_numpy(beta).to(cuda)))
    assert lk_err(lp[0], r_lp[0]) <= TOL
    assert_grad(g[0], r_g[0], TOL)


def test_noalloc_rejects_bad_arguments(cuda):
    import torch
    f = _fn()
    dummy = torch.zeros(16, device=cuda)
    d = dummy.data_ptr()
    assert f(d, 100, d, 1, 90, 3, 0, 1.0, d, 1, d, d, None) == hmc.EINVAL        # ldx not a multiple of 16
    assert f(d, 1 << 22, d, 1, 1 << 22, 21, 0, 1.0, d, 1, d, d, None) == hmc.EINVAL   # no tile for this stride
    assert "tile" in hmc.lib().hmc_last_error().decode()
    assert f(d, 256, d, 1, 200, 22, 0, 1.0, d, 1, d, d, None) == hmc.EINVAL       # 21 columns > 20
    # a label outside [0, K) is flagged by the fused pass
    X = np.ones((40, 8), np.float32)
    y = np.zeros(40, np.int32)
    y[17] = 3
    st, _, _ = _call(cuda, X, y, np.zeros((1, 2, 8), np.float32), 3, 16)
    assert st == hmc.ENONFINITE, hmc.lib().hmc_last_error().decode()
    # and the entry point works again afterwards
    y[17] = 2
    st, lp, g = _call(cuda, X, y, np.zeros((1, 2, 8), np.float32), 3, 16)
    assert st == hmc.OK
    _check_oracle(X, y, np.zeros((1, 2, 8), np.float32), lp, g, ("cauchy", 1.0))
