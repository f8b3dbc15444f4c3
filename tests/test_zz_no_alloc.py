"""The allocation-free entry point against the handle-based one.

hmc_logpost_grad_noalloc serves callers that cannot allocate device memory
at call time (a framework's pool allocator owns the GPU, or a tight loop
must not pay cudaMalloc's implicit synchronisation).  Its intermediates live
in the library's static device array; here it is called through the C ABI
twice in a row (the array keeps the first call's contents) and compared
with hmc_logpost_grad on the same inputs, within the FP32 tolerance of the
other parity tests.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1402_4089_gb300 import hmc, synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(a.astype(np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_matches_handle_path_twice(cuda):
    import torch
    L = hmc.lib()
    f = L.hmc_logpost_grad_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                  ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    n, p, K, chains = 3001, 700, 5, 2
    ldx = 1024
    X, y, _ = synthetic.make_problem(n, p, K, seed=21)
    rng = np.random.default_rng(22)
    stream = torch.cuda.current_stream(cuda)
    Xd = torch.zeros((n, ldx), dtype=torch.float32, device=cuda)
    Xd[:, :p] = torch.from_numpy(X).to(cuda)
    yd = torch.from_numpy(y).to(cuda)
    with hmc.create(X, y, K, "cauchy", 1.0, max_chains=chains) as h:
        for call in range(2):
            beta = (0.2 * rng.standard_normal((chains, K - 1, p))).astype(np.float32)
            bd = torch.from_numpy(beta).to(cuda)
            ref_lp, ref_g = h.logpost_grad(bd)
            lp = torch.full((chains,), float("nan"), dtype=torch.float64, device=cuda)
            g = torch.full((chains, K - 1, p), float("nan"), dtype=torch.float32, device=cuda)
            st = f(Xd.data_ptr(), ldx, yd.data_ptr(), n, p, K, hmc.PRIORS["cauchy"], 1.0, bd.data_ptr(), chains,
                   lp.data_ptr(), g.data_ptr(), stream.cuda_stream)
            assert st == hmc.OK, L.hmc_last_error().decode()
            torch.cuda.synchronize()
            r_lp, r_g = ref_lp.cpu().numpy(), ref_g.cpu().numpy()
            o_lp, o_g = lp.cpu().numpy(), g.cpu().numpy()
            for c in range(chains):
                assert abs(o_lp[c] - r_lp[c]) <= TOL * max(1.0, abs(r_lp[c])), (call, c, o_lp[c], r_lp[c])
                assert _rel(o_g[c], r_g[c].astype(np.float64)) <= TOL, (call, c)


def test_noalloc_rejects_oversize_and_bad_stride(cuda):
    import torch
    L = hmc.lib()
    f = L.hmc_logpost_grad_noalloc
    dummy = torch.zeros(16, device=cuda)
    # ldx not a multiple of 16
    assert f(dummy.data_ptr(), 100, dummy.data_ptr(), 1, 90, 3, 0, 1.0, dummy.data_ptr(), 1, dummy.data_ptr(),
             dummy.data_ptr(), None) == hmc.EINVAL
    # intermediates beyond the static maximum: 20 columns x 24576 x 4 B x (beta, grad, one partial) > 16 MiB? no:
    # ask for a stride that needs more than the array holds
    assert f(dummy.data_ptr(), 1 << 22, dummy.data_ptr(), 1, 1 << 22, 21, 0, 1.0, dummy.data_ptr(), 1,
             dummy.data_ptr(), dummy.data_ptr(), None) == hmc.EINVAL
    assert "scratch" in L.hmc_last_error().decode() or "tile" in L.hmc_last_error().decode()
