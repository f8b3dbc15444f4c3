"""The C-ABI library loads and exports every symbol include/hmc.h declares;
argument validation that happens before any device work (no GPU needed)."""
import ctypes
import subprocess

import pytest

from paper_1402_4089_gb300 import hmc


def test_header_declares_the_boundary():
    names = hmc.header_functions()
    for required in ["hmc_create", "hmc_create_batch", "hmc_destroy", "hmc_logpost_grad", "hmc_leapfrog",
                     "hmc_sample", "hmc_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(hmclib):
    out = subprocess.run(["nm", "-D", "--defined-only", hmc.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [f for f in hmc.header_functions() if f not in exported]
    assert not missing, missing
    for f in hmc.header_functions():
        assert getattr(hmclib, f) is not None


def test_default_opts_and_version(hmclib):
    o = hmc.default_opts()
    assert (o.x_storage, o.state, o.max_chains, o.engine, o.spin_limit) == (hmc.F32, hmc.F32, 1, 0, 0)
    assert list(o.tile) == [0, 0, 0, 0]
    assert b"sm_103a" in hmclib.hmc_version()


def _create(**kw):
    args = dict(X=None, x_dtype=hmc.F32, y=None, n=10, p=3, K=3, prior=0, scale=1.0, opts=None)
    args.update(kw)
    h = ctypes.c_void_p()
    o = args["opts"]
    st = hmc.lib().hmc_create(args["X"], args["x_dtype"], args["y"], args["n"], args["p"], args["K"], args["prior"],
                              args["scale"], ctypes.byref(o) if o is not None else None, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw,msg", [
    (dict(K=1), "K"), (dict(p=0), "p"), (dict(n=-1), "n"), (dict(scale=0.0), "prior_scale"),
    (dict(prior=7), "prior"), (dict(x_dtype=hmc.BF16), "x_dtype"), (dict(), "NULL X"),
])
def test_create_rejects_bad_arguments_before_device_work(hmclib, kw, msg):
    st, h = _create(**kw)
    assert st == hmc.EINVAL
    assert h.value is None
    assert msg.lower() in hmclib.hmc_last_error().decode().lower()


def test_create_rejects_bad_opts(hmclib):
    for field, val in [("state", hmc.BF16), ("max_chains", 0), ("engine", 5), ("spin_limit", -1)]:
        o = hmc.default_opts()
        setattr(o, field, val)
        st, _ = _create(opts=o)
        assert st == hmc.EINVAL, field
    o = hmc.default_opts()
    o.x_storage = hmc.F64               # F64 storage needs F64 state
    assert _create(opts=o)[0] == hmc.EINVAL
    o = hmc.default_opts()
    o.tile[0] = 17                       # cluster sizes are 1..16
    assert _create(opts=o)[0] == hmc.EINVAL


def test_null_handle_calls(hmclib):
    assert hmclib.hmc_destroy(None) == hmc.OK
    assert hmclib.hmc_logpost_grad(None, None, 1, None, None) == hmc.EINVAL
    assert hmclib.hmc_leapfrog(None, None, None, None, None, 1, 1, 0.1) == hmc.EINVAL
    assert hmclib.hmc_sample(None, 1, 1, 0.1, 1, 0, None, None, 1, None) == hmc.EINVAL
    assert hmclib.hmc_chain_size(None) == -1
