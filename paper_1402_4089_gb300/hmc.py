"""Python binding of libhmc (include/hmc.h): argument marshalling only.

Every step of the sampler runs in the library's CUDA kernels.  PyTorch
provides device memory and the stream; numpy arrays are accepted for
uploads and host-side outputs.  There is no CPU fallback: if ``libhmc.so``
is missing or cannot be loaded, importing the library raises.

Names follow the C ABI: ``create`` / ``create_batch`` (hmc_create[_batch]),
``Handle.logpost_grad`` (hmc_logpost_grad), ``Handle.leapfrog``
(hmc_leapfrog), ``Handle.sample`` (hmc_sample / hmc_sample_tempered).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhmc.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EUNSUPPORTED = range(7)
STATUS_NAMES = ["HMC_OK", "HMC_EINVAL", "HMC_ENOMEM", "HMC_ECUDA", "HMC_ETIMEOUT", "HMC_ENONFINITE",
                "HMC_EUNSUPPORTED"]
F64, F32, BF16, FP8E4M3 = range(4)
DTYPES = {"f64": F64, "f32": F32, "bf16": BF16, "fp8": FP8E4M3}
PRIORS = {"gaussian": 0, "cauchy": 1}
LAYOUTS = {"free": 0, "masked": 1, "unconstrained": 2}


class HmcError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {message}")


class Opts(ctypes.Structure):
    _fields_ = [("x_storage", ctypes.c_int), ("state", ctypes.c_int), ("max_chains", ctypes.c_int32),
                ("engine", ctypes.c_int32), ("spin_limit", ctypes.c_int64), ("stream", ctypes.c_void_p),
                ("tile", ctypes.c_int32 * 4), ("layout", ctypes.c_int32)]


class ChainStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("accepted", ctypes.c_int64), ("diverged", ctypes.c_int64),
                ("sum_abs_dH", ctypes.c_double), ("logpost", ctypes.c_double)]


_lib = None


def lib():
    """The loaded library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libhmc.so not found at {LIB_PATH}: run `python -m paper_1402_4089_gb300.build` "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "hmc_default_opts": (None, [ctypes.POINTER(Opts)]),
        "hmc_version": (ctypes.c_char_p, []),
        "hmc_last_error": (ctypes.c_char_p, []),
        "hmc_create": (st, [P, ctypes.c_int, P, I64, I64, I32, ctypes.c_int, D, ctypes.POINTER(Opts), ctypes.POINTER(P)]),
        "hmc_create_batch": (st, [I32, ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(P), ctypes.POINTER(I64),
                                  ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.c_int, D, ctypes.POINTER(Opts),
                                  ctypes.POINTER(P)]),
        "hmc_destroy": (st, [P]),
        "hmc_chain_size": (I64, [P]),
        "hmc_logpost_grad": (st, [P, P, I32, P, P]),
        "hmc_leapfrog": (st, [P, P, P, P, P, I32, I32, D]),
        "hmc_sample": (st, [P, I32, I32, D, I64, U64, P, P, I32, P]),
        "hmc_sample_tempered": (st, [P, I32, I32, D, I64, U64, P, P, I32, P, P]),
        "hmc_get_state": (st, [P, I32, P, P, P, P]),
        "hmc_annealing_schedule": (st, [D, D, I64, P]),
        "hmc_predict": (st, [P, I32, P, I64, P, ctypes.c_int, I64, P, P]),
        "hmc_get_x": (st, [P, I32, P, P]),
        "hmc_state_save": (st, [P, ctypes.c_char_p]),
        "hmc_state_load": (st, [P, ctypes.c_char_p]),
        "hmc_describe": (ctypes.c_char_p, [P]),
        "hmc_set_timing": (st, [P, I32]),
        "hmc_fused_kernel_time": (st, [P, ctypes.POINTER(D), ctypes.POINTER(I64)]),
        "hmc_first_pass_time": (st, [P, ctypes.POINTER(D)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status):
    if status != OK:
        raise HmcError(status, lib().hmc_last_error().decode())


def default_opts():
    o = Opts()
    lib().hmc_default_opts(ctypes.byref(o))
    return o


def _ptr(x):
    """Raw address of a torch tensor / numpy array / None (no copies made here)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays passed to libhmc must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to libhmc must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_ptr(stream):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    return getattr(stream, "cuda_stream", stream)


def _make_opts(x_storage, state, max_chains, engine, spin_limit, stream, tile, layout="free"):
    o = default_opts()
    o.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
    o.x_storage = DTYPES[x_storage] if isinstance(x_storage, str) else int(x_storage)
    o.state = DTYPES[state] if isinstance(state, str) else int(state)
    o.max_chains = int(max_chains)
    o.engine = int(engine)
    o.spin_limit = int(spin_limit)
    o.stream = _stream_ptr(stream)
    for i, v in enumerate(tile or (0, 0, 0, 0)):
        o.tile[i] = int(v)
    return o


def _x_in_dtype(X):
    dt = getattr(X, "dtype", None)
    s = str(dt)
    if "float64" in s:
        return F64
    if "float32" in s:
        return F32
    raise TypeError(f"X must be float32 or float64, got {dt}")


class Handle:
    """One uploaded problem (or batch of problems) and its persistent chain state."""

    def __init__(self, ptr, keep, shapes, state, max_chains, layout=0):
        self._h = ctypes.c_void_p(ptr)
        self._keep = keep
        self.shapes = shapes            # [(n, p, K)]
        self.state = state
        self.max_chains = max_chains
        self.layout = layout

    def rows(self, b=0):
        """Coefficient rows per chain of problem b in the beta layout (K-1, or K for the
        masked and unconstrained layouts)."""
        return self.shapes[b][2] - (1 if self.layout == LAYOUTS["free"] else 0)

    # -- plumbing
    def close(self):
        if self._h:
            _check(lib().hmc_destroy(self._h))
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def nprob(self):
        return len(self.shapes)

    @property
    def chain_size(self):
        return int(lib().hmc_chain_size(self._h))

    def describe(self):
        import json
        return json.loads(lib().hmc_describe(self._h).decode())

    def torch_dtype(self):
        import torch
        return torch.float64 if self.state == F64 else torch.float32

    def np_dtype(self):
        return np.float64 if self.state == F64 else np.float32

    # -- compute
    def logpost_grad(self, beta, chains=None, logpost=None, grad=None):
        """log K and its gradient at `beta` (beta layout, host or device).  Outputs are
        allocated like `beta` (same device / numpy) unless given."""
        chains = self._chains_of(beta, chains)
        logpost, grad = self._alloc_like(beta, chains, logpost, grad)
        _check(lib().hmc_logpost_grad(self._h, _ptr(beta), chains, _ptr(logpost), _ptr(grad)))
        return logpost, grad

    def leapfrog(self, beta, eta, L, eps, grad=None, logpost=None, chains=None):
        """L leapfrog updates of (beta, eta) in place; grad / logpost are outputs at the
        new beta (grad is also the input gradient when given)."""
        chains = self._chains_of(beta, chains)
        _check(lib().hmc_leapfrog(self._h, _ptr(beta), _ptr(eta), _ptr(grad), _ptr(logpost), chains, int(L),
                                  float(eps)))
        return beta, eta, grad, logpost

    def sample(self, chains, L, eps, iters, seed, beta0=None, samples=None, thin=1, temps=None):
        """HMC iterations; returns per-(problem, chain) stats as a list of dicts."""
        stats = (ChainStats * (self.nprob * chains))()
        t = None
        if temps is not None:
            t = np.ascontiguousarray(temps, dtype=np.float64)
            if t.shape[0] < iters:
                raise ValueError("temps must have one entry per iteration")
        if t is None:
            _check(lib().hmc_sample(self._h, chains, int(L), float(eps), int(iters), int(seed), _ptr(beta0),
                                    _ptr(samples), int(thin), ctypes.cast(stats, ctypes.c_void_p)))
        else:
            _check(lib().hmc_sample_tempered(self._h, chains, int(L), float(eps), int(iters), int(seed), _ptr(beta0),
                                             _ptr(samples), int(thin), ctypes.cast(stats, ctypes.c_void_p),
                                             t.ctypes.data))
        return [dict(iterations=s.iterations, accepted=s.accepted, diverged=s.diverged, sum_abs_dH=s.sum_abs_dH,
                     logpost=s.logpost) for s in stats]

    def predict(self, draws, Xnew, b=0, prob=None, cls=None):
        """Posterior predictive (hmc_predict): mean softmax over the coefficient draws
        ([ndraws][rows][p] of the state type) for the rows of Xnew, and its argmax.
        Outputs are allocated like Xnew (numpy or the same device) unless given."""
        n, p, K = self.shapes[b]
        ndraws, r = divmod(draws.numel() if hasattr(draws, "numel") else draws.size, self.rows(b) * p)
        if r or ndraws < 1:
            raise ValueError("draws must hold whole coefficient states of problem b")
        n_new = int(Xnew.shape[0])
        if prob is None and cls is None:
            if isinstance(Xnew, np.ndarray):
                prob, cls = np.empty((n_new, K), np.float64), np.empty(n_new, np.int32)
            else:
                import torch
                prob = torch.empty((n_new, K), dtype=torch.float64, device=Xnew.device)
                cls = torch.empty(n_new, dtype=torch.int32, device=Xnew.device)
        _check(lib().hmc_predict(self._h, int(b), _ptr(draws), int(ndraws), _ptr(Xnew), _x_in_dtype(Xnew), n_new,
                                 _ptr(prob), _ptr(cls)))
        return prob, cls

    def get_state(self, chains, beta=None, grad=None, logpost=None):
        nxt = ctypes.c_int64(0)
        _check(lib().hmc_get_state(self._h, chains, _ptr(beta), _ptr(grad), _ptr(logpost), ctypes.byref(nxt)))
        return nxt.value

    def save_state(self, path):
        """Checkpoint the chain state (beta, grad, log K, next iteration) to `path`."""
        _check(lib().hmc_state_save(self._h, os.fsencode(path)))

    def load_state(self, path):
        """Resume from a checkpoint written by save_state for the same problems."""
        _check(lib().hmc_state_load(self._h, os.fsencode(path)))

    def get_x(self, b=0):
        """X of problem b as stored on the device (raw element bits) and the FP8 scales."""
        n, p, _ = self.shapes[b]
        xt = self._x_storage
        dt = {F64: np.float64, F32: np.float32, BF16: np.uint16, FP8E4M3: np.uint8}[xt]
        out = np.empty((n, p), dtype=dt)
        sc = np.empty(p, dtype=np.float32) if xt == FP8E4M3 else None
        _check(lib().hmc_get_x(self._h, b, _ptr(out), _ptr(sc)))
        return out, sc

    def set_timing(self, on, every=1):
        """Time the fused launches with CUDA events (every `every`-th launch)."""
        _check(lib().hmc_set_timing(self._h, (max(1, int(every)) if on else 0)))

    def fused_kernel_time(self):
        ms = ctypes.c_double(0)
        n = ctypes.c_int64(0)
        _check(lib().hmc_fused_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def first_pass_time(self):
        """Two-pass engine: milliseconds of the timed launches spent in the first pass."""
        ms = ctypes.c_double(0)
        _check(lib().hmc_first_pass_time(self._h, ctypes.byref(ms)))
        return ms.value

    # -- helpers
    def _chains_of(self, beta, chains):
        if chains is not None:
            return int(chains)
        numel = beta.numel() if hasattr(beta, "numel") else beta.size
        c, r = divmod(numel, self.chain_size)
        if r or c < 1:
            raise ValueError(f"beta has {numel} elements, not a multiple of the chain size {self.chain_size}")
        return c

    def _alloc_like(self, beta, chains, logpost, grad):
        if isinstance(beta, np.ndarray):
            if logpost is None:
                logpost = np.empty(self.nprob * chains, dtype=np.float64)
            if grad is None:
                grad = np.empty_like(beta)
        else:
            import torch
            if logpost is None:
                logpost = torch.empty(self.nprob * chains, dtype=torch.float64, device=beta.device)
            if grad is None:
                grad = torch.empty_like(beta)
        return logpost, grad


def create(X, y, K, prior="gaussian", prior_scale=1.0, x_storage="f32", state="f32", max_chains=1, engine=0,
           spin_limit=0, stream=None, tile=None, layout="free"):
    """Upload one problem (X: float32/float64 n x p, host numpy or device tensor; y: int32).
    ``layout``: "free" (K-1 rows per chain), "masked" (K rows, row K held at zero) or
    "unconstrained" (K free rows)."""
    o = _make_opts(x_storage, state, max_chains, engine, spin_limit, stream, tile, layout)
    n, p = int(X.shape[0]), int(X.shape[1])
    h = ctypes.c_void_p()
    _check(lib().hmc_create(_ptr(X), _x_in_dtype(X), _ptr(y), n, p, int(K), PRIORS[prior], float(prior_scale),
                            ctypes.byref(o), ctypes.byref(h)))
    hd = Handle(h.value, None, [(n, p, int(K))], o.state, int(max_chains), o.layout)
    hd._x_storage = o.x_storage
    return hd


def create_batch(Xs, ys, Ks, prior="gaussian", prior_scale=1.0, x_storage="f32", state="f32", max_chains=1,
                 engine=0, spin_limit=0, stream=None, tile=None, layout="free"):
    """Upload several independent problems into one handle."""
    o = _make_opts(x_storage, state, max_chains, engine, spin_limit, stream, tile, layout)
    m = len(Xs)
    xin = {_x_in_dtype(X) for X in Xs}
    if len(xin) != 1:
        raise TypeError("all X of a batch must share one dtype")
    Xp = (ctypes.c_void_p * m)(*[_ptr(X) for X in Xs])
    yp = (ctypes.c_void_p * m)(*[_ptr(y) for y in ys])
    ns = (ctypes.c_int64 * m)(*[int(X.shape[0]) for X in Xs])
    ps = (ctypes.c_int64 * m)(*[int(X.shape[1]) for X in Xs])
    ks = (ctypes.c_int32 * m)(*[int(k) for k in Ks])
    h = ctypes.c_void_p()
    _check(lib().hmc_create_batch(m, Xp, xin.pop(), yp, ns, ps, ks, PRIORS[prior], float(prior_scale),
                                  ctypes.byref(o), ctypes.byref(h)))
    hd = Handle(h.value, None, [(int(X.shape[0]), int(X.shape[1]), int(k)) for X, k in zip(Xs, Ks)], o.state,
                int(max_chains), o.layout)
    hd._x_storage = o.x_storage
    return hd


def annealing_temperatures(iters, t0=1.0e3, r=0.9):
    """Acceptance temperatures of the annealed burn-in of Sec. 3.2 for `iters`
    iterations (hmc_annealing_schedule); pass the result as ``temps`` to
    ``Handle.sample``."""
    out = np.empty(int(iters), dtype=np.float64)
    _check(lib().hmc_annealing_schedule(float(t0), float(r), int(iters), out.ctypes.data if out.size else None))
    return out


def header_functions(path=None):
    """Names of the functions declared in include/hmc.h."""
    import re
    path = path or os.path.join(HERE, "..", "include", "hmc.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hmc_[a-z_0-9]+)\s*\(", text)))
