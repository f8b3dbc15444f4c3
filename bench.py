#!/usr/bin/env python
"""Benchmark of the HMC hot path on GB300: prints ONE JSON line.

A step is one HMC iteration over the synthetic workload: momentum draw, L
leapfrog updates (each one gradient evaluation of every chain -- the fused
pass, or the two passes of the two-pass engine, over X -- then the
fixed-order split-K reduction and the leapfrog update), the Metropolis test
and the keep/restore select -- all on the device, replayed from one CUDA
graph.  The default workload is the largest configuration: n = 1e5, p = 2e4,
K = 10, 8 chains, X in BF16 (4 GB), L = 100.  ``value`` is gradient
evaluations per second (chains * L per step) with X resident in HBM; ``e2e``
is the same metric through the C ABI with host buffers (the chain state
uploaded and the sample read back every step); ``roofline`` is the dominant
kernel's algorithmic bytes per launch over its duration against the measured
HBM copy bandwidth (``gradient_roofline``: one gradient against X read once);
``cpu_baseline`` is the FP64 oracle on the host cores on a bounded sample of
the same workload; ``ess`` compares ESS/s of FP32 single-chain and BF16
multi-chain sampling from stationary chains at equal posterior accuracy.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload autodiff|precision|batched|highdim_fp32|plain_fp64|mnist_shaped|
                                batched_uneven|sweep]
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gradient evals/s"
UNIT = "grad_evals/s"
XBYTES = {"f64": 8, "f32": 4, "bf16": 2, "fp8": 1}
# Sources of each engine's fused kernel: a recorded DRAM-traffic figure is used
# only while these files are unchanged since the ncu capture.
KERNEL_SOURCES = {
    "simt": ["paper_1402_4089_gb300/csrc/lpg_simt.cuh", "paper_1402_4089_gb300/csrc/device_common.cuh"],
    "tcgen05": ["paper_1402_4089_gb300/csrc/lpg_tc.cu", "paper_1402_4089_gb300/csrc/tc_common.cuh",
                "paper_1402_4089_gb300/csrc/device_common.cuh"],
    "tcgen05_2pass": ["paper_1402_4089_gb300/csrc/lpg_tc2.cu", "paper_1402_4089_gb300/csrc/tc_common.cuh",
                      "paper_1402_4089_gb300/csrc/device_common.cuh"],
    "simt_2pass": ["paper_1402_4089_gb300/csrc/lpg_simt2.cu", "paper_1402_4089_gb300/csrc/device_common.cuh"],
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="autodiff",
                    help="autodiff (default: n=1e5 p=2e4 K=10, 8 chains, BF16 X), precision, batched, highdim_fp32, "
                         "plain_fp64, mnist_shaped, batched_uneven, sweep")
    ap.add_argument("--engine", type=int, default=0, help="library engine (0 auto, 1 CUDA cores, 2 fused tcgen05, "
                                                           "3 two-pass tcgen05, 4 two-pass CUDA cores)")
    ap.add_argument("--xdtype", default=None, help="override the workload's X storage (f32, bf16, fp8, f64)")
    ap.add_argument("--chains", type=int, default=None)
    ap.add_argument("--L", type=int, default=None)
    ap.add_argument("--tile", default=None, help="S,BM,NT,NSTAGE override")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-autotune", action="store_true", help="use the library's tile choice instead of measuring")
    ap.add_argument("--ess-iters", type=int, default=1000, help="timed HMC iterations of each ESS/s run (0: skip)")
    ap.add_argument("--ess-burn", type=int, default=1000, help="untimed burn-in iterations before each ESS/s run")
    ap.add_argument("--ess-chains", type=int, default=8, help="chains of the BF16 multi-chain ESS/s run")
    ap.add_argument("--ess-coords", type=int, default=4000, help="coordinates (seeded subset) of the ESS estimates")
    ap.add_argument("--sweep-limit", type=int, default=0, help="sweep workload: first k shapes only (0: all 224)")
    ap.add_argument("--sweep-oracle-np", type=float, default=2e7,
                    help="sweep workload: time the oracle only where N p is at most this")
    return ap.parse_args()


def workload_spec(args):
    from paper_1402_4089_gb300 import synthetic
    spec = dict(synthetic.WORKLOADS[args.workload])
    if args.xdtype:
        spec["xdtype"] = args.xdtype
    if args.chains:
        spec["chains"] = args.chains
    if args.L:
        spec["L"] = args.L
    return spec


DATA_TEXT = {"mnist_shaped": "synthetic (seeded; 60000 x 785 design of pixel-like grey levels with an intercept "
                             "column, labels from the softmax model: the shape of the Sec. 3.2 run, no image data)"}


def prior_text(prior):
    kind, scale = prior
    return f"N(0,{scale}^2)" if kind == "gaussian" else f"Cauchy(0,{scale})"


def config_of(args, spec, xbytes_total):
    anneal = (f" annealed burn-in T0={spec['t0']:g} r={spec['r']} over {spec['burn_in']} its"
              if "burn_in" in spec else "")
    return {
        "workload": f"{args.workload}: n={spec['n']} p={spec['p']} K={spec['K']} chains={spec['chains']} "
                    f"L={spec['L']} eps={spec['eps']} prior={prior_text(spec['prior'])} X={spec['xdtype']}{anneal}",
        "n": spec["n"], "p": spec["p"], "K": spec["K"], "chains": spec["chains"], "L": spec["L"],
        "eps": spec["eps"], "x_storage": spec["xdtype"],
        "l2": f"inputs larger than L2: X is {xbytes_total / 1e6:.0f} MB > 129 MB L2, re-streamed every gradient"
        if xbytes_total > 129e6 else "X smaller than L2 (129 MB): no flush between steps",
        "step": "one HMC iteration: momentum draw, L fused gradient passes + split-K reduce/leapfrog, accept, select",
    }


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid, enabled=True):
        self.uuid = uuid
        self.enabled = enabled
        self.proc = None
        self.path = None

    def __enter__(self):
        if not self.enabled:
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", self.uuid, "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.enabled or self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value, dist, device):
    """The largest `value` over all ranks (every rank gets it); `value` itself
    when not distributed."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------ measurements
def measured_peaks():
    """(HBM GB/s, sustained BF16 TFLOP/s, source) from MEASURED_PEAKS.json, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops_sustained", 1700.0)), "measured"
    return 6800.0, 1700.0, "fallback"


def code_only(text):
    """C++/CUDA source without comments and blank lines (string literals kept), so a
    comment edit does not count as a kernel change."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(ln.rstrip() for ln in "".join(out).splitlines() if ln.strip())


def kernel_source_hash(engine, read=None):
    """Hash of the code (comments stripped) of an engine's kernel sources; `read`
    maps a repository path to its text (default: the working tree)."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[engine]:
        if read is None:
            with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
                text = f.read()
        else:
            text = read(rel)
        h.update(code_only(text).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload, xdt, engine, kernel=None):
    """DRAM bytes per launch from a committed ncu summary of this workload and X
    storage (and, for the two-pass engine, kernel), if it was taken on the current
    kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{workload}:{xdt}" + (f":{kernel}" if kernel else ""))
    if not e or e.get("engine") != engine or e.get("source_sha") != kernel_source_hash(engine):
        return None
    return e.get("bytes_per_launch")


def blas_threads_default():
    """Threads the host BLAS may use: the CPUs this process may run on (the BLAS
    default), unless a thread-count variable limits it."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            cores = min(cores, int(os.environ[var]))
    return cores


def oracle_rate(X64, y, spec, seconds):
    """Oracle leapfrog steps (one FP64 gradient each) per second on the rows given."""
    from oracle import hmc as ohmc
    from oracle import model
    kind, scale = spec["prior"]
    K = spec["K"]
    rng = np.random.default_rng(0)
    beta = np.zeros((K - 1, X64.shape[1]))
    eta = rng.standard_normal(beta.shape)
    t0 = time.perf_counter()
    g = model.grad_log_kernel(X64, y, beta, kind, scale)
    t_one = time.perf_counter() - t0
    steps = max(1, int(seconds / max(t_one, 1e-6)))
    t0 = time.perf_counter()
    ohmc.leapfrog(X64, y, beta, eta, spec["eps"], steps, kind, scale, grad0=g)
    return steps, time.perf_counter() - t0


def sample_rows(n, p, spec, seconds):
    """Rows of the bounded CPU sample: all of them when an FP64 copy of X is at most
    2 GB, else a leading block sized for about `seconds` of oracle gradients."""
    if n * p * 8 <= 2e9:
        return n
    return int(min(n, max(500, 2e9 / (8 * p))))


def cpu_baseline(X, y, spec, seconds):
    """The FP64 oracle as it stands: leapfrog steps (one gradient each) on the host,
    over the leading rows of X when the whole workload is too large for a bounded
    sample (the oracle's cost is linear in the rows, so the rate is scaled by
    rows / n); plus the same with the host BLAS held to one thread (a subprocess)."""
    n, p = X.shape
    m = sample_rows(n, p, spec, seconds)
    X64 = np.asarray(X[:m], dtype=np.float64)
    steps, el = oracle_rate(X64, y[:m], spec, seconds)
    value = steps / el * m / n
    one = None
    try:
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = ("import json,sys,numpy as np;sys.path.insert(0,%r);import bench;from paper_1402_4089_gb300 import synthetic;"
                "X,y,_,spec=synthetic.make_workload(%r,n=%d);spec=dict(spec,**json.loads(%r));"
                "s,e=bench.oracle_rate(np.asarray(X,dtype=np.float64),y,spec,%f);print(s/e)"
                % (ROOT, spec["name"], min(m, 4000), json.dumps({"eps": spec["eps"]}), max(2.0, seconds / 3)))
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        if r.returncode == 0:
            one = float(r.stdout.strip().splitlines()[-1]) * min(m, 4000) / n
    except (subprocess.SubprocessError, ValueError, OSError):
        one = None
    rows = "all" if m == n else f"the first {m} of {n}"
    return {"value": value, "unit": UNIT, "cores": blas_threads_default(), "kind": "oracle",
            "value_1thread": one,
            "sample": f"{steps} FP64 leapfrog steps (one gradient each) over {rows} rows in {el:.1f} s, numpy/BLAS on "
                      f"the host with its default threads (= cores); rate scaled to the full {n} rows "
                      f"(linear in rows); value_1thread: the same on at most 4000 rows with BLAS held to 1 thread"}


def oracle_accuracy(h, X, y, spec, xdt, tdt, dev, chains_to_check):
    """Error of the GPU log K and gradient at the chains' current state against the
    FP64 oracle, evaluated in row blocks: on the X values the device stores
    (arithmetic error) and on the original X (total error)."""
    import torch
    from oracle import model, quant
    K, chains = spec["K"], spec["chains"]
    kind, scale = spec["prior"]
    n, p = X.shape
    beta = torch.empty((chains, K - 1, p), dtype=tdt, device=dev)
    h.get_state(chains, beta=beta)
    lp, g = h.logpost_grad(beta)
    torch.cuda.synchronize()
    bits, sc = h.get_x()
    B = max(1, int(2e8 // p))

    def stored(a):
        if xdt == "bf16":
            return quant.bf16_decode(bits[a:a + B])
        if xdt == "fp8":
            return quant.fp8_dequantize(bits[a:a + B], sc)
        return bits[a:a + B]

    bs = [beta[c].double().cpu().numpy() for c in chains_to_check]
    lk_s, g_s, _ = model.log_kernel_and_grad_by_rows(((stored(a), y[a:a + B]) for a in range(0, n, B)), bs, kind, scale)
    lk_t, g_t, _ = model.log_kernel_and_grad_by_rows(((X[a:a + B], y[a:a + B]) for a in range(0, n, B)), bs, kind, scale)
    out = {"chains": list(chains_to_check), "state": "after the timed iterations",
           "tol_grad": {"f64": 1e-11, "f32": 1e-5, "bf16": 1e-2, "fp8": 1e-2}[xdt]}
    for tag, lks, gs in (("stored_x", lk_s, g_s), ("original_x", lk_t, g_t)):
        el, eg, ee = [], [], []
        for i, c in enumerate(chains_to_check):
            gc = g[c].double().cpu().numpy()
            el.append(abs(float(lp[c]) - lks[i]) / max(1.0, abs(lks[i])))
            eg.append(float(np.linalg.norm(gc - gs[i]) / max(np.linalg.norm(gs[i]), 1e-300)))
            ee.append(float(np.abs(gc - gs[i]).max() / max(np.abs(gs[i]).max(), 1e-30)))
        out[tag] = {"logk_rel_err": max(el), "grad_rel_err": max(eg), "grad_elem_err": max(ee)}
    out["vs"] = ("stored_x: FP64 oracle on the X values the device stores (arithmetic error); original_x: on the FP32 "
                 "input X (total error, storage rounding included)")
    return out


def _mean_z(sa, sb):
    """|m_a - m_b| / sqrt(MCSE_a^2 + MCSE_b^2) per coordinate for draws [N, chains, coords]
    (MCSE = sd / sqrt(ESS), ESS as in the throughput report)."""
    from paper_1402_4089_gb300 import diagnostics
    out = []
    for s_ in (sa, sb):
        flat = s_.reshape(-1, s_.shape[2])
        out.append((flat.mean(axis=0), flat.std(axis=0) / np.sqrt(np.maximum(diagnostics.ess(s_), 1.0))))
    return np.abs(out[0][0] - out[1][0]) / np.sqrt(out[0][1] ** 2 + out[1][1] ** 2 + 1e-300)


def _zsum(z):
    return {"frac_above_3": round(float(np.mean(z > 3.0)), 4), "max_z": round(float(z.max()), 2)}


def ess_comparison(args, dev):
    """ESS/s of the FP32 single-chain CUDA-core path and of the BF16 multi-chain
    tensor-core path on the high-dimensional problem (n=1e4, p=5000, K=10), both
    from stationary chains: `ess_burn` iterations from beta = 0 (not timed), then
    `ess_iters` timed iterations whose draws are kept on the device.  ESS
    (Geyer, chains pooled) and MCSE on a seeded subset of coordinates; the two
    posteriors' means are compared per coordinate within 3 combined MCSE, next to
    two controls at one precision (the BF16 chains split in two groups, the FP32
    chain's first and second halves) that show how often the same criterion
    fails between runs of one sampler on this problem (the chains' mixing, not the
    precision), and the split-free R-hat of the BF16 chains."""
    import torch
    from paper_1402_4089_gb300 import diagnostics, hmc, synthetic
    X, y, _, spec = synthetic.make_workload("highdim_fp32")
    K, p, L, eps = spec["K"], spec["p"], spec["L"], spec["eps"]
    kind, scale = spec["prior"]
    rng = np.random.default_rng(7)
    coords = np.sort(rng.choice((K - 1) * p, size=min(args.ess_coords, (K - 1) * p), replace=False))
    idx = torch.from_numpy(coords).to(dev)
    runs = {}
    rhat = np.ones(1)
    for tag, xs, chains, engine in (("fp32_1chain", "f32", 1, 1), (f"bf16_{args.ess_chains}chains", "bf16", args.ess_chains, 0)):
        stream = torch.cuda.Stream(device=dev)
        h = hmc.create(X, y, K, kind, scale, x_storage=xs, max_chains=chains, engine=engine, stream=stream)
        h.sample(chains, L, eps, args.ess_burn, 11, beta0=torch.zeros((chains, K - 1, p), device=dev))
        draws = torch.empty((args.ess_iters, chains, K - 1, p), dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = h.sample(chains, L, eps, args.ess_iters, 12, samples=draws)
        e1.record(stream)
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        sub = draws.reshape(args.ess_iters, chains, -1)[:, :, idx].double().cpu().numpy()
        del draws
        e = diagnostics.ess(sub)
        if chains > 1:
            h2 = chains // 2
            ctrl = (f"{tag}: chains 0-{h2 - 1} against {h2}-{chains - 1}", _mean_z(sub[:, :h2], sub[:, h2:]))
            n_ = sub.shape[0]
            cm, cv = sub.mean(axis=0), sub.var(axis=0, ddof=1)
            W, B = cv.mean(axis=0), n_ * cm.var(axis=0, ddof=1)
            rhat = np.sqrt(((n_ - 1) / n_ * W + B / n_) / np.where(W > 0, W, 1.0))
        else:
            h2 = sub.shape[0] // 2
            ctrl = (f"{tag}: first {h2} draws against the last {sub.shape[0] - h2}", _mean_z(sub[:h2], sub[h2:]))
        flat = sub.reshape(-1, sub.shape[2])
        mean, sd = flat.mean(axis=0), flat.std(axis=0)
        runs[tag] = {"x_storage": xs, "chains": chains, "engine": h.describe()["engine"], "iters": args.ess_iters,
                     "burn_in": args.ess_burn, "seconds": round(secs, 3), "ess_min": round(float(e.min()), 2),
                     "ess_median": round(float(np.median(e)), 2), "ess_min_per_s": round(float(e.min()) / secs, 3),
                     "ess_median_per_s": round(float(np.median(e)) / secs, 3),
                     "accept_rate": round(sum(s["accepted"] for s in st) / max(1, sum(s["iterations"] for s in st)), 4),
                     "_m": mean, "_se": sd / np.sqrt(np.maximum(e, 1.0)), "_ctrl": ctrl}
        h.close()
    a, b = list(runs.values())
    z = np.abs(a["_m"] - b["_m"]) / np.sqrt(a["_se"] ** 2 + b["_se"] ** 2 + 1e-300)
    controls = {}
    for r in runs.values():
        controls[r["_ctrl"][0]] = _zsum(r["_ctrl"][1])
        del r["_m"], r["_se"], r["_ctrl"]
    tags = list(runs)
    return {"problem": "highdim_fp32: n=10000 p=5000 K=10, N(0,1) prior, L=100, eps=2e-3", "coords": int(coords.size),
            **runs,
            "ess_per_s_ratio_min": round(runs[tags[1]]["ess_min_per_s"] / max(runs[tags[0]]["ess_min_per_s"], 1e-12), 2),
            "ess_per_s_ratio_median": round(runs[tags[1]]["ess_median_per_s"] /
                                            max(runs[tags[0]]["ess_median_per_s"], 1e-12), 2),
            "equal_accuracy": {"criterion": "|m_a - m_b| <= 3 sqrt(MCSE_a^2 + MCSE_b^2) per coordinate; pass if at most "
                                            "1% of coordinates exceed it and none exceeds 5",
                               "frac_above_3": round(float(np.mean(z > 3.0)), 4), "max_z": round(float(z.max()), 2),
                               "pass": bool(np.mean(z > 3.0) <= 0.01 and z.max() <= 5.0),
                               "controls_same_precision": controls,
                               "bf16_rhat": {"median": round(float(np.median(rhat)), 3), "max": round(float(rhat.max()), 3)}}}


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    from paper_1402_4089_gb300 import build, hmc, synthetic, tune

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    build.build()

    spec = workload_spec(args)
    spec["name"] = args.workload
    X, y, btrue, _ = synthetic.make_workload(args.workload)
    n, p, K = spec["n"], spec["p"], spec["K"]
    chains, L, eps = spec["chains"], spec["L"], spec["eps"]
    kind, scale = spec["prior"]
    xdt = spec["xdtype"]
    state = "f64" if xdt == "f64" else "f32"
    tile = tuple(int(v) for v in args.tile.split(",")) if args.tile else None
    stream = torch.cuda.Stream(device=dev)
    Xin = X if xdt != "f64" else X.astype(np.float64)
    tile_source, tune_table = ("given", None) if tile else ("library", None)
    engine = args.engine
    big = n * p > 2e8
    if tile is None and not args.no_autotune and not engine and not big:
        with torch.cuda.stream(stream):
            t_eng, t_tile, tune_table = tune.autotune(Xin, y, K, kind, scale, x_storage=xdt, state=state,
                                                      chains=chains, stream=stream)
        if t_tile is not None:
            engine, tile, tile_source = t_eng, t_tile, "autotuned"
    elif big and tile is None and not args.no_autotune:
        tile_source = "library (autotune skipped: every candidate would upload the whole X again)"
    h = hmc.create(Xin, y, K, kind, scale, x_storage=xdt, state=state, max_chains=chains, stream=stream, tile=tile,
                   engine=engine)
    desc_all = h.describe()
    desc = desc_all["problems"][0]
    eng_name = desc_all["engine"]
    tdt = torch.float64 if state == "f64" else torch.float32
    seed = 20140217
    zeros = torch.zeros((chains, K - 1, p), dtype=tdt, device=dev)

    # annealed burn-in (Sec. 3.2): warm-up and timed iterations accept at the
    # schedule's temperatures, in order
    temps_w = temps_t = None
    if "burn_in" in spec:
        sched = hmc.annealing_temperatures(args.warmup + args.steps, spec["t0"], spec["r"])
        temps_w, temps_t = sched[:args.warmup], sched[args.warmup:]

    # warm-up (includes graph capture)
    h.sample(chains, L, eps, args.warmup, seed, beta0=zeros, temps=temps_w)
    torch.cuda.synchronize()

    # timed region: K iterations from the cached graph, CUDA events around every
    # 10th gradient evaluation (an event node per launch would slow the graph itself)
    h.set_timing(True, every=10)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    with Clocks(uuid, enabled=not args.no_clocks) as clk:
        ev0.record(stream)
        stats = h.sample(chains, L, eps, args.steps, seed, temps=temps_t)
        ev1.record(stream)
        torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    fused_ms, fused_n = h.fused_kernel_time()
    first_ms = h.first_pass_time()
    h.set_timing(False)
    elapsed = max_over_ranks(elapsed, dist, dev)
    grads = chains * L * args.steps
    value = world * grads / elapsed
    groups = -(-chains // desc["group_chains"])
    # traj_start + per leapfrog step (per chain group: [operand boxes +] the pass(es), then the
    # reduce/update) + select
    per_group = {"simt": 1, "tcgen05": 2, "tcgen05_2pass": 3, "simt_2pass": 2}[eng_name]
    launches_per_step = 1 + L * (groups * per_group + 1) + 1

    # rooflines: the gradient (X once) and the dominant kernel
    xb = XBYTES[xdt]
    c_launch = min(chains, desc["group_chains"]) * (K - 1)
    hbm_peak, tc_peak, peak_kind = measured_peaks()
    per_grad_s = (fused_ms / 1e3) / max(fused_n, 1)          # one gradient of the launch's chains
    x_bytes = n * p * xb
    grad_bytes = x_bytes + 4 * n + 8 * p * c_launch
    grad_flops = 4.0 * n * p * c_launch                       # two contractions, 2 n p C each
    if eng_name in ("tcgen05_2pass", "simt_2pass"):
        # residual bytes: BF16 operand boxes (tensor cores) or the state type (CUDA cores)
        rb = 2 if eng_name == "tcgen05_2pass" else XBYTES[state]
        ta = (first_ms / 1e3) / max(fused_n, 1)
        tb = per_grad_s - ta
        passes = {"A (logits, softmax, residual)": (ta, x_bytes + 4 * n + 4 * p * c_launch + rb * n * c_launch),
                  "B (X^T R)": (tb, x_bytes + rb * n * c_launch + 4 * p * c_launch)}
        dom = max(passes, key=lambda k: passes[k][0])
        t_dom, b_dom = passes[dom]
        if eng_name == "tcgen05_2pass":
            kernel = f"tc2::{'logits_kernel' if dom.startswith('A') else 'grad_kernel'} (tcgen05, pass {dom})"
        else:
            kernel = (f"simt2::{'logits_kernel + softmax_kernel' if dom.startswith('A') else 'grad_kernel'} "
                      f"(CUDA cores, pass {dom})")
        f_dom = 2.0 * n * p * c_launch
        traffic = recorded_traffic(args.workload, xdt, eng_name, "A" if dom.startswith("A") else "B")
        per_pass = {k: {"us": round(v[0] * 1e6, 2), "bytes": int(v[1]), "gbs": round(v[1] / v[0] / 1e9, 1),
                        "frac": round(v[1] / v[0] / 1e9 / hbm_peak, 4),
                        "tflops": round(2.0 * n * p * c_launch / v[0] / 1e12, 1)} for k, v in passes.items()}
    else:
        t_dom, b_dom, f_dom = per_grad_s, grad_bytes, grad_flops
        kernel = {"tcgen05": "lpg_tc_kernel (tcgen05)", "simt": "lpg_kernel (CUDA cores)"}[eng_name]
        traffic = recorded_traffic(args.workload, xdt, eng_name)
        per_pass = None
    achieved = b_dom / t_dom / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
            "kernel": kernel + f" X={xdt} C={c_launch}", "avg_launch_us": round(t_dom * 1e6, 2),
            "algorithmic_bytes": int(b_dom),
            "launches_timed": fused_n, "timed_launches_from": "every 10th gradient of the timed region",
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback 6.8 TB/s"}
    gradient = {"us": round(per_grad_s * 1e6, 2), "x_once_bytes": int(grad_bytes),
                "x_once_gbs": round(grad_bytes / per_grad_s / 1e9, 1),
                "x_once_frac": round(grad_bytes / per_grad_s / 1e9 / hbm_peak, 4),
                "note": "one gradient evaluation of the launch's chains against X read once from HBM (the per-gradient "
                        "HBM roofline)" + ("; the two-pass engine reads X twice when X exceeds L2" if per_pass else "")}
    tensor = None
    if xdt in ("bf16", "fp8"):
        tensor = {"achieved_tflops": round(f_dom / t_dom / 1e12, 2), "peak": tc_peak, "unit": "TFLOP/s",
                  "frac": round(f_dom / t_dom / 1e12 / tc_peak, 4),
                  "flops": "algorithmic 2 n p C per contraction (the two-term coefficient MMAs of the logits pass "
                           "issue twice that)", "peak_source": f"{peak_kind} bf16_tflops_sustained"}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        hb = torch.zeros((chains, K - 1, p), dtype=tdt).pin_memory()
        hs = torch.empty((1, chains, K - 1, p), dtype=tdt).pin_memory()
        hbn, hsn = hb.numpy(), hs.numpy()
        h.sample(chains, L, eps, 1, seed, beta0=hbn, samples=hsn)   # warm (graph for host samples)
        steps_e2e = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in range(steps_e2e):
            h.sample(chains, L, eps, 1, seed + 1 + t, beta0=hbn, samples=hsn)
            hbn[...] = hsn[0]
        e1.record(stream)
        torch.cuda.synchronize()
        el = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
        nbytes = chains * (K - 1) * p * (8 if state == "f64" else 4)
        e2e = {"value": round(world * chains * L * steps_e2e / el, 2), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes + chains * 40,
               "note": "per step: upload the chain state (pinned host), one HMC iteration from it (plus the "
                       "gradient at the uploaded state), read the sample back"}

    cpu, accuracy = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(X, y, spec, args.cpu_seconds)
        accuracy = oracle_accuracy(h, X, y, spec, xdt, tdt, dev, sorted({0, chains - 1}))
    acc = sum(s["accepted"] for s in stats) / max(1, sum(s["iterations"] for s in stats))
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": xdt,
        "data": DATA_TEXT.get(args.workload, "synthetic (seeded, shaped like the paper's high-dimensional multinomial "
                                             "setting; random-init coefficients)"),
        "config": config_of(args, spec, n * p * xb),
        "roofline": roof, "gradient_roofline": gradient, "passes": per_pass, "tensor": tensor,
        "cpu_baseline": cpu, "accuracy": accuracy, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
        "accept_rate": round(acc, 4), "impl": "ours", "clocks": clk.summary(), "engine": eng_name,
        "tile_source": tile_source, "tune": sorted(tune_table, key=lambda r: r["us"])[:6] if tune_table else None,
        "tile": {k: desc[k] for k in ("S", "BM", "CR", "NSTAGE", "PC", "nclusters", "group_chains", "smem",
                                      "pass_a", "pass_b") if k in desc},
    }
    h.close()
    del X, Xin
    if args.ess_iters > 0 and rank == 0:
        line["ess"] = ess_comparison(args, dev)
    if "burn_in" in spec:
        its = spec["iters"]
        line["paper_run"] = {
            "iterations": its, "estimated_s": round(elapsed / args.steps * its, 3),
            "note": f"{spec['burn_in']} annealed burn-in + {its - spec['burn_in']} sampling iterations at the "
                    f"measured ms_per_step (sampling at eps={spec['eps_sample']} costs the same per iteration); "
                    "context only: Sec. 3.2 reports 3 min 54 s for this run shape on real digit data on a Tesla K20"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------- many uneven problems, one launch
def run_batch_uneven(args):
    """The 32 independent regressions of the batching workload (n ~ U[500, 20000],
    p ~ U[100, 4000], K ~ U{3..20}, one chain each, BF16 X) as one batch handle:
    every fused pass covers all problems in one persistent launch."""
    import torch
    from paper_1402_4089_gb300 import build, hmc, synthetic

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    spec = dict(synthetic.WORKLOADS["batched"])
    xdt = args.xdtype or "bf16"
    L = args.L or spec["L"]
    eps, chains = spec["eps"], 1
    kind, scale = spec["prior"]
    shapes = synthetic.batched_shapes()
    probs = [synthetic.make_problem(n, p, K, seed=0, sub=100 + i) for i, (n, p, K) in enumerate(shapes)]
    stream = torch.cuda.Stream(device=dev)
    h = hmc.create_batch([pr[0] for pr in probs], [pr[1] for pr in probs], [K for (_, _, K) in shapes], kind, scale,
                         x_storage=xdt, max_chains=chains, stream=stream, engine=args.engine)
    desc = h.describe()
    seed = 20140217
    h.sample(chains, L, eps, args.warmup, seed)
    torch.cuda.synchronize()
    h.set_timing(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    with Clocks(uuid, enabled=not args.no_clocks) as clk:
        ev0.record(stream)
        stats = h.sample(chains, L, eps, args.steps, seed)
        ev1.record(stream)
        torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    fused_ms, fused_n = h.fused_kernel_time()
    h.set_timing(False)
    elapsed = max_over_ranks(elapsed, dist, dev)
    nprob = len(shapes)
    grads = nprob * chains * L * args.steps
    xb = XBYTES[xdt]
    alg = sum(n * p * xb + 4 * n + 8 * p * (K - 1) * chains for (n, p, K) in shapes)
    per_launch = (fused_ms / 1e3) / max(fused_n, 1)
    launches_per_grad = fused_n / max(1, L)          # timed launches: the last iteration
    peak, _, peak_kind = measured_peaks()
    achieved = alg / (per_launch * launches_per_grad) / 1e9
    line = {
        "metric": METRIC, "value": round(world * grads / elapsed, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": xdt,
        "data": "synthetic (seeded; 32 uneven multinomial regressions)",
        "config": {"workload": f"batched_uneven: {nprob} problems n~U[500,20000] p~U[100,4000] K~U{{3..20}}, "
                               f"1 chain each, L={L} eps={eps} X={xdt}, one fused launch per gradient step",
                   "total_x_bytes": sum(n * p * xb for (n, p, K) in shapes),
                   "l2": "inputs larger than L2: X of all problems re-streamed every gradient"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": recorded_traffic("batched_uneven", xdt, "tcgen05"),
                     "kernel": ({"tcgen05": "lpg_tc_kernel_batched (tcgen05), all problems per launch",
                                 "simt": "lpg_kernel_batched (CUDA cores), all problems per launch",
                                 "tcgen05_2pass": "tc2 passes A + B (tcgen05), one pair per problem"}.get(
                                     desc.get("engine"), desc.get("engine")) if desc.get("batched_launch") or
                                desc.get("engine") == "tcgen05_2pass" else f"{desc.get('engine')}, one launch per problem"),
                     "avg_launch_us": round(per_launch * 1e6, 2), "launches_timed": fused_n,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
        "cpu_baseline": None, "e2e": None, "gpu_launches": None,
        "accept_rate": round(sum(s["accepted"] for s in stats) / max(1, sum(s["iterations"] for s in stats)), 4),
        "impl": "ours", "clocks": clk.summary(), "batched_launch": desc.get("batched_launch"), "engine": desc.get("engine"),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# --------------------------------------------------------- Table 1 timing sweep
def run_sweep(args):
    """The timing sweep of Sec. 3.1 (Table 1): for each of the 224 (N, K, p)
    shapes, X and B iid N(0, 1e-3), one gradient evaluation and one leapfrog step
    (which includes its gradient: the update is fused into the gradient's
    reduction), each the mean of 5 runs timed with CUDA events; next to it the
    FP64 oracle's gradient on the host for shapes with N p <= --sweep-oracle-np
    (one run after a warm one).  Both halves of the paper's figures: the
    identifiable model (the free (K-1)-row block, equal to the masked p x K
    gradient of the Appendix; Figs 1-2) and the model without the
    identifiability constraint (K free rows; Figs 3-4).  Runs on one GPU (rank
    0; other ranks wait)."""
    import torch
    from paper_1402_4089_gb300 import build, hmc, synthetic

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    build.build()
    from oracle import model
    shapes = synthetic.sweep_shapes()
    if args.sweep_limit:
        shapes = shapes[:args.sweep_limit]
    stream = torch.cuda.Stream(device=dev)
    rows = []
    t_start = time.perf_counter()
    for layout in ("free", "unconstrained"):
        for (n, p, K) in shapes:
            X, y, B = synthetic.sweep_problem(n, p, K)
            if layout == "unconstrained":
                B = np.concatenate([B, np.zeros((1, p))])
            try:
                h = hmc.create(X, y, K, "cauchy", 1.0, x_storage="f32", max_chains=1, stream=stream, layout=layout)
            except hmc.HmcError as e:
                rows.append([layout, n, K, p, None, None, None, None, str(e)[:120], None])
                continue
            with torch.cuda.stream(stream):
                beta = torch.from_numpy(B.astype(np.float32)[None]).to(dev)
                lp, g = h.logpost_grad(beta)
                h.logpost_grad(beta, logpost=lp, grad=g)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(5):
                    h.logpost_grad(beta, logpost=lp, grad=g)
                e1.record(stream)
                b2 = beta.clone()
                eta = torch.zeros_like(b2)
                h.leapfrog(b2, eta, 1, 1e-3, grad=g, logpost=lp)
                e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e2.record(stream)
                for _ in range(5):
                    h.leapfrog(b2, eta, 1, 1e-3, grad=g, logpost=lp)
                e3.record(stream)
                stream.synchronize()
            g_us = e0.elapsed_time(e1) * 1e3 / 5
            lf_us = e2.elapsed_time(e3) * 1e3 / 5
            eng = h.describe()["engine"]
            h.close()
            cpu_us = None
            if n * p <= args.sweep_oracle_np:
                X64 = X.astype(np.float64)
                model.grad_log_kernel_layout(X64, y, B, "cauchy", 1.0, layout)
                t0 = time.perf_counter()
                model.grad_log_kernel_layout(X64, y, B, "cauchy", 1.0, layout)
                cpu_us = (time.perf_counter() - t0) * 1e6
            rows.append([layout, n, K, p, round(g_us, 2), round(lf_us, 2), None if cpu_us is None else round(cpu_us, 1),
                         None if cpu_us is None else round(cpu_us / g_us, 2), None, eng])
    wall = time.perf_counter() - t_start
    # The headline value uses the same shapes as the reference arm: identifiable
    # model, N p <= the oracle cap (where the GPU runs the shape).
    same = [1e6 / r[4] for r in rows if r[0] == "free" and r[4] is not None and r[1] * r[3] <= args.sweep_oracle_np]
    every = [1e6 / r[4] for r in rows if r[0] == "free" and r[4] is not None]
    sp = {lay: [r[7] for r in rows if r[0] == lay and r[7] is not None] for lay in ("free", "unconstrained")}
    big = [r for r in rows if r[0] == "free" and r[1] * r[3] >= 5000 * 5000 and r[4] is not None]
    line = {
        "metric": METRIC, "value": round(float(np.median(same)), 2) if same else None, "unit": UNIT, "n_gpus": 1,
        "steps": 5, "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; X and B iid N(0, 1e-3), labels from the model)",
        "config": {"workload": f"sweep: Table 1 grid, {len(shapes)} (N, K, p) shapes x 2 models (identifiable, "
                               f"unconstrained), 1 chain, Cauchy(0,1) prior, X=f32",
                   "value": "median over the identifiable-model shapes with N p <= oracle_np_cap (the reference "
                            "arm's shape set) of GPU gradient evaluations per second",
                   "oracle_np_cap": args.sweep_oracle_np},
        "impl": "ours", "gpu_launches": None, "cpu_baseline": None, "e2e": None, "roofline": None,
        "sweep": {"columns": ["model", "N", "K", "p", "gpu_grad_us", "gpu_leapfrog_step_us", "oracle_grad_us",
                              "speedup_grad", "unsupported", "engine"],
                  "rows": rows, "wall_s": round(wall, 1),
                  "value_all_shapes": round(float(np.median(every)), 2) if every else None,
                  "unsupported_shapes": sum(1 for r in rows if r[4] is None),
                  "engines": {e: sum(1 for r in rows if r[9] == e) for e in sorted({r[9] for r in rows if r[9]})},
                  "speedup_median": {k: (round(float(np.median(v)), 1) if v else None) for k, v in sp.items()},
                  "speedup_max": {k: (round(float(np.max(v)), 1) if v else None) for k, v in sp.items()},
                  "gpu_grad_us_median_large": round(float(np.median([r[4] for r in big])), 2) if big else None,
                  "note": "oracle: plain numpy FP64 (BLAS matmuls) on the host cores, one gradient after a warm one; "
                          "GPU: mean of 5 calls through the C ABI (fused pass + fixed-order reduction)"},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 oracle, timed as it stands on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import hmc as ohmc
    from oracle import model
    from paper_1402_4089_gb300 import synthetic

    if args.workload == "sweep":
        # the oracle's gradient over the Table 1 shapes it finishes quickly (N p <= cap)
        rates, used, t_all = [], 0, time.perf_counter()
        for (n, p, K) in synthetic.sweep_shapes()[:args.sweep_limit or None]:
            if n * p > args.sweep_oracle_np:
                continue
            X, y, B = synthetic.sweep_problem(n, p, K)
            X64 = X.astype(np.float64)
            model.grad_log_kernel(X64, y, B, "cauchy", 1.0)
            t0 = time.perf_counter()
            model.grad_log_kernel(X64, y, B, "cauchy", 1.0)
            rates.append(1.0 / (time.perf_counter() - t0))
            used += 1
        value = float(np.median(rates)) if rates else 0.0
        el = time.perf_counter() - t_all
        sample = (f"one FP64 gradient (after a warm one) at each of {used} Table 1 shapes with N p <= "
                  f"{args.sweep_oracle_np:g} (identifiable model: the product arm's headline shape set)")
        print(json.dumps({
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": used, "warmup": used, "ms_per_step": round(el / max(used, 1) * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"sweep: Table 1 grid, {used} shapes, 1 chain, Cauchy(0,1) prior",
                       "value": "median over shapes of oracle gradient evaluations per second"},
            "impl": "reference",
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}), flush=True)
        return

    spec = workload_spec(args)
    X, y, _, _ = synthetic.make_workload(args.workload)
    n, p = X.shape
    m = sample_rows(n, p, spec, 10.0)                        # rows the oracle runs on (all, or a leading block)
    X64 = np.asarray(X[:m], dtype=np.float64)
    ys = y[:m]
    del X
    kind, scale = spec["prior"]
    K = spec["K"]
    rng = np.random.default_rng(0)
    beta = np.zeros((K - 1, p))
    eta = rng.standard_normal(beta.shape)
    t0 = time.perf_counter()
    g = model.grad_log_kernel(X64, ys, beta, kind, scale)
    t_one = time.perf_counter() - t0
    budget = 150.0 / max(1, args.steps + args.warmup)        # whole run within a few minutes
    per_step = max(1, min(spec["L"], int(budget / max(t_one, 1e-6))))
    for _ in range(args.warmup):
        ohmc.leapfrog(X64, ys, beta, eta, spec["eps"], per_step, kind, scale, grad0=g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        beta, eta, _, g = ohmc.leapfrog(X64, ys, beta, eta, spec["eps"], per_step, kind, scale, grad0=g)
    el = time.perf_counter() - t0
    value = args.steps * per_step / el * m / n               # the oracle's cost is linear in the rows
    cores = blas_threads_default()
    rows = "all rows" if m == n else f"the first {m} of {n} rows (rate scaled by rows / n: the cost is linear in rows)"
    sample = (f"each step: {per_step} FP64 leapfrog steps (one gradient each) over {rows} "
              f"(a bounded sample of one {spec['L']}-step HMC iteration); numpy/BLAS, default threads")
    line = {
        "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args, spec, n * p * XBYTES[spec["xdtype"]]), "impl": "reference",
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched_uneven":
        run_batch_uneven(args)
    elif args.workload == "sweep":
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
