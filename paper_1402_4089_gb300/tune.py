"""Tile autotuner for the fused log-posterior + gradient pass.

The library picks a tile (cluster size S, ring slots) from an occupancy model;
this module measures instead.  For one problem shape it creates a handle per
candidate tile, times the fused pass with the library's own CUDA-event timer
(events on the handle's stream around each fused launch) and keeps the
fastest.  Results are cached per device and problem shape in a JSON file
(``HMC_TUNE_CACHE``, default ``~/.cache/paper_1402_4089_gb300/tune.json``).

The figure of merit is the fused-kernel time of one call for all chains (a
tile that fits fewer chains per launch pays for more launches).

Candidates: CUDA-core engine, S in {1, 2, 3, 4, 5, 6, 8, 10, 12, 16} x ring
slots {2, 3, 4}; fused tensor-core engine (BF16 or FP8 X), S in {16, 8, 4, 2,
1} x ring slots {2, 3, 4}; two-pass tensor-core engine (BF16 or FP8 X) and two-pass
CUDA-core engine (FP32 / FP64 X), whose plans the library derives from the
shape (one candidate each).  With engine 0 every engine the
storage type allows is a candidate.  Tiles the library rejects for the shape
are skipped.
"""
import json
import os

import numpy as np

from . import hmc

SIMT_S = (1, 2, 3, 4, 5, 6, 8, 10, 12, 16)
TC_S = (16, 8, 4, 2, 1)
RING = (2, 3, 4)


def _cache_path():
    p = os.environ.get("HMC_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1402_4089_gb300", "tune.json")


def _key(device_name, n, p, K, x_storage, state, chains, engine):
    return f"{device_name}|n={n}|p={p}|K={K}|x={x_storage}|st={state}|chains={chains}|engine={engine}"


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    p = _cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1)
        os.replace(tmp, p)
    except OSError:
        pass


def time_tile(X, y, K, prior, prior_scale, x_storage, state, chains, engine, tile, stream=None, reps=5, warmup=2,
              layout="free"):
    """Median time (us) of the fused launches of one log-posterior + gradient call for all
    `chains` (a tile may split the chains into several launches), or None if the library
    rejects the tile."""
    import torch
    try:
        h = hmc.create(X, y, K, prior, prior_scale, x_storage=x_storage, state=state, max_chains=chains,
                       engine=engine, stream=stream, tile=tile, layout=layout)
    except hmc.HmcError:
        return None, None
    try:
        d = h.describe()
        dev = torch.device("cuda", torch.cuda.current_device())
        p = int(X.shape[1])
        beta = torch.zeros((chains, h.rows(), p), dtype=h.torch_dtype(), device=dev)
        for _ in range(warmup):
            h.logpost_grad(beta)
        times = []
        for _ in range(reps):
            h.set_timing(True)          # resets the accumulated time
            h.logpost_grad(beta)
            torch.cuda.synchronize()
            ms, _ = h.fused_kernel_time()
            times.append(ms * 1e3)
        h.set_timing(False)
        return float(np.median(times)), d
    finally:
        h.close()


def autotune(X, y, K, prior="gaussian", prior_scale=1.0, x_storage="f32", state="f32", chains=1, engine=0,
             stream=None, reps=5, use_cache=True, verbose=False, layout="free"):
    """Fastest (engine, tile) for this problem: returns (engine, tile tuple for hmc.create, table of
    measurements); (engine, None, table) when no explicit tile runs."""
    import torch
    n, p = int(X.shape[0]), int(X.shape[1])
    if engine:
        engines = (engine,)
    else:
        engines = {"bf16": (2, 3, 1), "fp8": (3, 2, 1)}.get(x_storage, (1, 4))
    key = _key(torch.cuda.get_device_name(), n, p, K, x_storage, state, chains, engine) + \
        ("" if layout == "free" else f"|layout={layout}")
    cache = _load() if use_cache else {}
    if key in cache:
        e = cache[key]
        return int(e["engine"]), tuple(e["tile"]), e.get("table", [])
    table = []
    for eng in engines:
        cands = [(0, 0)] if eng in (3, 4) else [(S, ns) for S in (TC_S if eng == 2 else SIMT_S) for ns in RING]
        for S, ns in cands:
            us, d = time_tile(X, y, K, prior, prior_scale, x_storage, state, chains, eng, (S, 0, 0, ns),
                              stream=stream, reps=reps, layout=layout)
            if us is None:
                continue
            pr = d["problems"][0]
            row = dict(engine=eng, S=S, ring=ns, us=round(us, 2), clusters=pr.get("nclusters"),
                       group_chains=pr.get("group_chains"), smem=pr.get("smem"))
            table.append(row)
            if verbose:
                print("tune", json.dumps(row), flush=True)
    if not table:
        # No explicit tile runs for this shape: leave the choice to the library.
        return engine, None, table
    best = min(table, key=lambda r: r["us"])
    tile = (best["S"], 0, 0, best["ring"])
    if use_cache:
        cache = _load()
        cache[key] = dict(engine=best["engine"], tile=list(tile), table=table)
        _store(cache)
    return best["engine"], tile, table
