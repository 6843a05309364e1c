"""Autotuner for batched generation.

Chooses the work-item tile (edges per claimed item) and the number of
resident CTAs of the persistent batch kernel by timing the candidates on the
device with CUDA events, and caches the winner in a JSON file keyed by the
GPU and a signature of the job mix (kinds and size classes), so a later
process with a similar batch reuses it without timing.
"""
from __future__ import annotations

import json
import math
import os

TILE_CANDIDATES = (1024, 2048, 4096, 8192)
GRID_FRACTIONS = (1.0, 0.5)


def cache_path() -> str:
    base = os.environ.get("PGEN_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache",
                                                            "pgen")
    return os.path.join(base, "autotune.json")


def signature(jobs) -> str:
    """Job mix signature: per kind, counts in log2 size classes."""
    hist = {}
    for j in jobs:
        edges = j["n"] * j["m"] if j["kind"] == "pba" else j["n_edges"]
        cls = int(math.log2(max(edges, 1))) // 2 * 2
        key = f"{j['kind']}:{cls}"
        hist[key] = hist.get(key, 0) + 1
    return ",".join(f"{k}={hist[k]}" for k in sorted(hist))


def _load():
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(db):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(db, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_batch(jobs, id64: bool = False, reps: int = 2, use_cache: bool = True,
               tiles=TILE_CANDIDATES, fractions=GRID_FRACTIONS):
    """Return dict(tile_edges=..., grid_ctas=..., ms=...) for this job mix."""
    import torch

    import paper_1003_3684_gb300 as pg

    dev = torch.cuda.get_device_properties(torch.cuda.current_device())
    key = f"{dev.name}|{dev.multi_processor_count}|{'64' if id64 else '32'}|{signature(jobs)}"
    db = _load() if use_cache else {}
    if key in db:
        return dict(db[key], cached=True)
    best = None
    arena = None
    ws = torch.empty(pg.pg_batch_workspace_size(), dtype=torch.uint8, device="cuda")
    full = 0
    for tile in tiles:
        plan = pg.BatchPlan(jobs, tile_edges=tile, id64=id64)
        if arena is None:
            arena = torch.empty((max(plan.total_edges, 1), 2),
                                dtype=torch.int64 if id64 else torch.int32, device="cuda")
        if not full:
            full = dev.multi_processor_count * 4
        for frac in fractions:
            grid = 0 if frac == 1.0 else max(1, int(full * frac))
            pg.gen_batch(plan, arena=arena, workspace=ws, grid_ctas=grid)   # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                pg.gen_batch(plan, arena=arena, workspace=ws, grid_ctas=grid)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            if best is None or ms < best["ms"]:
                best = dict(tile_edges=tile, grid_ctas=grid, ms=ms)
    if use_cache:
        db = _load()
        db[key] = best
        _store(db)
    return dict(best, cached=False)
