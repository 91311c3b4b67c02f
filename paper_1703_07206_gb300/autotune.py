"""Launch-shape autotuner for libsgml grids.

Times a few cycles of the grid's own problem(s) for each candidate launch shape -- the column-tile
shape of the tiled phases (32 x 16 or 64 x 8), the z-slab height of the work partition (``slab_z``),
CTAs per SM, work pieces per CTA (``z_waves``) and
launch mode (one persistent cooperative launch per call, or one launch per phase) -- keeps the fastest, and caches the choice in a JSON file keyed by the problem
configuration (dimension, precision, level counts, device).  Results do not depend on the launch
shape, only the time does.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

from . import sgml

DEFAULT_CANDIDATES = [
    {"ctas_per_sm": 0, "z_waves": 1, "mode": 0, "tile_x": 64, "slab_z": 32},
    {"ctas_per_sm": 0, "z_waves": 1, "mode": 0, "tile_x": 64, "slab_z": 16},
    {"ctas_per_sm": 0, "z_waves": 1, "mode": 0, "tile_x": 64, "slab_z": 0},
    {"ctas_per_sm": 0, "z_waves": 1, "mode": 0, "tile_x": 32, "slab_z": 16},
    {"ctas_per_sm": 0, "z_waves": 2, "mode": 0, "tile_x": 64, "slab_z": 0},
    {"ctas_per_sm": 1, "z_waves": 1, "mode": 0, "tile_x": 64, "slab_z": 16},
    {"ctas_per_sm": 0, "z_waves": 1, "mode": 1, "tile_x": 64, "slab_z": 16},
]

CACHE = os.environ.get("SGML_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "sgml_autotune.json"))


def config_key(grid, device_name: str) -> str:
    sig = f"{grid.dim}|{grid.precision}|{','.join(map(str, grid.n_levels))}|{device_name}"
    return hashlib.sha1(sig.encode()).hexdigest()[:16]


def _time_cycles(grid, cycles):
    import torch
    torch.cuda.synchronize()
    grid.run_cycle(1)  # warm-up (and table rebuild after set_launch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grid.run_cycle(cycles)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / cycles


def tune(grid, candidates=None, cycles=3, cache_path: str | None = CACHE, use_cache=True):
    """Pick the fastest launch shape for `grid` (whose problems are already set), apply it and return
    {"choice": ..., "ms_per_cycle": {...}, "cached": bool}.  The grid's solution is advanced by the
    timing runs; call before sgml_solve_to_tol (which restarts from the boundary values)."""
    import torch
    key = config_key(grid, torch.cuda.get_device_name())
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        choice = cache[key]["choice"]
        grid.set_launch(**choice)
        return {"choice": choice, "ms_per_cycle": cache[key].get("ms_per_cycle", {}), "cached": True}
    times = {}
    for cand in candidates or DEFAULT_CANDIDATES:
        grid.set_launch(**cand)
        times[json.dumps(cand, sort_keys=True)] = _time_cycles(grid, cycles) * 1e3
    best = min(times, key=times.get)
    choice = json.loads(best)
    grid.set_launch(**choice)
    cache[key] = {"choice": choice, "ms_per_cycle": times}
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return {"choice": choice, "ms_per_cycle": times, "cached": False}
