"""Tile-shape autotuner of the voxelizer.

The voxelizer's tile is 8 x 16 x depth voxels with depth 8, 16 or 32
(dgr_set_tile_depth).  Deeper tiles share each lane's per-Gaussian set-up
over more z-voxels; shallower tiles give more CTAs to small grids.  The best
depth depends on the grid size and on the Gaussian scale law, so it is
measured: `tune(key, run)` times `run()` under each depth (CUDA events, after
a warm-up) and caches the winner in a JSON table keyed by `key`
(e.g. "grid=256x256x256/n=50000/scale=loguniform:0.5-6").  `run` must build
its workspace from the current depth (plans depend on it).
"""
from __future__ import annotations

import json
import os

import torch

from . import dgr

DEPTHS = (8, 16, 32)


def table_path() -> str:
    base = os.environ.get("DGR_AUTOTUNE_CACHE") or os.path.join(
        os.environ.get("XDG_CACHE_HOME", os.path.expanduser("~/.cache")), "dgr_b300")
    return os.path.join(base, "tile_depth.json")


def load_table() -> dict:
    try:
        with open(table_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def save_table(tab: dict):
    path = table_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(tab, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_ms(run, reps: int = 3) -> float:
    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(key: str, make_run, reps: int = 3, use_cache: bool = True) -> int:
    """make_run() -> run (a callable doing the work with a workspace planned for
    the current depth).  Returns the chosen depth and leaves it set."""
    tab = load_table() if use_cache else {}
    if key in tab:
        dgr.dgr_set_tile_depth(int(tab[key]["depth"]))
        return int(tab[key]["depth"])
    times = {}
    for d in DEPTHS:
        dgr.dgr_set_tile_depth(d)
        run = make_run()
        times[d] = time_ms(run, reps)
        del run
    best = min(times, key=times.get)
    dgr.dgr_set_tile_depth(best)
    if use_cache:
        tab = load_table()
        tab[key] = {"depth": best, "ms": {str(k): round(v, 4) for k, v in times.items()}}
        save_table(tab)
    return best
