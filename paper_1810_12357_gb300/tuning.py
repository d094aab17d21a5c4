"""Persisted choices of the row-tile tuner (ehc_tuning / ehc_batch_tuning).

The library times the row-tile kernel's two widths and three persistent grid
sizes at the first long substep call of a context and keeps the fastest (every
choice gives the same results).  This module keeps those choices in a JSON file
keyed by the GPU's name and a shape class of the system (atom count and rows of
cells, on a log2 scale, and the number of replicas), so that later contexts of
the same shape start with the tuned choice instead of timing again.  The file is
$EHC_TUNE_CACHE, or ~/.cache/ehc/tuning.json.
"""
from __future__ import annotations

import json
import math
import os


def cache_path() -> str:
    return os.environ.get("EHC_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "ehc",
                                                              "tuning.json")


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def shape_class(n_atoms: int, box, rc: float, skin: float = 0.0, replicas: int = 1) -> str:
    """Atom count and rows of cells (cells at least rc + |skin| wide) on a log2
    scale, and the number of replicas."""
    w = rc + abs(skin)
    rows = max(1, int(box[1] // w)) * max(1, int(box[2] // w))
    return f"n{round(2 * math.log2(max(n_atoms, 1))) / 2:g}_rows{round(math.log2(rows))}_rep{int(replicas)}"


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(key: str):
    """(tile_threads, grid_quarters) stored for this GPU and shape, or None."""
    e = _load(cache_path()).get(gpu_name(), {}).get(key)
    if not e:
        return None
    return int(e["tile_threads"]), int(e["grid_quarters"])


def store(key: str, tile_threads: int, grid_quarters: int) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    d = _load(path)
    d.setdefault(gpu_name(), {})[key] = {"tile_threads": int(tile_threads), "grid_quarters": int(grid_quarters)}
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
