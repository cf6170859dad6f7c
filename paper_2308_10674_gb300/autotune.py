"""Autotuner for the engine's launch-side choices on a given GPU and scan.

For each candidate configuration -- the step kernel's tile shape (CTAs per
frame, where more than one shape is built: 1, 2 or 4 at 128^2), the batch
size of a mini-batch scan, and graph replay of sweeps on or off -- it builds
a throw-away engine on the scan's own frames, runs one untimed sweep, times
the next ones with the engine's CUDA events and keeps the fastest.  The batch
size is part of the reconstruction (mini-batch ePIE averages over a batch),
so it is tuned only where the caller leaves it open; the tile shape and
graph replay change the schedule, not the result.  Results are cached per
(GPU, frame side, frame count, mode, candidates) in a JSON file.
"""
from __future__ import annotations

import json
import os

from . import _binding as B

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json")

# tile shapes (CTAs per frame) built per frame side; 0 = the default
TILES = {128: (1, 2, 4)}


def _gpu_name(device):
    try:
        import torch
        return torch.cuda.get_device_name(device)
    except Exception:
        return f"cuda:{device}"


def tune(d, mode=B.EPIE_MINIBATCH, batches=(64, 128, 256, 512, 1024), graph=(True, False),
         tiles=None, intensity_dtype=B.EPIE_U16, sweeps=2, device=0, cache=True,
         cache_path=None):
    """d: a scan dict from synth (N, H, W, P0, frames, pos, dark).  Returns
    (best, table) with best = {"batch": B, "graph": bool, "ctas_per_frame": T}
    and table the measured frame-updates/s per candidate."""
    tiles = tuple(tiles) if tiles is not None else TILES.get(int(d["N"]), (0,))
    path = cache_path or CACHE
    key = json.dumps([_gpu_name(device), int(d["N"]), int(len(d["pos"])), int(mode),
                      list(batches), list(graph), list(tiles), int(intensity_dtype)])
    store = {}
    if cache and os.path.exists(path):
        try:
            with open(path) as f:
                store = json.load(f)
        except (OSError, ValueError):
            store = {}
    if key in store:
        return store[key]["best"], store[key]["table"]
    cands = [(t, b, g) for t in tiles
             for b in (batches if mode == B.EPIE_MINIBATCH else (0,)) for g in graph]
    table, best, best_rate = {}, None, -1.0
    for t, b, g in cands:
        with B.Engine(d["N"], d["H"], d["W"], d["P0"], None, capacity=len(d["pos"]), mode=mode,
                      batch=max(b, 1), device=device, intensity_dtype=intensity_dtype,
                      flags=B.EPIE_GRAPH if g else 0, ctas_per_frame=t) as eng:
            if d.get("dark") is not None:
                eng.set_dark(d["dark"])
            eng.append(d["frames"], d["pos"])
            eng.iterate(1)
            eng.iterate(sweeps)
            ms, _ = eng.last_timing()
        rate = len(d["pos"]) * sweeps / (ms / 1e3)
        table[f"tile={t},batch={b},graph={int(g)}"] = rate
        if rate > best_rate:
            best_rate, best = rate, {"batch": b, "graph": bool(g), "ctas_per_frame": t}
    if cache:
        store[key] = {"best": best, "table": table}
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(store, f, indent=1)
        os.replace(tmp, path)
    return best, table
