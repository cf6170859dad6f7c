"""Autotuner for the engine's launch-side choices on a given GPU and scan.

For each candidate configuration -- the batch size of a mini-batch scan and
graph replay of sweeps on or off -- it builds a throw-away engine on the
scan's own frames, runs one untimed sweep and times the next ones with the
engine's CUDA events, and keeps the fastest.  Note that the batch size is
part of the reconstruction (mini-batch ePIE averages over a batch), so it is
tuned only where the user leaves it open.  Results are cached per (GPU,
frame side, frame count, mode, candidates) in a JSON file.
"""
from __future__ import annotations

import json
import os

from . import _binding as B

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json")


def _gpu_name(device):
    try:
        import torch
        return torch.cuda.get_device_name(device)
    except Exception:
        return f"cuda:{device}"


def tune(d, mode=B.EPIE_MINIBATCH, batches=(64, 128, 256, 512, 1024), graph=(True, False),
         intensity_dtype=B.EPIE_U16, sweeps=2, device=0, cache=True):
    """d: a scan dict from synth (N, H, W, P0, frames, pos, dark).  Returns
    (best, table) with best = {"batch": B, "graph": bool} and table the
    measured frame-updates/s per candidate."""
    key = json.dumps([_gpu_name(device), int(d["N"]), int(len(d["pos"])), int(mode),
                      list(batches), list(graph), int(intensity_dtype)])
    store = {}
    if cache and os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                store = json.load(f)
        except (OSError, ValueError):
            store = {}
    if key in store:
        return store[key]["best"], store[key]["table"]
    cands = [(b, g) for b in (batches if mode == B.EPIE_MINIBATCH else (0,)) for g in graph]
    table, best, best_rate = {}, None, -1.0
    for b, g in cands:
        with B.Engine(d["N"], d["H"], d["W"], d["P0"], None, capacity=len(d["pos"]), mode=mode,
                      batch=max(b, 1), device=device, intensity_dtype=intensity_dtype,
                      flags=B.EPIE_GRAPH if g else 0) as eng:
            if d.get("dark") is not None:
                eng.set_dark(d["dark"])
            eng.append(d["frames"], d["pos"])
            eng.iterate(1)
            eng.iterate(sweeps)
            ms, _ = eng.last_timing()
        rate = len(d["pos"]) * sweeps / (ms / 1e3)
        table[f"batch={b},graph={int(g)}"] = rate
        if rate > best_rate:
            best_rate, best = rate, {"batch": b, "graph": bool(g)}
    if cache:
        store[key] = {"best": best, "table": table}
        tmp = CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(store, f, indent=1)
        os.replace(tmp, CACHE)
    return best, table
