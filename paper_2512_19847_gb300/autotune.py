"""Tile-shape autotuner for the stencil kernels of a Solver or Batch.

Every tile shape the attached grids admit is timed on the handle's own solves
(a few IMEX steps, CUDA events on the handle's stream); the state is saved
before and restored bit for bit afterwards, so tuning never changes results.
The winner is cached in a JSON file keyed by GPU name, precision, scheme,
tableau size and the multiset of grid sizes.
"""
from __future__ import annotations

import json
import os

import torch

from . import api

TILES = {0: (32, 8), 1: (32, 4), 2: (16, 8), 3: (8, 8), 4: (64, 4), 5: (32, 16)}
DEFAULT_CACHE = os.environ.get("AP_DVM_AUTOTUNE_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "ap_dvm", "autotune.json"))


def _params_of(h):
    return dict(h._params)


def signature(h) -> str:
    ps = _params_of(h)
    sizes = sorted((p.nx, p.ny) for p in ps.values())
    counts = {}
    for s in sizes:
        counts[s] = counts.get(s, 0) + 1
    p0 = next(iter(ps.values()))
    gpu = torch.cuda.get_device_name()
    return json.dumps([gpu, int(p0.precision), int(p0.space_scheme), int(p0.s),
                       sorted([[a, b, c] for (a, b), c in counts.items()])])


def _save(h):
    saved = {}
    for slot, p in _params_of(h).items():
        if p.precision == api.FP32_DEV:
            saved[slot] = (h.get_populations(slot, dtype=torch.float32), None)
        elif p.precision == api.FP32_DEV_TH:   # the populations and the carried theta plane
            saved[slot] = (h.get_populations(slot, dtype=torch.float32), h.get_state(slot)[2].clone())
        else:
            saved[slot] = (h.get_state(slot), None)
    return saved


def _restore(h, saved):
    for slot, (X, theta) in saved.items():
        if X.dtype == torch.float32:
            h.set_populations(X, slot)
            if theta is not None:
                h.set_theta(theta, slot)
        else:
            h.set_state(X, slot)


def candidates(h):
    ps = list(_params_of(h).values())
    out = []
    for t, (tx, ty) in TILES.items():
        if all(p.nx >= tx and p.ny >= ty for p in ps):
            out.append(t)
    return out


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(h, steps: int = 2, path: str | None = DEFAULT_CACHE, use_cache: bool = True) -> dict:
    """Pick and set the fastest tile shape for the solves attached to h.
    Returns {"tile": t, "ms_per_step": {t: ms}, "cached": bool}."""
    key = signature(h)
    cache = load_cache(path) if (path and use_cache) else {}
    if key in cache:
        h.set_tile(int(cache[key]["tile"]))
        return {"tile": int(cache[key]["tile"]), "ms_per_step": cache[key]["ms_per_step"], "cached": True}
    saved = _save(h)
    stream = torch.cuda.current_stream()
    times = {}
    for t in candidates(h):
        h.set_tile(t)
        h.step(1)                      # warm-up: kernel attributes, work lists
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.step(steps)
        e1.record(stream)
        e1.synchronize()
        times[t] = e0.elapsed_time(e1) / steps
        _restore(h, saved)
    best = min(times, key=times.get)
    h.set_tile(best)
    _restore(h, saved)
    torch.cuda.synchronize()
    if path:
        cache = load_cache(path)
        cache[key] = {"tile": best, "ms_per_step": {str(k): v for k, v in times.items()}}
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return {"tile": best, "ms_per_step": {str(k): v for k, v in times.items()}, "cached": False}
