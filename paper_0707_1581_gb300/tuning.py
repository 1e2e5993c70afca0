"""A JSON cache of autotuner choices, keyed by what the choice depends on.

`autotune_cached(ctx, path)` looks the context's boxes up in the cache file;
on a hit it applies the recorded streaming pattern and launch shape
(flb_set_pattern, flb_set_launch), on a miss it runs flb_autotune(_ex) and
records the result.  The key holds the lattice, the storage format, every
box's size, whether the pattern was tuned, the GPU's name and the library
version; the choice is a pure function of those (the timings that produced it
are not repeated).  Host logic only -- the tuning itself runs in libflb.so.
"""
from __future__ import annotations

import json
import os

from . import flb


def tuning_key(ctx, tune_pattern: bool, device: str) -> str:
    boxes = [[c.nx, c.ny, c.nz] for c in ctx.cfgs]
    c0 = ctx.cfgs[0]
    return json.dumps({"lattice": int(c0.lattice), "store": int(c0.store),
                       "pattern": "tuned" if tune_pattern else int(c0.pattern),
                       "boxes": boxes, "device": device, "library": flb.flb_version()}, sort_keys=True)


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name() if torch.cuda.is_available() else "unknown"
    except Exception:
        return "unknown"


def autotune_cached(ctx, path: str, trials: int = 2, pattern: bool = False, device: str | None = None) -> dict:
    """Apply the cached choice for ctx, or tune and record it; returns the choice
    {"launch": [V, bx, by], "pattern": "ab"|"aa", "cached": bool}."""
    key = tuning_key(ctx, pattern, device or _device_name())
    cache = {}
    if os.path.exists(path):
        with open(path) as f:
            cache = json.load(f)
    if key in cache:
        rec = cache[key]
        if pattern and ctx.flb_get_pattern() != rec["pattern"]:
            ctx.flb_set_pattern(rec["pattern"])
        ctx.flb_set_launch(*rec["launch"])
        return {**rec, "cached": True}
    ctx.flb_autotune(trials, pattern=pattern)
    rec = {"launch": list(ctx.flb_get_launch()), "pattern": ctx.flb_get_pattern()}
    cache[key] = rec
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return {**rec, "cached": False}
