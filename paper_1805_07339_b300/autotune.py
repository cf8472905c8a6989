"""Autotune cache for batched plans.

The timing search itself is native (scn_plan_autotune); this module keys its
result by GPU, by the multiset of frame sizes and by the sampling patterns of a
plan, and keeps it in a JSON file so a later plan of the same shape skips the
search.
"""
from __future__ import annotations

import json
import os
from collections import Counter

from . import scn

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "scn", "autotune.json")


def plan_key(gpu_name: str, videos: list[dict]) -> str:
    """videos: dicts with width, height, sampling (and frames, whose count is bucketed)."""
    sizes = Counter((v["width"], v["height"]) for v in videos)
    kinds = Counter(v.get("sampling", "?") for v in videos)
    frames = sum(len(v["frames"]) for v in videos)
    bucket = 1 << max(0, frames.bit_length() - 1)
    sz = ",".join(f"{w}x{h}:{c}" for (w, h), c in sorted(sizes.items()))
    kd = ",".join(f"{k}:{c}" for k, c in sorted(kinds.items()))
    return f"{gpu_name}|{sz}|{kd}|frames~{bucket}"


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune_plan(plan: int, key: str, cache_path: str | None = DEFAULT_CACHE, reps: int = 3, stream=None) -> dict:
    """Apply the cached shape for key, or search, apply and cache one.
    Returns {"tune": ..., "ms": ... or None, "cached": bool}."""
    cache = _load(cache_path) if cache_path else {}
    if key in cache:
        t = cache[key]["tune"]
        scn.scn_plan_set_tune(plan, **t)
        return {"tune": t, "ms": cache[key].get("ms"), "cached": True}
    best, ms = scn.scn_plan_autotune(plan, reps=reps, stream=stream)
    if cache_path:
        cache[key] = {"tune": best, "ms": ms}
        os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return {"tune": best, "ms": ms, "cached": False}
