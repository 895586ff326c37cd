"""Autotuner for the ragged-batch launch: picks the work-unit shape (four
shapes, three of them valid for six-level images) and the persistent grid
size (resident warps per SM) by timing every candidate on the caller's
actual layout, and caches the choice as JSON.

The cache key is (input dtype, coefficient dtype, level-count range, a
size class of the batch, SM count, device name); the size class buckets the
image count and the total pixel count by powers of two, so batches drawn
from the same distribution share one entry.
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional

import torch

from . import _lib
from .api import RaggedPlan

# unit name -> (unit code, unit height, warps per unit)
UNITS = {"64x128": (_lib.HAAR_UNIT_64x128, 64, 8), "32x256": (_lib.HAAR_UNIT_32x256, 32, 8),
         "64x64": (_lib.HAAR_UNIT_64x64, 64, 4), "128x128": (_lib.HAAR_UNIT_128x128, 128, 16)}
# persistent grid sizes tried, as resident warps per SM (blocks per SM =
# warps / warps per unit): the register cap allows 48
WARPS_PER_SM = (16, 24, 32, 48)
BLOCKS_PER_SM = tuple(sorted({w // n for _, _, n in UNITS.values() for w in WARPS_PER_SM}))


def candidates(max_levels: int):
    """(name, unit, blocks per SM) of every configuration eligible for a
    batch whose deepest image has max_levels levels (a sixth level needs a
    unit at least 64 rows high)."""
    out = []
    for name, (unit, uh, nw) in UNITS.items():
        if max_levels > 5 and uh < 64:
            continue
        for w in WARPS_PER_SM:
            out.append((name, unit, w // nw))
    return out


def default_cache_path() -> str:
    root = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(root, "fasthaar", "autotune.json")


def cache_key(items, in_dtype, coef_dtype, device) -> str:
    props = torch.cuda.get_device_properties(device)
    n = len(items)
    px = sum(h * w for h, w, _ in items)
    lv = [L for _, _, L in items]
    return "|".join([
        str(in_dtype).replace("torch.", ""), str(coef_dtype).replace("torch.", ""),
        f"L{min(lv)}-{max(lv)}", f"n2^{round(math.log2(max(n, 1)))}",
        f"px2^{round(math.log2(max(px, 1)))}", f"sm{props.multi_processor_count}",
        props.name.replace(" ", "_"),
    ])


def _time_round_trip(plan: RaggedPlan, x, c, y, reps: int) -> float:
    for _ in range(2):
        plan.dwt(x, c)
        plan.idwt(c, y)
    torch.cuda.synchronize(plan.device)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        plan.dwt(x, c)
        plan.idwt(c, y)
    b.record()
    torch.cuda.synchronize(plan.device)
    return a.elapsed_time(b) / reps


def tune_ragged(items, device, x: torch.Tensor, coef_dtype=torch.float32, out_dtype=None,
                reps: int = 5, cache_path: Optional[str] = None, use_cache: bool = True):
    """Returns (unit, blocks_per_sm, report) for the ragged batch ``items``
    ((h, w, levels) per image) with input buffer ``x`` (flat, packed layout).
    Every candidate runs DWT + IDWT on scratch buffers; the fastest wins."""
    out_dtype = out_dtype or (torch.float32 if x.dtype == torch.uint8 else x.dtype)
    path = cache_path or default_cache_path()
    key = cache_key(items, x.dtype, coef_dtype, device)
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            e = cache[key]
            return e["unit"], e["blocks_per_sm"], {"cached": True, "key": key, **e}
    max_levels = max(L for _, _, L in items)
    timings = {}
    best = None
    for uname, unit, bps in candidates(max_levels):
        plan = RaggedPlan(items, device, unit, bps)
        c = plan.empty(coef_dtype)
        y = plan.empty(out_dtype)
        ms = _time_round_trip(plan, x, c, y, reps)
        timings[f"{uname}/bps{bps}"] = round(ms, 4)
        if best is None or ms < best[0]:
            best = (ms, unit, bps, uname)
        del plan, c, y
    _, unit, bps, uname = best
    entry = {"unit": unit, "unit_name": uname, "blocks_per_sm": bps, "ms": round(best[0], 4),
             "timings": timings}
    if use_cache:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            cache[key] = entry
            with open(path + ".tmp", "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
            os.replace(path + ".tmp", path)
        except OSError:
            pass
    return unit, bps, {"cached": False, "key": key, **entry}
