"""Band width and hub threshold for batches of graphs, picked by measurement.

Two layout choices of the generator change its speed but never its output:
the width of the radial bands (bands = ceil(R / width)) and the candidate
count above which a band's vertices are queried one warp each
(hub_candidates).  The best values depend on n, alpha and kbar.  This tuner
groups a batch's graphs by size class (half decades of n), generates a
sample of each class under every candidate setting, and keeps the fastest
setting per class.  The graphs themselves are the same under every setting.
"""
from __future__ import annotations

import math
import time

from . import _lib as H

WIDTHS = (1.25, 1.5, 2.0, 2.5)
HUB_CANDIDATES = (256, 512, 1024)


def size_class(n: int) -> int:
    return int(math.floor(2.0 * math.log10(max(2, n))))


def _with_setting(it, width, hub):
    n, alpha, kbar, seed = it
    R = H.hrg_solve_radius(n, alpha, kbar)
    return {"n": n, "alpha": alpha, "avg_degree": kbar, "seed": seed,
            "bands": max(1, min(64, int(math.ceil(R / width)))), "hub_candidates": hub}


def _time_batch(ctx, items, reps, stream):
    import torch

    best = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = H.generate_batch(ctx, items, stream=stream)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
        del g
    return best


def tune(ctx, items, per_class: int = 96, reps: int = 2, stream=None) -> dict:
    """{size class: (width, hub_candidates)} for the classes present in
    items, each from the fastest of all settings on up to per_class of its
    graphs."""
    classes = {}
    for it in items:
        classes.setdefault(size_class(it[0]), []).append(it)
    table = {}
    for c, its in sorted(classes.items()):
        sample = its[:per_class]
        H.generate_batch(ctx, [_with_setting(it, 1.5, 512) for it in sample], stream=stream)  # warm the workspace
        timings = {}
        for w in WIDTHS:
            for h in HUB_CANDIDATES:
                timings[(w, h)] = _time_batch(ctx, [_with_setting(it, w, h) for it in sample], reps, stream)
        table[c] = min(timings, key=timings.get)
    return table


def apply(items, table: dict, default=(1.5, 512)):
    """The items as dicts carrying the tuned bands and hub threshold."""
    return [_with_setting(it, *table.get(size_class(it[0]), default)) for it in items]
