"""Band width and hub threshold for batches of graphs, picked by measurement.

Two layout choices of the generator change its speed but never its output:
the width of the radial bands (bands = ceil(R / width)) and the candidate
count above which a band's vertices are queried one warp each
(hub_candidates).  The best values depend on n, alpha and kbar.  This tuner
groups a batch's graphs by size class (half decades of n) and picks one
setting per class by timing the whole batch: starting from the defaults,
each class in turn (the one with most vertices first) tries every setting
while the other classes keep theirs, and takes the fastest if it beats the
current layout by more than a noise margin.  The classes of one batch share
its launches, so a setting is judged by what it does to the batch, not to
its class alone.  The graphs themselves are the same under every setting.
"""
from __future__ import annotations

import math

from . import _lib as H

WIDTHS = (1.25, 1.5, 2.0, 2.5)
HUB_CANDIDATES = (256, 512, 1024)
DEFAULT = (1.5, 512)


def size_class(n: int) -> int:
    return int(math.floor(2.0 * math.log10(max(2, n))))


def _with_setting(it, width, hub):
    n, alpha, kbar, seed = it
    R = H.hrg_solve_radius(n, alpha, kbar)
    return {"n": n, "alpha": alpha, "avg_degree": kbar, "seed": seed,
            "bands": max(1, min(64, int(math.ceil(R / width)))), "hub_candidates": hub}


def _time_batch(ctx, prepared, reps, stream):
    """Fastest of reps calls of generate_batch, in ms (CUDA events on the
    stream the batch runs on)."""
    import torch

    st = stream if stream is not None else torch.cuda.current_stream(torch.device("cuda", ctx.device))
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        g = H.generate_batch(ctx, prepared, stream=stream)
        b.record(st)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
        del g
    return best


def tune(ctx, items, per_class: int | None = None, reps: int = 2, stream=None, min_gain: float = 0.01) -> dict:
    """{size class: (width, hub_candidates)} for every class present in
    items, by coordinate descent over the classes on the whole batch (the
    first per_class graphs of each class, in batch order, if per_class is
    set).  A class keeps DEFAULT unless a setting makes the batch faster by
    more than the fraction min_gain; each timing is the fastest of reps
    calls."""
    classes = {}
    for it in items:
        classes.setdefault(size_class(it[0]), []).append(it)
    if per_class is not None:
        seen = {}
        sample = []
        for it in items:
            c = size_class(it[0])
            if seen.get(c, 0) < per_class:
                seen[c] = seen.get(c, 0) + 1
                sample.append(it)
    else:
        sample = list(items)
    table = {c: DEFAULT for c in classes}
    if not sample:
        return table
    H.generate_batch(ctx, H.BatchItems(apply(sample, table)), stream=stream)  # warm the workspace
    current = _time_batch(ctx, H.BatchItems(apply(sample, table)), reps, stream)
    for c in sorted(classes, key=lambda k: -sum(it[0] for it in classes[k])):
        best, best_ms = table[c], current
        for w in WIDTHS:
            for h in HUB_CANDIDATES:
                if (w, h) == table[c]:
                    continue
                ms = _time_batch(ctx, H.BatchItems(apply(sample, {**table, c: (w, h)})), reps, stream)
                if ms < best_ms:
                    best, best_ms = (w, h), ms
        if best_ms < current * (1.0 - min_gain):
            table[c], current = best, best_ms
    return table


def apply(items, table: dict, default=DEFAULT):
    """The items as dicts carrying the tuned bands and hub threshold."""
    return [_with_setting(it, *table.get(size_class(it[0]), default)) for it in items]
