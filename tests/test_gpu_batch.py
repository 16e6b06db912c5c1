"""Batches of graphs (hrg_generate_batch_begin): every graph of a batch must
be the graph a single-graph call with the same parameters produces, and the
graph the oracle produces."""
import numpy as np
import pytest

import oracle as O
from paper_1501_03545_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_1501_03545_gb300 import _lib as H

    assert torch.cuda.is_available()
    H.load()
    c = H.Context(0)
    yield c
    c.close()


def _graph(out, g):
    a, b = out["goff"][g], out["goff"][g + 1]
    off = out["row_off"][a:b + 1].cpu().numpy()
    col = out["col_idx"][int(off[0]):int(off[-1])].cpu().numpy()
    return out["r"][a:b].cpu().numpy(), out["phi"][a:b].cpu().numpy(), off - off[0], col


def _single(ctx, it, fp64=False):
    from paper_1501_03545_gb300 import _lib as H

    g = H.generate(ctx, it[0], it[1], it[2], it[3], fp64_only=fp64)
    return (g["r"].cpu().numpy(), g["phi"].cpu().numpy(), g["row_off"].cpu().numpy(), g["col_idx"].cpu().numpy())


MIXED = [
    (1000, 0.55, 32.0, 11), (2345, 1.5, 4.0, 12), (7001, 0.75, 10.0, 13), (60000, 0.55, 16.0, 14),
    (4096, 1.0, 8.0, 15), (31337, 0.6, 32.0, 16), (1500, 0.9, 16.0, 17), (100000, 0.55, 32.0, 18),
    (12000, 1.2, 6.0, 19), (2, 1.0, 0.5, 20), (3, 0.7, 1.0, 21), (50000, 0.8, 20.0, 22),
]


@pytest.mark.parametrize("fp64", [False, True])
def test_batch_equals_single_calls(ctx, fp64):
    from paper_1501_03545_gb300 import _lib as H

    out = H.generate_batch(ctx, MIXED, fp64_only=fp64)
    assert out["goff"][-1] == sum(it[0] for it in MIXED)
    total = 0
    for g, it in enumerate(MIXED):
        r, phi, off, col = _graph(out, g)
        r1, phi1, off1, col1 = _single(ctx, it, fp64)
        assert np.array_equal(phi, phi1) and np.array_equal(r, r1), g
        assert np.array_equal(off, off1), g
        assert np.array_equal(col, col1), g
        total += len(col)
    assert total == out["stats"]["n_entries"]


def test_batch_equals_oracle(ctx):
    from paper_1501_03545_gb300 import _lib as H

    items = [(800, 0.6, 12.0, 31), (2500, 1.1, 8.0, 32), (1200, 0.55, 30.0, 33), (3000, 1.45, 4.0, 34)]
    out = H.generate_batch(ctx, items)
    for g, (n, alpha, kbar, seed) in enumerate(items):
        r, phi, off, col = _graph(out, g)
        R = O.solve_radius(n, alpha, kbar)
        ro, phio = O.sample(n, alpha, R, seed)
        assert np.array_equal(phi, phio)
        assert np.max(np.abs(r - ro) / np.maximum(ro, 1e-300)) < 1e-14
        offo, colo = O.brute_csr(ro, phio, R)
        n_ties, _ = O.brute_ties(ro, phio, R)
        assert n_ties == 0
        assert np.array_equal(off, offo), g
        assert np.array_equal(col, colo), g


def test_batch_of_one(ctx):
    from paper_1501_03545_gb300 import _lib as H

    it = (40000, 0.7, 12.0, 5)
    out = H.generate_batch(ctx, [it])
    r, phi, off, col = _graph(out, 0)
    r1, phi1, off1, col1 = _single(ctx, it)
    assert np.array_equal(off, off1) and np.array_equal(col, col1) and np.array_equal(r, r1)


def test_batch_full_workload_sampled(ctx):
    """The 4096-graph batched workload; 24 graphs re-generated alone."""
    from paper_1501_03545_gb300 import _lib as H

    items = W.batch_items()
    out = H.generate_batch(ctx, items)
    off_all = out["row_off"]
    assert bool((off_all[1:] >= off_all[:-1]).all())
    rng = np.random.default_rng(5)
    pick = sorted(set(rng.integers(0, len(items), size=24).tolist()) | {0, len(items) - 1})
    for g in pick:
        r, phi, off, col = _graph(out, g)
        r1, phi1, off1, col1 = _single(ctx, items[g])
        assert np.array_equal(off, off1), g
        assert np.array_equal(col, col1), g
    st = out["stats"]
    assert st["n_entries"] == int(off_all[-1].item())


def test_batch_invalid_item(ctx):
    from paper_1501_03545_gb300 import _lib as H

    with pytest.raises(H.HrgError) as e:
        H.generate_batch(ctx, [(1000, 1.0, 6.0, 1), (1000, 0.4, 6.0, 2)])
    assert e.value.code == H.HRG_EINVAL and "item 1" in str(e.value)


def test_autotuned_layout_same_graphs(ctx):
    """The tuner changes band widths and hub thresholds, never the graphs."""
    from paper_1501_03545_gb300 import _lib as H
    from paper_1501_03545_gb300 import autotune

    items = W.batch_items(count=96, draw_seed=9)
    table = autotune.tune(ctx, items, per_class=12, reps=1)
    assert table and all(w in autotune.WIDTHS and h in autotune.HUB_CANDIDATES for w, h in table.values())
    tuned = autotune.apply(items, table)
    odd = [dict(t, bands=1 + (k % 64), hub_candidates=(64, 4096)[k % 2]) for k, t in enumerate(tuned)]
    a = H.generate_batch(ctx, items)
    for other in (tuned, odd):
        b = H.generate_batch(ctx, other)
        assert np.array_equal(a["row_off"].cpu().numpy(), b["row_off"].cpu().numpy())
        assert np.array_equal(a["col_idx"].cpu().numpy(), b["col_idx"].cpu().numpy())
        assert np.array_equal(a["r"].cpu().numpy(), b["r"].cpu().numpy())
