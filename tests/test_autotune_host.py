"""Host logic of the batch layout tuner (no GPU needed): the coordinate
descent over size classes on a fake batch timer.  It keeps the defaults when
no setting beats them by the margin, takes a setting that does, judges every
setting on the whole batch, and limits the timed batch to per_class graphs
of each class in batch order."""
from paper_1501_03545_gb300 import autotune as T

ITEMS = ([(1000 + 37 * k, 0.8, 8.0, k) for k in range(200)]
         + [(60_000 + k, 1.0, 4.0, 500 + k) for k in range(20)])


def _fake(monkeypatch, cost):
    seen = []

    def time_batch(ctx, prepared, reps, stream):
        ps = [prepared.arr[k] for k in range(len(prepared))]
        seen.append(ps)
        return cost(ps)

    monkeypatch.setattr(T, "_time_batch", time_batch)
    monkeypatch.setattr(T.H, "generate_batch", lambda *a, **k: None)
    return seen


def test_classes_and_defaults(monkeypatch):
    seen = _fake(monkeypatch, lambda ps: 10.0)
    table = T.tune(None, ITEMS, reps=1)
    assert table == {6: T.DEFAULT, 7: T.DEFAULT, 9: T.DEFAULT}
    # one timing of the current layout, then every other setting per class
    per_class = len(T.WIDTHS) * len(T.HUB_CANDIDATES) - 1
    assert len(seen) == 1 + 3 * per_class
    assert all(len(ps) == len(ITEMS) for ps in seen)


def test_gain_above_margin_taken_below_it_not(monkeypatch):
    def cost(ps):
        ms = 10.0
        for p in ps:
            c = T.size_class(p.n)
            if c == 7 and p.hub_candidates == 256:
                ms -= 5.0 / len(ps)  # ~2 % of the batch: taken
            if c == 9 and p.hub_candidates == 1024:
                ms -= 0.01 / len(ps)  # far below the 1 % margin: not taken
        return ms

    _fake(monkeypatch, cost)
    table = T.tune(None, ITEMS, reps=1)
    assert table[7][1] == 256 and table[9] == T.DEFAULT and table[6] == T.DEFAULT
    for c, (w, h) in table.items():
        assert w in T.WIDTHS and h in T.HUB_CANDIDATES
    # the tuned items carry the bands of the chosen width
    tuned = T.apply(ITEMS, table)
    for it, d in zip(ITEMS, tuned):
        w, h = table[T.size_class(it[0])]
        assert d["hub_candidates"] == h and d["n"] == it[0] and d["seed"] == it[3]
        assert d["bands"] >= 1


def test_per_class_sample_in_batch_order(monkeypatch):
    seen = _fake(monkeypatch, lambda ps: 10.0)
    T.tune(None, ITEMS, per_class=5, reps=1)
    first = [(p.n, p.seed) for p in seen[0]]
    want = [(it[0], it[3]) for it in ITEMS if T.size_class(it[0]) == 6][:5]
    want += [(it[0], it[3]) for it in ITEMS if T.size_class(it[0]) == 7][:5]
    want += [(it[0], it[3]) for it in ITEMS if T.size_class(it[0]) == 9][:5]
    assert sorted(first) == sorted(want) and len(first) == 15


def test_empty_batch(monkeypatch):
    seen = _fake(monkeypatch, lambda ps: 10.0)
    assert T.tune(None, [], reps=1) == {} and not seen
