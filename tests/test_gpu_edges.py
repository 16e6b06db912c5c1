"""Parity where the generator is most likely to go wrong, through the C ABI:

* pairs placed at the edge of the angular window of Sec. 2.1's circle (the
  closed-form half-width at a band's inner radius, which the device computes
  in FP32 and pads), at the radius of the 1e8-vertex workload (R = 39.03);
* the tie band: pairs whose cosh d equals cosh R to a few ulp, counted by the
  device (hrg_stats.ties) as the oracle counts them;
* every fallback branch of the count pass (row buffer full, hub pool or run
  table full, list of long hub ranges full), forced with tiny capacities
  (hrg_set_limits) and shown to have run by its counter.

Bar: the CSR equals the oracle's outside the listed tie band.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1501_03545_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = None


@pytest.fixture(scope="module")
def ctx():
    global H
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_03545_gb300 import _lib

    H = _lib
    c = _lib.Context(0)
    yield c
    c.set_limits()
    c.close()


def _np(t):
    return t.detach().cpu().numpy()


def _edge_keys(off, col):
    rows = np.repeat(np.arange(len(off) - 1, dtype=np.int64), np.diff(off))
    return rows * (1 << 32) + col.astype(np.int64)


def _assert_matches(g_off, g_col, o_off, o_col, ties):
    if np.array_equal(g_off, o_off) and np.array_equal(g_col, o_col):
        return 0
    diff = np.setxor1d(_edge_keys(g_off, g_col), _edge_keys(o_off, o_col))
    allowed = {int(i) * (1 << 32) + int(j) for i, j in ties} | {int(j) * (1 << 32) + int(i) for i, j in ties}
    bad = [int(x) for x in diff if int(x) not in allowed]
    assert not bad, [(x >> 32, x & 0xFFFFFFFF) for x in bad[:5]]
    return len(diff)


def _check_rows(off, col):
    n = len(off) - 1
    rows = np.repeat(np.arange(n), np.diff(off))
    assert np.all(col != rows)
    same = rows[1:] == rows[:-1]
    assert np.all(np.diff(col.astype(np.int64))[same] > 0)


def _window_edge_points(R, B, seed):
    """For queries at many radii r_q and every band inner radius b = R k / B
    (the device's band boundaries, same double arithmetic): candidates at
    r = b whose angular distance is theta(r_q, b) times 1 -+ {1e-4, 1e-6,
    1e-7}, theta the exact half-width (sin^2(theta/2) = (cosh R - cosh(r_q -
    b)) / (2 sinh r_q sinh b)), on alternating sides of the query.  The pairs
    inside are edges by a relative margin of the same order, those outside
    are not; a window narrower than theta by more than that drops an edge."""
    rng = np.random.default_rng(seed)
    r, phi = [], []
    cR = math.cosh(R)
    for k in range(1, B):
        b = R * float(k) / float(B)
        radii = list(rng.uniform(0.05, R, size=10)) + [R - b + 1e-3, R - b + 0.1, R - b + 1.0]
        for rq in radii:
            if not (0.0 < rq < R):
                continue
            X = (cR - math.cosh(rq - b)) / (2.0 * math.sinh(rq) * math.sinh(b))
            if not (0.0 < X < 1.0):
                continue
            th = 2.0 * math.asin(math.sqrt(X))
            if th > math.pi - 0.02:
                continue
            lo, hi = th * 1.001 + 1e-3, 2.0 * math.pi - th * 1.001 - 1e-3
            phq = float(rng.uniform(lo, hi))
            r.append(rq)
            phi.append(phq)
            for s, f in enumerate((1 - 1e-4, 1 - 1e-6, 1 - 1e-7, 1 + 1e-7, 1 + 1e-6, 1 + 1e-4)):
                r.append(b)
                phi.append(phq + th * f if s % 2 == 0 else phq - th * f)
    rb, pb = W.random_points(800, R, seed + 1)
    return np.concatenate([np.array(r), rb]), np.concatenate([np.array(phi), pb])


@pytest.mark.parametrize("fp64", [False, True], ids=["fp32filter", "fp64"])
def test_window_edge_pairs_match_oracle(ctx, fp64):
    R = O.solve_radius(W.LARGE.n, W.LARGE.alpha, W.LARGE.kbar)  # 39.03
    B = math.ceil(R / 1.7)  # the automatic band count
    r, phi = _window_edge_points(R, B, 5)
    assert np.all((phi >= 0) & (phi < 2 * math.pi)) and np.all((r >= 0) & (r < R))
    g = H.generate_from_points(ctx, torch.tensor(r, device="cuda"), torch.tensor(phi, device="cuda"), R,
                               fp64_only=fp64)
    assert g["stats"]["bands"] == B and g["stats"]["hub_queries"] > 0
    off, col = _np(g["row_off"]), _np(g["col_idx"])
    o_off, o_col = O.brute_csr(r, phi, R)
    nt, ties = O.brute_ties(r, phi, R)
    _assert_matches(off, col, o_off, o_col, ties)
    _check_rows(off, col)
    # the designed pairs near the edge really are split by the oracle
    v = np.array([O.cosh_dist(r[0], phi[0], r[k], phi[k]) for k in range(1, 7)])
    assert np.sum(v < math.cosh(R)) == 3, v / math.cosh(R) - 1


def _tie_points():
    """Antipodal pairs with r_i + r_j = R (rounded): cosh d = cosh R to a few
    ulp, inside the tie band; with them pairs at r_i + r_j = R (1 -+ 1e-9),
    outside it; and a random background."""
    R = 12.0
    r, phi = [], []
    for k in range(24):
        a = 0.1 + 0.25 * k
        ri = 1.5 + 0.35 * k
        for rj in (R - ri, R * (1 - 1e-9) - ri, R * (1 + 1e-9) - ri):
            r += [ri, rj]
            phi += [a, math.fmod(a + math.pi, 2 * math.pi)]
            a += 0.011
    rb, pb = W.random_points(1500, R, 77)
    return np.concatenate([np.array(r), rb]), np.concatenate([np.array(phi), pb]), R


@pytest.mark.parametrize("fp64", [False, True], ids=["fp32filter", "fp64"])
def test_tie_band_counted_like_the_oracle(ctx, fp64):
    r, phi, R = _tie_points()
    g = H.generate_from_points(ctx, torch.tensor(r, device="cuda"), torch.tensor(phi, device="cuda"), R,
                               fp64_only=fp64)
    nt, ties = O.brute_ties(r, phi, R)
    assert nt >= 24
    assert g["stats"]["ties"] == nt
    o_off, o_col = O.brute_csr(r, phi, R)
    _assert_matches(_np(g["row_off"]), _np(g["col_idx"]), o_off, o_col, ties)


def test_no_ties_on_the_small_workload(ctx):
    w = W.SMALL
    g = H.generate(ctx, w.n, w.alpha, w.kbar, w.seed)
    r, phi = O.sample(w.n, w.alpha, g["stats"]["R"], w.seed)
    nt, _ = O.brute_ties(r, phi, g["stats"]["R"])
    assert g["stats"]["ties"] == nt == 0


# (n, alpha, kbar, seed, hub_candidates): the small workload, a scaled copy of
# the 1e8 workload (long hub ranges: hub queries see whole outer bands), and
# a dense graph; low hub thresholds put more vertices on the hub path
FALLBACK_CASES = [(10_000, 1.0, 6.0, 1, 16), (30_011, 0.55, 16.0, 3, 64), (31_337, 0.6, 32.0, 16, 32)]
LIMITS = {
    "row_buffer": dict(row_buffer_ids=97),
    "hub_pool": dict(hub_pool_ids=300),
    "hub_runs": dict(hub_runs=3),
    "heavy_list": dict(heavy_segments=1),
    "all": dict(row_buffer_ids=97, hub_pool_ids=300, hub_runs=3, heavy_segments=1),
}


_ORACLE = {}


def _oracle_csr(n, alpha, kbar, seed, R):
    """The oracle's CSR and tie list of one case, computed once per module
    (all-pairs below 2e4 vertices, the band algorithm above)."""
    key = (n, alpha, kbar, seed, R)
    if key not in _ORACLE:
        r, phi = O.sample(n, alpha, R, seed)
        if n <= 20_000:
            off, col = O.brute_csr(r, phi, R)
            _, ties = O.brute_ties(r, phi, R)
        else:
            b = O.Bands(r, phi, R)
            off, col = b.csr()
            _, ties = b.ties()
            b.close()
        _ORACLE[key] = (off, col, ties)
    return _ORACLE[key]


@pytest.mark.parametrize("fp64", [False, True], ids=["fp32filter", "fp64"])
def test_fallback_branches_match_oracle(ctx, fp64):
    """Each limit alone and all together, on every case: the graph equals
    the one generated with automatic capacities (which equals the oracle's),
    and each limited buffer's fallback is seen to run by its counter."""
    seen = {w: {"rows_no_room": 0, "hub_rows_retraversed": 0, "heavy_retries": 0} for w in LIMITS}
    try:
        for n, alpha, kbar, seed, hub in FALLBACK_CASES:
            ctx.set_limits()
            ref = H.generate(ctx, n, alpha, kbar, seed, fp64_only=fp64, hub_candidates=hub)
            st = ref["stats"]
            assert st["rows_no_room"] == 0 and st["hub_rows_retraversed"] == 0 and st["heavy_retries"] == 0
            o_off, o_col, ties = _oracle_csr(n, alpha, kbar, seed, st["R"])
            _assert_matches(_np(ref["row_off"]), _np(ref["col_idx"]), o_off, o_col, ties)
            for which, lim in LIMITS.items():
                ctx.set_limits(**lim)
                g = H.generate(ctx, n, alpha, kbar, seed, fp64_only=fp64, hub_candidates=hub)
                ctx.set_limits()
                assert torch.equal(g["row_off"], ref["row_off"]), (n, which)
                assert torch.equal(g["col_idx"], ref["col_idx"]), (n, which)
                s = g["stats"]
                for k in seen[which]:
                    seen[which][k] += s[k]
                # a hub row is traversed again only when the pool overflowed, and then all of them are
                assert s["hub_rows_retraversed"] in (0, st["hub_queries"]), (n, which)
    finally:
        ctx.set_limits()
    for which, lim in LIMITS.items():
        if "row_buffer_ids" in lim:
            assert seen[which]["rows_no_room"] > 0, which
        if "hub_pool_ids" in lim or "hub_runs" in lim:
            assert seen[which]["hub_rows_retraversed"] > 0, which
        if "heavy_segments" in lim:
            assert seen[which]["heavy_retries"] > 0, which


def test_fallback_branches_in_a_batch(ctx):
    items = [(2_000, 0.55, 32.0, 41), (9_000, 0.9, 8.0, 42), (30_011, 0.55, 16.0, 3), (1_200, 1.4, 4.0, 43)]
    ref = H.generate_batch(ctx, items)
    try:
        ctx.set_limits(**LIMITS["all"])
        out = H.generate_batch(ctx, items)
    finally:
        ctx.set_limits()
    s = out["stats"]
    assert s["rows_no_room"] > 0 and s["hub_rows_retraversed"] > 0
    assert torch.equal(out["row_off"], ref["row_off"]) and torch.equal(out["col_idx"], ref["col_idx"])
    for g, (n, alpha, kbar, seed) in enumerate(items):
        a, b = out["goff"][g], out["goff"][g + 1]
        off = _np(out["row_off"][a:b + 1])
        col = _np(out["col_idx"][int(off[0]):int(off[-1])])
        o_off, o_col, ties = _oracle_csr(n, alpha, kbar, seed, O.solve_radius(n, alpha, kbar))
        _assert_matches(off - off[0], col, o_off, o_col, ties)


def test_limits_rejected(ctx):
    L = H.load()
    import ctypes

    bad = H.hrg_limits(-1, 0, 0, 0)
    assert L.hrg_set_limits(ctx.h, ctypes.byref(bad)) == H.HRG_EINVAL
    bad = H.hrg_limits(0, 1 << 40, 0, 0)
    assert L.hrg_set_limits(ctx.h, ctypes.byref(bad)) == H.HRG_EINVAL
    bad = H.hrg_limits(0, 0, 0, 0, -1)
    assert L.hrg_set_limits(ctx.h, ctypes.byref(bad)) == H.HRG_EINVAL
    assert L.hrg_set_limits(ctx.h, None) == H.HRG_OK


def test_workspace_cap_gives_enomem_and_the_context_recovers(ctx):
    """A device allocation that fails (forced here by a cap on the context's
    workspace, on the host, with no GPU fault) returns HRG_ENOMEM; the
    context then generates the same graph once the cap is lifted."""
    w = W.scaled(W.MEDIUM, 100_000)
    ref = H.Context(0)
    c = H.Context(0)
    try:
        a = H.generate(ref, w.n, w.alpha, w.kbar, w.seed)
        for cap in (1 << 20, 6 << 20):  # the first allocation, then one part-way through
            c.set_limits(workspace_bytes=cap)
            with pytest.raises(H.HrgError) as e:
                H.generate(c, w.n, w.alpha, w.kbar, w.seed)
            assert e.value.code == H.HRG_ENOMEM
            assert c.workspace_bytes() <= cap
        c.set_limits()
        b = H.generate(c, w.n, w.alpha, w.kbar, w.seed)
        for k in ("r", "phi", "row_off", "col_idx"):
            assert torch.equal(a[k], b[k]), k
        # a larger graph under a cap below what the context already holds
        # fails at its first growing buffer; the workspace given back and the
        # cap raised, it runs
        w2 = W.scaled(W.MEDIUM, 200_000)
        a2 = H.generate(ref, w2.n, w2.alpha, w2.kbar, w2.seed)
        c.set_limits(workspace_bytes=c.workspace_bytes() // 2)
        with pytest.raises(H.HrgError) as e:
            H.generate(c, w2.n, w2.alpha, w2.kbar, w2.seed)
        assert e.value.code == H.HRG_ENOMEM
        c.release_workspace()
        assert c.workspace_bytes() == 0
        c.set_limits(workspace_bytes=4 << 30)
        b2 = H.generate(c, w2.n, w2.alpha, w2.kbar, w2.seed)
        assert torch.equal(a2["row_off"], b2["row_off"]) and torch.equal(a2["col_idx"], b2["col_idx"])
    finally:
        c.close()
        ref.close()
