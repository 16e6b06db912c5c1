"""Vertex movement (hrg_update_begin): after k vertices move, the CSR must be
the threshold graph (Sec. 2.1) of the updated point set -- entry for entry
the oracle's CSR of those points, outside the oracle's tie band -- for single
and repeated updates, moves across band boundaries, through phi = 0 and to
and from the centre, on both predicate paths.  The paper's conclusion names
the dynamic model as future work without a law of motion, so the moves are
inputs (workloads.moves)."""
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
    c.close()


def _np(t):
    return t.detach().cpu().numpy()


def _keys(off, col):
    rows = np.repeat(np.arange(len(off) - 1, dtype=np.int64), np.diff(off))
    return rows * (1 << 32) + col.astype(np.int64)


def _assert_matches(g_off, g_col, o_off, o_col, ties):
    if np.array_equal(g_off, o_off) and np.array_equal(g_col, o_col):
        return
    diff = np.setxor1d(_keys(g_off, g_col), _keys(o_off, o_col))
    allowed = {int(i) * (1 << 32) + int(j) for i, j in ties} | {int(j) * (1 << 32) + int(i) for i, j in ties}
    bad = [int(x) for x in diff if int(x) not in allowed]
    assert not bad, [(x >> 32, x & 0xFFFFFFFF) for x in bad[:5]]


def _oracle(r, phi, R):
    if len(r) <= 20_000:
        off, col = O.brute_csr(r, phi, R)
        _, ties = O.brute_ties(r, phi, R)
        return off, col, ties
    b = O.Bands(r, phi, R)
    off, col = b.csr()
    _, ties = b.ties()
    b.close()
    return off, col, ties


def _check_rows(off, col):
    n = len(off) - 1
    assert off[0] == 0
    rows = np.repeat(np.arange(n), np.diff(off))
    assert np.all(col != rows)
    same = rows[1:] == rows[:-1]
    assert np.all(np.diff(col.astype(np.int64))[same] > 0)


@pytest.mark.parametrize("fp64", [False, True], ids=["fp32filter", "fp64"])
def test_repeated_updates_match_oracle(ctx, fp64):
    """The 1e6-vertex workload, then updates of k = 1, 100 and 10^4 vertices
    in a row on the same graph, each against the oracle's CSR of the points
    as they now are and against a fresh device build from those points."""
    w = W.MEDIUM
    g = H.generate(ctx, w.n, w.alpha, w.kbar, w.seed, fp64_only=fp64)
    R = g["stats"]["R"]
    r, phi, off, col = g["r"], g["phi"], g["row_off"], g["col_idx"]
    for step, k in enumerate((1, 100, 10_000)):
        ids, rn, pn = W.moves(_np(r), _np(phi), R, k, 50 + step)
        exp_r, exp_phi = _np(r).copy(), _np(phi).copy()
        exp_r[ids], exp_phi[ids] = rn, pn
        u = H.update_points(ctx, r, phi, off, col, R, torch.tensor(ids), torch.tensor(rn), torch.tensor(pn),
                            fp64_only=fp64)
        assert np.array_equal(_np(r), exp_r) and np.array_equal(_np(phi), exp_phi)
        o_off, o_col, ties = _oracle(exp_r, exp_phi, R)
        _assert_matches(_np(u["row_off"]), _np(u["col_idx"]), o_off, o_col, ties)
        _check_rows(_np(u["row_off"]), _np(u["col_idx"]))
        assert u["stats"]["ties"] == 0
        fresh = H.generate_from_points(ctx, r, phi, R, fp64_only=fp64)
        assert torch.equal(fresh["row_off"], u["row_off"]) and torch.equal(fresh["col_idx"], u["col_idx"])
        off, col = u["row_off"], u["col_idx"]


@pytest.mark.parametrize("k", [1, 700, 1500, 3000])
def test_updates_of_a_small_graph_match_brute_force(ctx, k):
    """n = 3000 (alpha 0.55, kbar 16): a single vertex, a quarter, half and
    all of the vertices move; the result against the all-pairs oracle."""
    n, alpha, kbar, seed = 3000, 0.55, 16.0, 9
    g = H.generate(ctx, n, alpha, kbar, seed)
    R = g["stats"]["R"]
    r, phi = g["r"], g["phi"]
    ids, rn, pn = W.moves(_np(r), _np(phi), R, k, 7 + k)
    u = H.update_points(ctx, r, phi, g["row_off"], g["col_idx"], R, torch.tensor(ids), torch.tensor(rn),
                        torch.tensor(pn))
    o_off, o_col, ties = _oracle(_np(r), _np(phi), R)
    _assert_matches(_np(u["row_off"]), _np(u["col_idx"]), o_off, o_col, ties)
    # and back again: the same vertices moved to their first places (the
    # oracle's radii, within 8 ulp of the device's) give the first graph again
    r0, phi0 = O.sample(n, alpha, R, seed)
    back = H.update_points(ctx, r, phi, u["row_off"], u["col_idx"], R, torch.tensor(ids), torch.tensor(r0[ids]),
                           torch.tensor(phi0[ids]))
    o_off, o_col, ties = _oracle(_np(r), _np(phi), R)
    _assert_matches(_np(back["row_off"]), _np(back["col_idx"]), o_off, o_col, ties)
    _assert_matches(_np(back["row_off"]), _np(back["col_idx"]), _np(g["row_off"]), _np(g["col_idx"]), ties)


def test_no_moves_copies_the_graph(ctx):
    w = W.scaled(W.LARGE, 200_000)
    g = H.generate(ctx, w.n, w.alpha, w.kbar, w.seed)
    e = torch.empty(0)
    u = H.update_points(ctx, g["r"], g["phi"], g["row_off"], g["col_idx"], g["stats"]["R"], e.to(torch.int32), e, e)
    assert torch.equal(u["row_off"], g["row_off"]) and torch.equal(u["col_idx"], g["col_idx"])


def test_update_of_the_large_workload_equals_a_fresh_build(ctx):
    """n = 1e8 (hub rows of millions of entries): 1000 moves, the update's
    CSR against the device's own build from the moved points (entry for
    entry); the sampled moved rows against the oracle's all-points scan."""
    w = W.LARGE
    g = H.generate(ctx, w.n, w.alpha, w.kbar, w.seed)
    R = g["stats"]["R"]
    r, phi = g["r"], g["phi"]
    sel = torch.randint(0, w.n, (1 << 16,), generator=torch.Generator().manual_seed(3))
    ids, rn, pn = W.moves(_np(r[sel.cuda()]), _np(phi[sel.cuda()]), R, 1000, 61)
    ids = _np(sel)[ids].astype(np.int32)
    ids, first = np.unique(ids, return_index=True)
    rn, pn = rn[first], pn[first]
    # two of them to the centre, where their rows hold millions of vertices
    rn[:2] = [0.5, 3.0]
    u = H.update_points(ctx, r, phi, g["row_off"], g["col_idx"], R, torch.tensor(ids), torch.tensor(rn),
                        torch.tensor(pn))
    del g
    fresh = H.generate_from_points(ctx, r, phi, R)
    assert torch.equal(fresh["row_off"], u["row_off"]) and torch.equal(fresh["col_idx"], u["col_idx"])
    del fresh
    rh, ph = _np(r), _np(phi)
    q = np.concatenate([ids[:2], ids[2::100]])
    cnt, o_off, rows = O.brute_rows(rh, ph, R, q)
    off = _np(u["row_off"])
    for i, v in enumerate(q):
        got = _np(u["col_idx"][int(off[v]):int(off[v + 1])])
        assert np.array_equal(got, rows[o_off[i]:o_off[i + 1]]), int(v)


def test_update_errors_leave_points_unchanged(ctx):
    n, alpha, kbar, seed = 5000, 0.8, 8.0, 5
    g = H.generate(ctx, n, alpha, kbar, seed)
    R = g["stats"]["R"]
    r0, p0 = g["r"].clone(), g["phi"].clone()
    bad = [
        ([3, 3], [1.0, 2.0], [0.1, 0.2]),          # a vertex twice
        ([3, n], [1.0, 2.0], [0.1, 0.2]),          # id out of range
        ([3, 4], [1.0, R], [0.1, 0.2]),            # radius at the rim
        ([3, 4], [1.0, -0.5], [0.1, 0.2]),         # negative radius
        ([3, 4], [1.0, 2.0], [0.1, 2 * math.pi]),  # angle 2 pi
        ([3, 4], [1.0, float("nan")], [0.1, 0.2]),
    ]
    for ids, rn, pn in bad:
        with pytest.raises(H.HrgError) as e:
            H.update_points(ctx, g["r"], g["phi"], g["row_off"], g["col_idx"], R, torch.tensor(ids, dtype=torch.int32),
                            torch.tensor(rn, dtype=torch.float64), torch.tensor(pn, dtype=torch.float64))
        assert e.value.code == H.HRG_EINVAL
        assert torch.equal(g["r"], r0) and torch.equal(g["phi"], p0)
    # the context still works
    u = H.update_points(ctx, g["r"], g["phi"], g["row_off"], g["col_idx"], R, torch.tensor([3], dtype=torch.int32),
                        torch.tensor([1.0], dtype=torch.float64), torch.tensor([0.1], dtype=torch.float64))
    o_off, o_col, ties = _oracle(_np(g["r"]), _np(g["phi"]), R)
    _assert_matches(_np(u["row_off"]), _np(u["col_idx"]), o_off, o_col, ties)
