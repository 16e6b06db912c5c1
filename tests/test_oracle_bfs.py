"""Pins of the oracle's breadth-first search and diameter bounds (Sec. 4.1's
longest shortest path) to things other than itself: hop distances against
scipy's unweighted shortest paths; the bounds against the exact diameter
from all-pairs shortest paths (equal on trees, where a double sweep is
exact; bracketing it elsewhere); closed forms of paths, cycles and stars."""
import numpy as np
import pytest

import oracle as O


def csr(n, edges):
    rows = [[] for _ in range(n)]
    for u, v in edges:
        rows[u].append(v)
        rows[v].append(u)
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([w for r in rows for w in sorted(r)], dtype=np.int32)
    return off, col


def all_pairs(off, col):
    sp = pytest.importorskip("scipy.sparse")
    cg = pytest.importorskip("scipy.sparse.csgraph")
    n = len(off) - 1
    A = sp.csr_matrix((np.ones(len(col)), col, off), shape=(n, n))
    return cg.shortest_path(A, unweighted=True, directed=False)


@pytest.mark.parametrize("n", [2, 3, 10, 57])
def test_path_cycle_star(n):
    off, col = csr(n, [(i, i + 1) for i in range(n - 1)])
    lo, hi, _, size = O.diameter_bounds(off, col)
    assert lo == n - 1 and size == n and hi >= n - 1
    if n >= 3:
        off, col = csr(n, [(i, (i + 1) % n) for i in range(n)])
        lo, hi, _, _ = O.diameter_bounds(off, col)
        assert lo == n // 2 and hi == 2 * (n // 2)
        off, col = csr(n, [(0, i) for i in range(1, n)])
        assert O.diameter_bounds(off, col)[:2] == (2, 2)


@pytest.mark.parametrize("seed", range(5))
def test_random_trees_exact(seed):
    rng = np.random.default_rng(seed)
    n = 300
    edges = [(int(rng.integers(0, v)), v) for v in range(1, n)]
    off, col = csr(n, edges)
    D = all_pairs(off, col)
    lo, hi, _, size = O.diameter_bounds(off, col, sweeps=2)
    assert lo == int(D.max()) and size == n and lo <= hi


@pytest.mark.parametrize("seed", range(4))
def test_bounds_bracket_diameter_and_distances_match(seed):
    rng = np.random.default_rng(100 + seed)
    n = 160
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.015]
    off, col = csr(n, edges)
    D = all_pairs(off, col)
    root = int(np.argmax(np.diff(off)))
    comp = np.isfinite(D[root])
    lo, hi, roots, size = O.diameter_bounds(off, col)
    exact = int(D[np.ix_(comp, comp)].max())
    assert lo <= exact <= hi and size == int(comp.sum()) and roots[0] == root
    for s in (0, root, n - 1):
        dist, ecc = O.bfs(off, col, s)
        ref = np.where(np.isfinite(D[s]), D[s], -1).astype(np.int64)
        assert np.array_equal(dist, ref) and ecc == int(ref.max())


def test_hyperbolic_graph_distances():
    g = O.generate(3000, 0.8, 8.0, 6)
    D = all_pairs(g["row_off"], g["col_idx"])
    for s in (0, 17, 2999):
        dist, _ = O.bfs(g["row_off"], g["col_idx"], s)
        assert np.array_equal(dist, np.where(np.isfinite(D[s]), D[s], -1).astype(np.int64))
