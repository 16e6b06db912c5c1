"""Pins of the oracle's graph properties (Sec. 4.1) to things other than
itself: closed forms of complete graphs, stars and cycles; matrix powers of
the adjacency matrix (triangles = trace(A^3)/6, triangles at v = (A^3)_vv / 2,
triads = paths of length two = (sum(A^2) - trace(A^2)) / 2); and the exact
discrete maximum-likelihood exponent of a zeta-distributed sample (Hurwitz
zeta likelihood maximised numerically) for the tail-exponent approximation."""
import math

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


def adjacency(off, col):
    n = len(off) - 1
    A = np.zeros((n, n))
    for v in range(n):
        A[v, col[off[v]:off[v + 1]]] = 1.0
    return A


@pytest.mark.parametrize("n", range(1, 13))
def test_complete_graph(n):
    off, col = csr(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    p = O.graph_props(off, col, 1)
    assert p["triangles"] == math.comb(n, 3)
    assert p["triads"] == n * math.comb(n - 1, 2)
    assert p["max_degree"] == n - 1
    assert p["entries"] == n * (n - 1)
    assert list(p["triangles_per_vertex"]) == [math.comb(n - 1, 2)] * n
    if n >= 3:
        assert p["clustering"] == 1.0 and p["avg_local_clustering"] == 1.0
    else:
        assert math.isnan(p["clustering"]) and p["avg_local_clustering"] == 0.0


@pytest.mark.parametrize("k", [1, 2, 5, 40])
def test_star(k):
    off, col = csr(k + 1, [(0, i) for i in range(1, k + 1)])
    p = O.graph_props(off, col, 1)
    assert p["triangles"] == 0 and p["triads"] == math.comb(k, 2)
    assert p["avg_local_clustering"] == 0.0
    assert (p["clustering"] == 0.0) if k >= 2 else math.isnan(p["clustering"])


@pytest.mark.parametrize("n", range(3, 11))
def test_cycle(n):
    off, col = csr(n, [(i, (i + 1) % n) for i in range(n)])
    p = O.graph_props(off, col, 1)
    assert p["triads"] == n
    assert p["triangles"] == (1 if n == 3 else 0)


def test_empty_and_edgeless():
    off, col = csr(5, [])
    p = O.graph_props(off, col, 1)
    assert p["triangles"] == 0 and p["triads"] == 0 and p["entries"] == 0
    assert math.isnan(p["clustering"]) and math.isnan(p["gamma"])


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_random_graphs_against_matrix_powers(seed):
    rng = np.random.default_rng(seed)
    n = 90
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.12 + 0.05 * seed]
    off, col = csr(n, edges)
    p = O.graph_props(off, col, 3)
    A = adjacency(off, col)
    A2 = A @ A
    A3 = A2 @ A
    assert p["triangles"] == round(np.trace(A3) / 6)
    assert np.array_equal(p["triangles_per_vertex"], np.round(np.diag(A3) / 2).astype(np.int64))
    assert p["triads"] == round((A2.sum() - np.trace(A2)) / 2)


def test_hyperbolic_graph_against_matrix_powers():
    g = O.generate(1500, 0.75, 10.0, 11)
    off, col = g["row_off"], g["col_idx"]
    p = O.graph_props(off, col, 5)
    A = adjacency(off, col)
    A2 = A @ A
    A3 = A2 @ A
    assert p["triangles"] == round(np.trace(A3) / 6) and p["triangles"] > 1000
    assert np.array_equal(p["triangles_per_vertex"], np.round(np.diag(A3) / 2).astype(np.int64))
    assert p["triads"] == round((A2.sum() - np.trace(A2)) / 2)
    d = A.sum(axis=1)
    assert p["tail_count"] == int((d >= 5).sum())
    assert p["max_degree"] == int(d.max())


def test_tail_exponent_against_exact_discrete_mle():
    special = pytest.importorskip("scipy.special")
    optimize = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(7)
    gamma_true, d_min = 2.5, 10
    deg = rng.zipf(gamma_true, size=4_000_000)
    deg = deg[deg >= d_min].astype(np.int64)
    off = np.zeros(len(deg) + 1, dtype=np.int64)
    off[1:] = np.cumsum(deg)
    p = O.graph_props(off, np.zeros(0, dtype=np.int32), d_min, triangles=False)
    assert p["tail_count"] == len(deg)
    # exact discrete MLE: maximise -gamma sum ln d - N ln zeta(gamma, d_min)
    sl = np.log(deg.astype(np.float64)).sum()
    N = len(deg)
    res = optimize.minimize_scalar(lambda g: g * sl + N * math.log(special.zeta(g, d_min)),
                                   bounds=(1.5, 4.0), method="bounded", options={"xatol": 1e-8})
    assert abs(res.x - gamma_true) < 0.02, res.x
    assert abs(p["gamma"] - res.x) < 0.01, (p["gamma"], res.x)
