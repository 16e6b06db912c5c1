"""Pins of the oracle's random long-range edges (Sec. 4.2) to things other
than itself: for n = 2^b the vertex of a 64-bit word is its top b bits; the
endpoints are uniform (chi-square); the merged graph equals the adjacency
matrix with the drawn pairs set, built densely."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("bits,seed", [(1, 3), (10, 5), (20, 2**40 + 7), (30, 11)])
def test_power_of_two_vertex_count_takes_top_bits(bits, seed):
    n = 1 << bits
    u, v = O.random_pairs(n, 200, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for k in range(200):
        x = O.philox([k & 0xFFFFFFFF, (k >> 32) | 0x80000000, 0, 0], key)
        a = (int(x[0]) << 32) | int(x[1])
        b = (int(x[2]) << 32) | int(x[3])
        assert u[k] == a >> (64 - bits) and v[k] == b >> (64 - bits)


def test_endpoints_uniform():
    stats = pytest.importorskip("scipy.stats")
    n, count = 1000, 200_000
    u, v = O.random_pairs(n, count, 17)
    assert u.min() >= 0 and v.min() >= 0 and u.max() < n and v.max() < n
    for x in (u, v):
        c = np.bincount(x, minlength=n)
        assert stats.chisquare(c).pvalue > 1e-4


def dense(off, col):
    n = len(off) - 1
    A = np.zeros((n, n), dtype=bool)
    for r in range(n):
        A[r, col[off[r]:off[r + 1]]] = True
    return A


@pytest.mark.parametrize("n,alpha,kbar,gseed,count,seed", [(1500, 0.8, 10.0, 4, 3000, 9), (60, 1.0, 6.0, 2, 4000, 1),
                                                            (800, 0.6, 12.0, 5, 0, 3)])
def test_merge_equals_dense_construction(n, alpha, kbar, gseed, count, seed):
    g = O.generate(n, alpha, kbar, gseed)
    A = dense(g["row_off"], g["col_idx"])
    before = int(A.sum()) // 2
    u, v = O.random_pairs(n, count, seed)
    keep = u != v
    A[u[keep], v[keep]] = True
    A[v[keep], u[keep]] = True
    off, col, added = O.add_random_edges(g["row_off"], g["col_idx"], count, seed)
    rows, cols = np.nonzero(A)
    ref_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=ref_off[1:])
    assert np.array_equal(off, ref_off)
    assert np.array_equal(col, cols.astype(np.int32))
    assert added == int(A.sum()) // 2 - before
    if n == 60:
        assert added < count // 2  # repeats and present edges were dropped
