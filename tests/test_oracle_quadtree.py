"""The paper's own generator (Algorithm 1 with the polar quadtree of Sec. 3),
kept as a second CPU baseline: its graphs equal the oracle's brute force
where FP64 resolves the Poincare disk, its radial splits give every depth-3
cell a 4^-3 share of the points (Lemma 4), and Proposition 1's circle meets
the query's ray at hyperbolic distance R on both sides."""
import math

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("n,alpha,kbar,seed,cap,R", [(3000, 0.6, 16.0, 1, 1, None), (10_000, 1.0, 6.0, 1, 64, None),
                                                     (20_000, 0.75, 10.0, 2, 64, None),
                                                     (20_000, 0.55, 16.0, 3, 7, None), (2, 0.8, 1.0, 5, 1, 3.0),
                                                     (500, 0.8, 40.0, 4, 3, None), (3000, 0.9, 0.0, 6, 16, 2.0)])
def test_equals_brute_force(n, alpha, kbar, seed, cap, R):
    g = O.generate(n, alpha, kbar, seed, method="brute", R=R)
    off, col, _ = O.quadtree_csr(g["r"], g["phi"], g["R"], alpha, cap)
    assert np.array_equal(off, g["row_off"])
    assert np.array_equal(col, g["col_idx"])


def test_depth3_cells_hold_equal_mass():
    stats = pytest.importorskip("scipy.stats")
    n, alpha = 200_000, 0.8
    R = O.solve_radius(n, alpha, 10.0)
    r, phi = O.sample(n, alpha, R, 12)
    counts = O.quadtree_depth_counts(r, phi, R, alpha, 3, capacity=1)
    assert counts.sum() == n
    assert stats.chisquare(counts).pvalue > 1e-4


@pytest.mark.parametrize("R,rh", [(10.0, 0.5), (10.0, 7.0), (12.0, 3.0), (6.0, 5.5), (8.0, 1.0), (3.0, 9.0)])
def test_proposition1_circle_meets_ray_at_distance_R(R, rh):
    # radii up to rh + R = 17, where FP64 still resolves the disk (1 - r_E ~ 1e-7)
    c, rad = O.quadtree_circle(R, 1.3, rh)
    out_e = c + rad  # the boundary point beyond the query on its ray
    assert abs(2 * math.atanh(out_e) - rh - R) < 1e-6 * R
    in_e = c - rad   # the other boundary point: on the ray, or through the origin
    if in_e >= 0:
        assert abs(rh - 2 * math.atanh(in_e) - R) < 1e-6 * R
    else:
        assert abs(rh + 2 * math.atanh(-in_e) - R) < 1e-6 * R
