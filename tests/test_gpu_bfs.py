"""Parity of the device breadth-first search and diameter bounds (hrg_bfs,
hrg_diameter_bounds through the C ABI) with the oracle on the oracle's own
graphs, and Sec. 4.2's claim that 0.5 % random long-range edges shorten the
diameter of a graph of average degree 10 (here gamma = 3: from 44-46 hops
to 27-30)."""
import math

import numpy as np
import pytest

import oracle as O

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


def dev(off, col):
    return (torch.from_numpy(np.asarray(off, dtype=np.int64)).cuda(),
            torch.from_numpy(np.asarray(col, dtype=np.int32)).cuda())


@pytest.mark.parametrize("n,alpha,kbar,seed", [(20_000, 0.75, 10.0, 2), (100_000, 1.0, 6.0, 3), (3000, 1.4, 4.0, 5)])
def test_bfs_and_bounds_match_oracle(ctx, n, alpha, kbar, seed):
    g = O.generate(n, alpha, kbar, seed)
    off, col = dev(g["row_off"], g["col_idx"])
    deg = np.diff(g["row_off"])
    for s in (-1, 0, n - 1, int(np.argmin(deg))):
        dist, ecc, reached, far, src = H.bfs(ctx, off, col, s)
        ref, ref_ecc = O.bfs(g["row_off"], g["col_idx"], src)
        assert src == (int(np.argmax(deg)) if s < 0 else s)
        assert np.array_equal(dist.cpu().numpy(), ref)
        assert ecc == ref_ecc and reached == int((ref >= 0).sum())
        assert far == int(np.flatnonzero(ref == ref_ecc)[0])
    assert H.diameter_bounds(ctx, off, col) == tuple(O.diameter_bounds(g["row_off"], g["col_idx"]))


def test_edgeless_and_single_vertex(ctx):
    for n in (1, 5):
        off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
        dist, ecc, reached, far, src = H.bfs(ctx, off, None, -1)
        assert ecc == 0 and reached == 1 and far == src == 0
        assert dist.cpu().tolist() == [0] + [-1] * (n - 1)
        assert H.diameter_bounds(ctx, off, None) == (0, 0, [0], 1)


def test_invalid_arguments(ctx):
    g = O.generate(500, 0.8, 8.0, 1)
    off, col = dev(g["row_off"], g["col_idx"])
    with pytest.raises(H.HrgError) as e:
        H.bfs(ctx, off, col, 500)
    assert e.value.code == H.HRG_EINVAL
    with pytest.raises(H.HrgError) as e:
        H.diameter_bounds(ctx, off, col, sweeps=0)
    assert e.value.code == H.HRG_EINVAL


def test_long_range_edges_shorten_the_diameter(ctx):
    """Sec. 4.2 / appendix: adding 0.5 % random edges to a graph of average
    degree 10 shortens its diameter (the paper: by about half)."""
    n, alpha, kbar, seed = 200_000, 1.0, 10.0, 4
    g = H.generate(ctx, n, alpha, kbar, seed)
    m = g["col_idx"].numel() // 2
    lr = H.add_random_edges(ctx, g["row_off"], g["col_idx"], count=int(math.ceil(0.005 * m)), seed=99)
    lo0, hi0, _, size0 = H.diameter_bounds(ctx, g["row_off"], g["col_idx"])
    lo1, hi1, _, size1 = H.diameter_bounds(ctx, lr["row_off"], lr["col_idx"])
    assert size1 >= size0 > 0.9 * n
    assert hi1 < lo0 and lo1 <= 0.7 * lo0, (lo0, hi0, lo1, hi1)
