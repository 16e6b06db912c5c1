"""Parity of the device's random long-range edges (Sec. 4.2,
hrg_add_random_edges through the C ABI) with the oracle: the merged CSR and
the added-edge count bit-identical on the oracle's own graphs, in a batch's
shared CSR, on tiny vertex sets (many repeats and self-pairs), and the
appendix's claim that 0.5 % random edges leave the clustering and the degree
tail nearly unchanged on the 1e6-vertex workload."""
import ctypes
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


def dev(off, col):
    return (torch.from_numpy(np.asarray(off, dtype=np.int64)).cuda(),
            torch.from_numpy(np.asarray(col, dtype=np.int32)).cuda())


@pytest.mark.parametrize("n,alpha,kbar,gseed", [(20_000, 0.8, 10.0, 3), (60, 1.0, 6.0, 2), (5_000, 0.55, 16.0, 8)])
@pytest.mark.parametrize("frac,seed", [(0.0, 1), (0.005, 7), (0.05, 2**63 + 5), (3.0, 11)])
def test_matches_oracle(ctx, n, alpha, kbar, gseed, frac, seed):
    g = O.generate(n, alpha, kbar, gseed)
    m = int(g["row_off"][-1]) // 2
    count = int(math.ceil(frac * m))
    ref_off, ref_col, ref_added = O.add_random_edges(g["row_off"], g["col_idx"], count, seed)
    out = H.add_random_edges(ctx, *dev(g["row_off"], g["col_idx"]), count=count, seed=seed)
    assert out["added"] == ref_added
    assert np.array_equal(out["row_off"].cpu().numpy(), ref_off)
    assert np.array_equal(out["col_idx"].cpu().numpy(), ref_col)


def test_single_vertex_and_empty_graph(ctx):
    for n in (1, 2, 7):
        off = np.zeros(n + 1, dtype=np.int64)
        col = np.zeros(0, dtype=np.int32)
        ref_off, ref_col, ref_added = O.add_random_edges(off, col, 25, 4)
        out = H.add_random_edges(ctx, torch.from_numpy(off).cuda(), None, count=25, seed=4)
        assert out["added"] == ref_added
        assert np.array_equal(out["row_off"].cpu().numpy(), ref_off)
        assert np.array_equal(out["col_idx"].cpu().numpy(), ref_col)


def test_graph_of_a_batch(ctx):
    items = [(3000, 0.8, 10.0, 101), (5000, 0.6, 16.0, 102)]
    b = H.generate_batch(ctx, items)
    for k, it in enumerate(items):
        lo, hi = b["goff"][k], b["goff"][k + 1]
        a = H.add_random_edges(ctx, b["row_off"][lo:hi + 1], b["col_idx"], count=400, seed=k)
        s = H.generate(ctx, *it)
        ref = H.add_random_edges(ctx, s["row_off"], s["col_idx"], count=400, seed=k)
        assert a["added"] == ref["added"]
        assert torch.equal(a["row_off"], ref["row_off"]) and torch.equal(a["col_idx"], ref["col_idx"])


def test_errors(ctx):
    g = O.generate(2000, 0.8, 10.0, 1)
    off, col = dev(g["row_off"], g["col_idx"])
    L = H.load()
    n = off.numel() - 1
    o = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    c = torch.empty(10, dtype=torch.int32, device="cuda")
    ne, added = ctypes.c_int64(), ctypes.c_int64()
    rc = L.hrg_add_random_edges(ctx.h, n, ctypes.c_void_p(off.data_ptr()), ctypes.c_void_p(col.data_ptr()), 100, 3,
                                None, ctypes.c_void_p(o.data_ptr()), ctypes.c_void_p(c.data_ptr()), 10,
                                ctypes.byref(ne), ctypes.byref(added))
    assert rc == H.HRG_EOVERFLOW and ne.value == int(g["row_off"][-1]) + 2 * added.value
    rc = L.hrg_add_random_edges(ctx.h, n, ctypes.c_void_p(off.data_ptr()), ctypes.c_void_p(col.data_ptr()), -1, 3,
                                None, ctypes.c_void_p(o.data_ptr()), ctypes.c_void_p(c.data_ptr()), 10,
                                ctypes.byref(ne), ctypes.byref(added))
    assert rc == H.HRG_EINVAL


def test_appendix_claim_on_the_1e6_workload(ctx):
    """0.5 % random edges on graphs of average degree 10: the clustering
    coefficient changes by less than 0.03 and the degree tail stays put."""
    w = W.MEDIUM
    g = H.generate(ctx, w.n, w.alpha, w.kbar, w.seed)
    m = g["col_idx"].numel() // 2
    lr = H.add_random_edges(ctx, g["row_off"], g["col_idx"], count=int(math.ceil(0.005 * m)), seed=99)
    assert 0.99 * 0.005 * m < lr["added"] <= 0.005 * m + 1
    p0 = H.graph_props(ctx, g["row_off"], g["col_idx"], d_min=30)
    p1 = H.graph_props(ctx, lr["row_off"], lr["col_idx"], d_min=30)
    assert abs(p1["avg_local_clustering"] - p0["avg_local_clustering"]) < 0.03
    assert abs(p1["clustering"] - p0["clustering"]) < 0.03
    assert abs(p1["gamma"] - p0["gamma"]) < 0.02
