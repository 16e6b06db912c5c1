"""The request server: results in the mix of a continuous batch equal the
results of the same requests generated alone; memory admission holds."""
import numpy as np
import pytest

from paper_1501_03545_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# a bound on every wait, so that a request that never runs fails the test
# instead of holding it
WAIT_S = 300.0


@pytest.fixture(scope="module")
def H():
    import torch

    from paper_1501_03545_gb300 import _lib

    assert torch.cuda.is_available()
    _lib.load()
    return _lib


def _alone(H, ctx, n, alpha, kbar, seed):
    g = H.generate(ctx, n, alpha, kbar, seed)
    return (g["r"].cpu().numpy(), g["phi"].cpu().numpy(), g["row_off"].cpu().numpy(), g["col_idx"].cpu().numpy())


def test_mix_equals_alone(H):
    reqs = W.serving_requests(40, n_hi=4e5, draw_seed=3)
    srv = H.Server(0, slots=2)
    ctx = H.Context(0)
    try:
        tickets = [srv.submit(n, a, k, s) for (_, n, a, k, s) in reqs]
        sizes = []
        for t, (_, n, a, k, s) in zip(tickets, reqs):
            res = srv.wait(t, timeout_s=WAIT_S)
            assert res.status == H.HRG_OK, srv.last_error()
            assert res.n == n
            sizes.append(res.batch_size)
            r, phi, off, col = srv.fetch(res)
            r1, phi1, off1, col1 = _alone(H, ctx, n, a, k, s)
            assert np.array_equal(phi, phi1) and np.array_equal(r, r1)
            assert np.array_equal(off, off1)
            assert np.array_equal(col, col1)
            srv.release(t)
        assert max(sizes) > 1  # some requests really ran batched with others
        c = srv.counters()
        # released: only the workers' resident workspaces stay counted
        assert c["completed"] == len(reqs) and c["queued"] == 0 and c["in_use_bytes"] == c["resident_bytes"] > 0
    finally:
        ctx.close()
        srv.close()


def test_memory_admission(H):
    # a budget that holds about two of these requests at a time
    n, kbar = 200_000, 16.0
    per = 16 * n + 8 * (n + 1) + 4 * 1.1 * kbar * n + 160 * n + 4 * 1.1 * kbar * n
    srv = H.Server(0, slots=3, mem_budget_bytes=int(2.5 * per))
    try:
        with pytest.raises(H.HrgError) as e:
            srv.submit(3_000_000, 0.8, 16.0, 1)
        assert e.value.code == H.HRG_ENOMEM
        tickets = [srv.submit(n, 0.8, kbar, 100 + k) for k in range(8)]
        for t in tickets:
            res = srv.wait(t, timeout_s=WAIT_S)
            assert res.status == H.HRG_OK
            assert res.batch_size <= 2
            srv.release(t)
        c = srv.counters()
        assert c["peak_in_use_bytes"] <= c["budget_bytes"]
        assert c["completed"] == 8
    finally:
        srv.close()


def test_unknown_ticket_and_timeout(H):
    srv = H.Server(0, slots=1)
    try:
        with pytest.raises(H.HrgError):
            srv.wait(12345)
        t = srv.submit(5_000_000, 0.6, 24.0, 9)
        try:
            srv.wait(t, timeout_s=0.0)
        except TimeoutError:
            pass  # still running: the limit was respected
        res = srv.wait(t, timeout_s=WAIT_S)
        assert res.status == H.HRG_OK and res.n_entries > 0
        srv.release(t)
    finally:
        srv.close()


def test_served_graphs_equal_the_oracle(H):
    """A few served graphs (of a mixed batch) against the oracle's all-pairs
    CSR directly, not through a single-graph call."""
    import oracle as O

    reqs = [(3000, 0.6, 12.0, 71), (5000, 1.1, 6.0, 72), (2500, 0.9, 24.0, 73), (4000, 0.55, 16.0, 74)]
    srv = H.Server(0, slots=1)
    try:
        tickets = [srv.submit(n, a, k, sd) for (n, a, k, sd) in reqs]
        for t, (n, a, k, sd) in zip(tickets, reqs):
            res = srv.wait(t, timeout_s=WAIT_S)
            assert res.status == H.HRG_OK
            r, phi, off, col = srv.fetch(res)
            R = O.solve_radius(n, a, k)
            ro, po = O.sample(n, a, R, sd)
            assert np.array_equal(phi, po)
            o_off, o_col = O.brute_csr(ro, po, R)
            nt, _ = O.brute_ties(ro, po, R)
            assert nt == 0
            assert np.array_equal(off, o_off) and np.array_equal(col, o_col)
            srv.release(t)
    finally:
        srv.close()


def test_admission_counts_resident_workspace(H):
    """Two workers run a large request, then small ones.  Each worker's
    workspace stays resident after its batch, so the counted bytes must
    cover the real drop of free device memory (cudaMemGetInfo), and a budget
    too small for the next request beside the resident workspaces makes the
    idle workers free theirs instead of overcommitting."""
    import torch

    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    srv = H.Server(0, slots=2)
    try:
        big = srv.submit(6_000_000, 0.6, 16.0, 5)
        res = srv.wait(big, timeout_s=WAIT_S)
        assert res.status == H.HRG_OK
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        c = srv.counters()
        assert c["resident_bytes"] > 0
        # what the server counts covers what the device lost (pool granularity aside)
        assert c["peak_in_use_bytes"] >= (free0 - free1) - (256 << 20), (c, free0 - free1)
        srv.release(big)
        small = [srv.submit(50_000 + 1000 * k, 0.8, 8.0, 20 + k) for k in range(6)]
        for t in small:
            assert srv.wait(t, timeout_s=WAIT_S).status == H.HRG_OK
            srv.release(t)
        c = srv.counters()
        assert c["in_use_bytes"] == c["resident_bytes"] and c["peak_in_use_bytes"] <= c["budget_bytes"]
    finally:
        srv.close()
    # a budget that holds one large request but not a second one beside a resident workspace
    n = 3_000_000
    per = 16 * n + 8 * (n + 1) + 4 * (1.1 * 16.0 * n + 1024) + 250 * n + 4 * (1.1 * 16.0 * n + 1024) + (1 << 26)
    srv = H.Server(0, slots=2, mem_budget_bytes=int(1.6 * per))
    try:
        for k in range(4):
            t = srv.submit(n, 0.6, 16.0, 40 + k)
            assert srv.wait(t, timeout_s=WAIT_S).status == H.HRG_OK
            srv.release(t)
        c = srv.counters()
        assert c["completed"] == 4 and c["peak_in_use_bytes"] <= c["budget_bytes"]
    finally:
        srv.close()
