"""The request server: results in the mix of a continuous batch equal the
results of the same requests generated alone; memory admission holds."""
import numpy as np
import pytest

from paper_1501_03545_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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
            res = srv.wait(t)
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
        assert c["completed"] == len(reqs) and c["queued"] == 0 and c["in_use_bytes"] == 0
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
            res = srv.wait(t)
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
        res = srv.wait(t)
        assert res.status == H.HRG_OK and res.n_entries > 0
        srv.release(t)
    finally:
        srv.close()
