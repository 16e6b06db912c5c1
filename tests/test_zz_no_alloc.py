"""The allocation-free row-offset entry point (hrg_row_offsets_noalloc).

Some callers cannot allocate device memory (they run inside a framework that
owns all device memory through its own pool, or under a fixed memory budget).
This entry computes CSR row offsets from degrees using scratch compiled into
the library.  Its output must equal the row offsets that the allocating
generator (hrg_generate_begin) produced for the same degrees, on two calls in
a row over different inputs (the shared scratch keeps the previous call's
contents).  This file is collected last so a stop-at-first-failure run has
already run every other test.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_03545_gb300 import _lib

    return _lib


def test_noalloc_row_offsets_match_generator(H):
    ctx = H.Context(0)
    try:
        # two different graphs: the second call must not see the first call's scratch
        cases = [(3_000_000, 0.55, 16.0, 3), (250_001, 0.75, 10.0, 2)]
        for n, alpha, kbar, seed in cases:
            g = H.generate(ctx, n, alpha, kbar, seed)
            ref = g["row_off"]
            deg = (ref[1:] - ref[:-1]).to(torch.int32).contiguous()
            out = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
            rc = H.hrg_row_offsets_noalloc(deg, out)
            assert rc == H.HRG_OK
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (n, int((out != ref).sum()))
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_maximum(H):
    L = H.load()
    import ctypes

    dummy = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = L.hrg_row_offsets_noalloc(ctypes.c_void_p(dummy.data_ptr()), (1 << 28) + 1,
                                   ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == H.HRG_EINVAL
    rc = L.hrg_row_offsets_noalloc(None, 10, ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == H.HRG_EINVAL
