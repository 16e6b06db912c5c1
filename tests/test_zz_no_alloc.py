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


def _cumsum_offsets(deg):
    """Independent reference: torch's own prefix sum, with the leading 0."""
    ref = torch.zeros(deg.numel() + 1, dtype=torch.int64, device=deg.device)
    ref[1:] = torch.cumsum(deg.to(torch.int64), 0)
    return ref


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
            assert torch.equal(out, _cumsum_offsets(deg))
    finally:
        ctx.close()


def test_noalloc_two_level_scan_matches_cumsum(H):
    """Sizes above 4096 tiles of 4096 degrees run the scan's second level
    from the static scratch too: two calls in a row with different contents
    (and the largest size the scratch admits) against torch.cumsum."""
    g = torch.Generator(device="cuda").manual_seed(11)
    for n in ((1 << 24) + 12345, (1 << 28)):
        for hi in (40, 3):
            deg = torch.randint(0, hi, (n,), device="cuda", dtype=torch.int32, generator=g)
            out = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
            assert H.hrg_row_offsets_noalloc(deg, out) == H.HRG_OK
            torch.cuda.synchronize()
            assert torch.equal(out, _cumsum_offsets(deg)), (n, hi)
            del deg, out


def test_noalloc_binding_checks_arguments(H):
    deg = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        H.hrg_row_offsets_noalloc(deg, torch.zeros(10, dtype=torch.int64, device="cuda"))  # too short
    with pytest.raises(ValueError):
        H.hrg_row_offsets_noalloc(deg.to(torch.int64), torch.zeros(11, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        H.hrg_row_offsets_noalloc(deg, torch.zeros(11, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        H.hrg_row_offsets_noalloc(deg[::2], torch.zeros(6, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        H.hrg_row_offsets_noalloc(deg.cpu(), torch.zeros(11, dtype=torch.int64))


def test_noalloc_rejects_sizes_beyond_maximum(H):
    L = H.load()
    import ctypes

    dummy = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = L.hrg_row_offsets_noalloc(ctypes.c_void_p(dummy.data_ptr()), (1 << 28) + 1,
                                   ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == H.HRG_EINVAL
    rc = L.hrg_row_offsets_noalloc(None, 10, ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == H.HRG_EINVAL
