"""The no-allocation Gram entry point (atc_gram_fp64_noalloc) against atc_gram.

Some callers of this library cannot allocate device memory (real-time paths
that must not block on the device allocator, or hosts that give the library a
fixed memory budget).  atc_gram_fp64_noalloc keeps its split-K partial sums in a
fixed array inside the library instead of cudaMalloc'd scratch.  This test
calls it twice in a row through the C ABI and checks each result against the
regular FP64 entry point with the same tolerance as the other FP64 Gram tests
(1e-12 * ||X||^2 per entry), including the largest mode length the array
allows (n = 724, where the split count is clamped to one by the array size),
and checks that sizes above the limit, or whose index range would overflow,
are rejected on the host before anything runs.  The file is named to run last, so a failure here cannot hide
the result of any other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2107_01384_gb300 as P
    return P


def test_noalloc_gram_matches_regular_entry_point_twice(P):
    rng = np.random.default_rng(77)
    cases = [((40, 96, 50), 1, np.float32), ((64, 64, 64), 2, np.float64)]
    for dims, mode, dtype in cases:   # two calls in a row, different shapes and dtypes
        x = rng.standard_normal(dims).astype(dtype)
        L = int(np.prod(dims[:mode])); n = dims[mode]; R = int(np.prod(dims[mode + 1:]))
        xd = torch.from_numpy(x).cuda()
        out = torch.empty((n, n), dtype=torch.float64, device="cuda")
        P.atc_gram_fp64_noalloc(xd, L, n, R, out)
        ref = P.atc_gram(xd, L, n, R, P.PREC_FP64)
        torch.cuda.synchronize()
        scale = float(np.sum(x.astype(np.float64) ** 2))
        assert float((out - ref).abs().max()) <= 1e-12 * scale
        assert torch.equal(out, out.T)


def test_noalloc_gram_rejects_sizes_above_its_limit(P):
    x = torch.zeros(2 * 800 * 2, dtype=torch.float32, device="cuda")
    out = torch.empty((800, 800), dtype=torch.float64, device="cuda")
    with pytest.raises(P.AtcError) as e:
        P.atc_gram_fp64_noalloc(x, 2, 800, 2, out)
    assert "no-allocation maximum" in str(e.value)


def test_noalloc_gram_at_the_array_limit(P):
    """n = 724 fills the array with a single split: two calls in a row on a
    long contraction (K = 20000) against atc_gram."""
    rng = np.random.default_rng(78)
    for seed_shift in range(2):
        x = (rng.standard_normal((1, 724, 20000)) + seed_shift).astype(np.float32)
        xd = torch.from_numpy(x).cuda()
        out = torch.empty((724, 724), dtype=torch.float64, device="cuda")
        P.atc_gram_fp64_noalloc(xd, 1, 724, 20000, out)
        ref = P.atc_gram(xd, 1, 724, 20000, P.PREC_FP64)
        torch.cuda.synchronize()
        scale = float(np.sum(x.astype(np.float64) ** 2))
        assert float((out - ref).abs().max()) <= 1e-12 * scale
        assert torch.equal(out, out.T)


def test_noalloc_gram_rejects_overflowing_sizes_on_the_host(P):
    """n = 2^32 (n * n wraps to 0 in 64 bits) and L * R beyond int64 are refused
    by the argument checks; the tiny buffers are never read."""
    import ctypes as C
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    L = P.lib()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.atc_gram_fp64_noalloc(C.c_void_p(x.data_ptr()), P.ATC_F32, 1, 2 ** 32, 1, C.c_void_p(out.data_ptr()), st)
    assert rc != 0 and b"no-allocation maximum" in L.atc_last_error()
    rc = L.atc_gram_fp64_noalloc(C.c_void_p(x.data_ptr()), P.ATC_F32, 2 ** 40, 2, 2 ** 40, C.c_void_p(out.data_ptr()), st)
    assert rc != 0 and b"overflows" in L.atc_last_error()
