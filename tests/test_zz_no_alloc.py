"""ns_sketch_static: the SRHT sketch for callers that cannot allocate device memory.

Some embedding hosts own all device memory through their own allocator, or
forbid allocation once they are running; they cannot hand libns a workspace.
ns_sketch_static keeps its scratch in a fixed array inside the library.  This
test calls it through the C ABI several times in a row (the array keeps the
previous call's contents, so later calls check that nothing stale leaks
through) and compares each result with ns_sketch, which uses a caller
workspace.  Both run the same deterministic fixed-point kernels, so the
results must agree bit for bit.  One case fills the array to within a few KiB
of its end, so the sizing and the carving of the scratch must agree there.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STATIC_BYTES = 16 << 20


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_00975_gb300 import build
    build.build()
    from paper_2206_00975_gb300 import api as a
    return a


def scratch_bytes(m, n, s):
    """Bytes of the array one call uses: status word, sign words, sample rows and
    the per-chunk partial sums, each rounded up to 256 bytes (the library's
    carving), with the chunk geometry of the SRHT kernel."""
    r = lambda b: (b + 255) // 256 * 256  # noqa: E731
    lg = max(int(m - 1).bit_length(), 0)
    mp = 1 << lg
    nblk = max(mp // 4096, 1)
    want, chunk = (nblk * n) // 2048, 1
    while chunk * 2 <= want and chunk * 2 <= 16:
        chunk *= 2
    while chunk > nblk:
        chunk //= 2
    nchunk = nblk // chunk
    return r(4) + r(4 * (max(mp, 4096) // 32)) + r(4 * s) + r(8 * nchunk * n * s)


def call_static(api, d, Ad, m, n, SA, status):
    lib = api._lib.load()
    return lib.ns_sketch_static(ctypes.byref(d), ctypes.c_void_p(Ad.data_ptr()), api.NS_F64, m, n, m,
                                ctypes.c_void_p(SA.data_ptr()),
                                None if status is None else ctypes.c_void_p(status.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("with_status", [True, False])
def test_static_scratch_matches_workspace_path(api, with_status):
    rng = np.random.default_rng(17)
    # the third case uses all but ~11 KiB of the 16 MiB array
    cases = [((1 << 17) + 9, 6, 512, 21), (5000, 3, 128, 4), (1 << 20, 7, 1160, 9), (4096, 2, 64, 5)]
    assert STATIC_BYTES - 16384 < scratch_bytes(1 << 20, 7, 1160) <= STATIC_BYTES
    for m, n, s, seed in cases:   # calls in a row, different shapes and seeds
        A = rng.standard_normal((m, n))
        Ad = api.colmajor(A, device="cuda")
        d = api.desc(api.NS_SRHT, s=s, seed=seed)
        ref = api.ns_sketch(d, Ad)
        SA = torch.full((n, s), float("nan"), dtype=torch.float64, device="cuda").t()
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda") if with_status else None
        assert call_static(api, d, Ad, m, n, SA, status) == 0
        torch.cuda.synchronize()
        assert torch.equal(SA, ref), (m, n, s)
        if with_status:
            assert int(status.item()) == 0


def test_static_scratch_reports_nonfinite_input(api):
    m, n, s = 9000, 3, 128
    A = np.random.default_rng(3).standard_normal((m, n))
    A[4321, 1] = np.nan
    Ad = api.colmajor(A, device="cuda")
    d = api.desc(api.NS_SRHT, s=s, seed=1)
    SA = torch.empty((n, s), dtype=torch.float64, device="cuda").t()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert call_static(api, d, Ad, m, n, SA, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == api._lib.NS_ERR_NONFINITE


def test_static_scratch_rejects_oversized(api):
    # scratch beyond the fixed 16 MiB array is refused before any launch,
    # including the case one step past the one that just fits above
    assert scratch_bytes(1 << 20, 7, 1170) > STATIC_BYTES
    lib = api._lib.load()
    fake = ctypes.c_void_p(0x100000)
    for m, n, s in ((1 << 22, 512, 8192), (1 << 20, 7, 1170)):
        d = api.desc(api.NS_SRHT, s=s, seed=0)
        st = lib.ns_sketch_static(ctypes.byref(d), fake, api.NS_F64, m, n, m, fake, None, None)
        assert st == api._lib.NS_ERR_WORKSPACE
