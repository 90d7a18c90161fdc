"""ns_sketch_static: the SRHT sketch for callers that cannot allocate device memory.

Some embedding hosts own all device memory through their own allocator, or
forbid allocation once they are running; they cannot hand libns a workspace.
ns_sketch_static keeps its scratch in a fixed array inside the library.  This
test calls it through the C ABI twice in a row (the array keeps the previous
call's contents, so the second call checks that nothing stale leaks through)
and compares each result with ns_sketch, which uses a caller workspace.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_00975_gb300 import build
    build.build()
    from paper_2206_00975_gb300 import api as a
    return a


def test_static_scratch_matches_workspace_path(api):
    rng = np.random.default_rng(17)
    cases = [((1 << 17) + 9, 6, 512, 21), (5000, 3, 128, 4)]
    for m, n, s, seed in cases:   # two calls in a row, different shapes and seeds
        A = rng.standard_normal((m, n))
        Ad = api.colmajor(A, device="cuda")
        d = api.desc(api.NS_SRHT, s=s, seed=seed)
        ref = api.ns_sketch(d, Ad)
        SA = torch.full((n, s), float("nan"), dtype=torch.float64, device="cuda").t()
        lib = api._lib.load()
        st = lib.ns_sketch_static(ctypes.byref(d), ctypes.c_void_p(Ad.data_ptr()), api.NS_F64, m, n, m,
                                  ctypes.c_void_p(SA.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        got, want = SA.cpu().numpy(), ref.cpu().numpy()
        assert np.max(np.abs(got - want)) <= 1e-12 * np.linalg.norm(A)


def test_static_scratch_rejects_oversized(api):
    # scratch beyond the fixed 16 MiB array is refused before any launch
    d = api.desc(api.NS_SRHT, s=8192, seed=0)
    lib = api._lib.load()
    fake = ctypes.c_void_p(0x100000)
    st = lib.ns_sketch_static(ctypes.byref(d), fake, api.NS_F64, 1 << 22, 512, 1 << 22, fake, None)
    assert st == api._lib.NS_ERR_WORKSPACE
