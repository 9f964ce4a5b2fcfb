"""heat1d_run_sync_noalloc: the synchronous run for callers that cannot
allocate device memory (for example code inside a host callback or an
allocator hook, or a loop that forbids allocation after start-up).

The entry point keeps its scratch in a fixed array inside the library, so
calls share it.  The test calls it through the C ABI twice in a row, on two
different rods, and checks each output against the handle API's
heat1d_run_sync on the same input (same kernel: identical bit for bit, so
within the 1e-12 bound the other FP64 tests use), then repeats the first call
to show that nothing is left over from the second.

The file name sorts last so that a run that stops at the first failure has
already run every other test.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_1510_08982_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401
    from paper_1510_08982_gb300 import build, heat1d
    build.build()
    return heat1d


def handle_result(H, rod, K, S, dtype):
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype=dtype, segments=S) as h:
        h.set_u(rod.u0)
        h.run_sync(K)
        h.sync()
        return h.get_u(device=False)


def noalloc_call(H, rod, K, S, dtype):
    import torch
    tdt = torch.float64 if dtype == "float64" else torch.float32
    u_in = torch.tensor(rod.u0, dtype=tdt, device="cuda")
    u_out = torch.full_like(u_in, float("nan"))
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    lib = H.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.heat1d_run_sync_noalloc(ctypes.c_void_p(u_in.data_ptr()), ctypes.c_void_p(u_out.data_ptr()), rod.N,
                                     rod.r, rod.c1, rod.cN, H.F64 if dtype == "float64" else H.F32, K, S, stream,
                                     ctypes.c_void_p(status.data_ptr()))
    assert rc == H.OK, H.last_error()
    torch.cuda.synchronize()
    assert int(status.item()) == H.OK
    return u_out.cpu().numpy()


def check(got, ref):
    assert got.dtype == ref.dtype
    assert np.abs(got.astype(np.float64) - ref.astype(np.float64)).max() <= 1e-12
    assert np.array_equal(got, ref)


def test_noalloc_matches_handle_api_on_consecutive_calls(lib):
    rod_a = inputs.small_rod(K=3000)                     # N=1024, FP64, 8 segments
    rod_b = inputs.sine_mode_rod(N=50_000, K=1200, seed=4, m_max=64)  # FP32, 37 segments, ragged split
    ref_a = handle_result(lib, rod_a, rod_a.K, 8, "float64")
    ref_b = handle_result(lib, rod_b, rod_b.K, 37, "float32")
    check(noalloc_call(lib, rod_a, rod_a.K, 8, "float64"), ref_a)
    check(noalloc_call(lib, rod_b, rod_b.K, 37, "float32"), ref_b)
    # the shared scratch keeps the second call's contents; a repeat of the
    # first call must not see them
    check(noalloc_call(lib, rod_a, rod_a.K, 8, "float64"), ref_a)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    import torch
    H = lib
    u = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")
    v = torch.zeros_like(u)
    L = H.load()
    rc = L.heat1d_run_sync_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()), u.numel(), 0.25,
                                   0.0, 0.0, H.F64, 10, 257, None, None)
    assert rc == H.ERR_INVAL and "256" in H.last_error()
    rc = L.heat1d_run_sync_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()), u.numel(), 0.25,
                                   0.0, 0.0, H.F64, 10, 8, None, None)
    assert rc == H.ERR_INVAL
    big = torch.zeros(1 << 22, dtype=torch.float64, device="cuda")
    big2 = torch.zeros_like(big)
    rc = L.heat1d_run_sync_noalloc(ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big2.data_ptr()), big.numel(),
                                   0.25, 0.0, 0.0, H.F64, 10, 16, None, None)
    assert rc == H.ERR_INVAL and "exceed one CTA" in H.last_error()
