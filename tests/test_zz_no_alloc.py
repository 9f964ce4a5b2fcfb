"""heat1d_run_sync_noalloc: the synchronous run for callers that cannot
allocate device memory (for example code inside a host callback or an
allocator hook, a plug-in that may not grow the process's device memory, or a
loop that forbids allocation after start-up).

The entry point keeps its scratch in a fixed array inside the library, so
calls share it.  The tests call it through the C ABI:
- twice in a row on two different rods, and once more on the first, each
  output against the CPU oracle (FP64: the oracle's double sweep; FP32: its
  float mode), bit for bit and within the 1e-12 bound of the FP64 tests, and
  against the handle API's heat1d_run_sync on the same input;
- with segments = 0 (one CTA per SM), with K = 0 and with status_out = NULL;
- with the device's free memory (cudaMemGetInfo) and torch's allocated bytes
  read before and after repeated calls: neither may change.

The file name sorts last so that a run that stops at the first failure has
already run every other test.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from paper_1510_08982_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


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


def oracle_result(rod, K, dtype):
    return oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, K, dtype=np.float64 if dtype == "float64" else np.float32)


class Call:
    """Device buffers of one rod, allocated once, and the raw C-ABI call."""

    def __init__(self, H, rod, dtype):
        import torch
        self.H, self.rod, self.dtype = H, rod, dtype
        tdt = torch.float64 if dtype == "float64" else torch.float32
        self.u_in = torch.tensor(rod.u0, dtype=tdt, device="cuda")
        self.u_out = torch.full_like(self.u_in, float("nan"))
        self.status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")

    def __call__(self, K, S, with_status=True):
        import torch
        H = self.H
        self.u_out.fill_(float("nan"))
        self.status.fill_(12345)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = H.load().heat1d_run_sync_noalloc(
            ctypes.c_void_p(self.u_in.data_ptr()), ctypes.c_void_p(self.u_out.data_ptr()), self.rod.N, self.rod.r,
            self.rod.c1, self.rod.cN, H.F64 if self.dtype == "float64" else H.F32, K, S, stream,
            ctypes.c_void_p(self.status.data_ptr()) if with_status else None)
        assert rc == H.OK, H.last_error()
        torch.cuda.synchronize()
        if with_status:
            assert int(self.status.item()) == H.OK
        return self.u_out.cpu().numpy()


def check(got, ref):
    assert got.dtype == ref.dtype
    err = float(np.abs(got.astype(np.float64) - ref.astype(np.float64)).max())
    assert err <= TOL64, err
    assert np.array_equal(got, ref), "not bit-identical (max err %g)" % err


def test_noalloc_matches_oracle_on_consecutive_calls(lib):
    rod_a = inputs.small_rod(K=3000)                                   # N=1024, FP64, 8 segments
    rod_b = inputs.sine_mode_rod(N=50_000, K=1200, seed=4, m_max=64)   # FP32, 37 segments, ragged split
    ca, cb = Call(lib, rod_a, "float64"), Call(lib, rod_b, "float32")
    ref_a, ref_b = oracle_result(rod_a, rod_a.K, "float64"), oracle_result(rod_b, rod_b.K, "float32")
    check(ca(rod_a.K, 8), ref_a)
    check(cb(rod_b.K, 37), ref_b)
    # the shared scratch keeps the second call's contents; a repeat of the
    # first call must not see them
    check(ca(rod_a.K, 8), ref_a)
    # the handle API runs the same kernel with the same defaults
    check(handle_result(lib, rod_a, rod_a.K, 8, "float64"), ref_a)
    check(handle_result(lib, rod_b, rod_b.K, 37, "float32"), ref_b)


def test_noalloc_one_segment_per_sm_zero_steps_and_no_status(lib):
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    rod = inputs.sine_mode_rod(N=300_000, K=700, seed=8, m_max=64)    # segments = 0: one per SM (<= 256)
    c = Call(lib, rod, "float64")
    check(c(rod.K, 0), oracle_result(rod, rod.K, "float64"))
    check(c(rod.K, 0, with_status=False), oracle_result(rod, rod.K, "float64"))
    # K = 0: u(0) with the ends forced
    check(c(0, 0), oracle_result(rod, 0, "float64"))
    check(c(0, 100, with_status=False), oracle_result(rod, 0, "float64"))
    assert min(nsm, 256) <= rod.N


def test_noalloc_allocates_nothing(lib):
    """After one call of each shape, repeated calls change neither the
    device's free memory (cudaMemGetInfo) nor torch's allocated bytes."""
    import torch
    rod_a = inputs.small_rod(K=2000)
    rod_b = inputs.sine_mode_rod(N=80_000, K=900, seed=6, m_max=64)
    ca, cb = Call(lib, rod_a, "float64"), Call(lib, rod_b, "float32")
    ref_a, ref_b = oracle_result(rod_a, rod_a.K, "float64"), oracle_result(rod_b, rod_b.K, "float32")
    ca(rod_a.K, 8)
    cb(rod_b.K, 0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        check(ca(rod_a.K, 8), ref_a)
        check(cb(rod_b.K, 0), ref_b)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0


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
