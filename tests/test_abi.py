"""The C ABI library builds, loads and exports every symbol of include/heat1d.h
(CPU only: no compute call is made without a GPU)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_1510_08982_gb300 import build as build_mod
from paper_1510_08982_gb300 import heat1d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "heat1d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(heat1d_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return heat1d.load()


def test_header_declares_the_binding_names():
    assert header_functions() == sorted(heat1d.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_opts_struct_layout_matches_header():
    # int64 segments, 4 x int32, int64 spin_limit, int32 stall + 7 reserved
    assert ctypes.sizeof(heat1d.Opts) == 8 + 4 * 4 + 8 + 4 + 7 * 4
    assert heat1d.Opts.spin_limit_ns.offset == 24


def test_default_opts(lib):
    o = heat1d.default_opts()
    assert o.segments == 0 and o.q == 0 and o.stall_segment == -1


def test_create_rejects_bad_arguments_without_a_gpu(lib):
    # argument checks come before any CUDA call
    assert not lib.heat1d_create(2, 0.25, 0.0, 1.0, heat1d.F64)
    assert "N must be" in heat1d.last_error()
    assert not lib.heat1d_create(100, 0.75, 0.0, 1.0, heat1d.F64)
    assert "r must be" in heat1d.last_error()
    assert not lib.heat1d_create(100, 0.25, 0.0, 1.0, 7)
    assert "dtype" in heat1d.last_error()


def test_build_is_in_tree_for_sm103a():
    assert build_mod.LIB.startswith(os.path.join(ROOT, "paper_1510_08982_gb300"))
    assert "arch=compute_103a,code=sm_103a" in build_mod.ARCH


def test_every_entry_point_rejects_a_null_handle_without_a_gpu(lib):
    """Each call checks its handle (and null buffers) before any CUDA call and
    reports HEAT1D_ERR_INVAL with a message; destroy accepts NULL."""
    buf = ctypes.create_string_buffer(64)
    o = heat1d.default_opts()
    calls = {
        "heat1d_set_stream": (None, None),
        "heat1d_set_snapshots": (None, None, 1, 1),
        "heat1d_set_opts": (None, ctypes.byref(o)),
        "heat1d_get_opts": (None, ctypes.byref(o)),
        "heat1d_num_segments": (None, None),
        "heat1d_set_u": (None, buf, 0),
        "heat1d_get_u": (None, buf, 0),
        "heat1d_run_sync": (None, 10),
        "heat1d_run_async": (None, 10, None, 0),
        "heat1d_trace_bytes": (None, 10),
        "heat1d_replay": (None, 10, buf, 0),
        "heat1d_sync": (None,),
        "heat1d_run_async_blocked": (None, 10, None, 0),
        "heat1d_replay_blocked": (None, 10, buf, 0),
        "heat1d_blocked_trace_bytes": (None, 10),
        "heat1d_adjoint": (None, 10, None, 0, buf, 0, buf, None, None),
        "heat1d_vjp": (None, 10, None, 0, buf, 0, buf, None),
        "heat1d_batch_run": (None, buf, None),
        "heat1d_batch_sync": (None,),
        "heat1d_batch_describe": (None, buf),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == heat1d.ERR_INVAL, name
        assert heat1d.last_error(), name
    lib.heat1d_destroy(None)
    lib.heat1d_batch_destroy(None)


def test_buffer_and_batch_arguments_are_checked_without_a_gpu(lib):
    a = ctypes.create_string_buffer(64)
    b = ctypes.create_string_buffer(64)
    f = lib.heat1d_run_sync_noalloc
    assert f(None, b, 10, 0.25, 0.0, 1.0, heat1d.F64, 5, 0, None, None) == heat1d.ERR_INVAL
    assert f(a, a, 10, 0.25, 0.0, 1.0, heat1d.F64, 5, 0, None, None) == heat1d.ERR_INVAL
    assert "differ" in heat1d.last_error()
    assert f(a, b, 2, 0.25, 0.0, 1.0, heat1d.F64, 5, 0, None, None) == heat1d.ERR_INVAL
    assert not lib.heat1d_batch_create(None, 5, heat1d.F64, None)
    rod = heat1d.RodSpec(0, 100, 10, 0.25, 0.0, 1.0)
    assert not lib.heat1d_batch_create(ctypes.byref(rod), 1, 7, None)
    assert "dtype" in heat1d.last_error()
    assert lib.heat1d_adjoint_batched(0, 100, 10, None, None, None, heat1d.F64, None, None, 0, 0, 3, None, 0,
                                      None, None, None, None, None) == heat1d.ERR_INVAL


def test_normal_build_is_not_bounds_checked(lib):
    """The normal library reports that it is not the checked build, and its
    self-test refuses before launching anything (no GPU needed)."""
    if os.environ.get("HEAT1D_CHECKED") == "1":
        pytest.skip("the checked build is loaded in this process")
    assert lib.heat1d_checked() == 0
    assert lib.heat1d_checked_selftest() == heat1d.ERR_INVAL


def test_checked_build_compiles():
    """The bounds-checked variant builds for sm_103a beside the normal one
    (its checks run on the GPU: tests/test_gpu_checked.py)."""
    path = build_mod.build(checked=True)
    assert path.endswith("libheat1d_checked.so") and os.path.exists(path)
