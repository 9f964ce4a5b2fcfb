"""Python binding of libheat1d (C ABI in include/heat1d.h).

Argument marshalling only: every step of a run executes in the library's CUDA
kernels.  PyTorch provides device memory and the CUDA stream (each call is
enqueued on ``torch.cuda.current_stream()``).  There is no CPU fallback: if
the library is missing, ``load()`` raises.

Names follow the C ABI: ``Heat1d.run_sync``, ``run_async``, ``replay``,
``trace_bytes``, ``sync``, ``set_u``, ``get_u``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# HEAT1D_CHECKED=1 in the environment loads the bounds-checked build
# (libheat1d_checked.so, built by build.build(checked=True)) instead.
LIB_PATH = os.path.join(_PKG, "libheat1d_checked.so" if os.environ.get("HEAT1D_CHECKED") == "1" else "libheat1d.so")

F32, F64 = 0, 1
OK, ERR_INVAL, ERR_CUDA, ERR_TIMEOUT, ERR_NOT_RESIDENT, ERR_TRACE, ERR_OOM, ERR_BOUNDS = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {OK: "HEAT1D_OK", ERR_INVAL: "HEAT1D_ERR_INVAL", ERR_CUDA: "HEAT1D_ERR_CUDA",
                ERR_TIMEOUT: "HEAT1D_ERR_TIMEOUT", ERR_NOT_RESIDENT: "HEAT1D_ERR_NOT_RESIDENT",
                ERR_TRACE: "HEAT1D_ERR_TRACE", ERR_OOM: "HEAT1D_ERR_OOM", ERR_BOUNDS: "HEAT1D_ERR_BOUNDS"}

# Every symbol the header declares (checked by the CPU test suite).
EXPORTS = ["heat1d_default_opts", "heat1d_create", "heat1d_destroy", "heat1d_last_error", "heat1d_set_stream",
           "heat1d_set_snapshots", "heat1d_set_opts", "heat1d_get_opts", "heat1d_num_segments", "heat1d_set_u", "heat1d_get_u",
           "heat1d_run_sync", "heat1d_run_async", "heat1d_trace_bytes", "heat1d_replay", "heat1d_sync",
           "heat1d_run_async_blocked", "heat1d_replay_blocked", "heat1d_blocked_trace_bytes", "heat1d_blocked_segments",
           "heat1d_async_cluster", "heat1d_checked", "heat1d_checked_selftest",
           "heat1d_batch_run_async", "heat1d_batch_replay", "heat1d_batch_trace_bytes", "heat1d_batch_rod_parts",
           "heat1d_batch_create", "heat1d_batch_run", "heat1d_batch_sync", "heat1d_batch_describe",
           "heat1d_batch_destroy", "heat1d_run_batched", "heat1d_adjoint", "heat1d_vjp",
           "heat1d_adjoint_batched", "heat1d_run_sync_noalloc", "heat1d_probe_fma", "heat1d_state_bytes",
           "heat1d_get_state", "heat1d_set_state"]


class Heat1dError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, str(code)), msg))
        self.code = code


def checked() -> bool:
    """Whether the loaded library is the bounds-checked build."""
    return bool(load().heat1d_checked())


def checked_selftest() -> int:
    """Checked build: the status of a kernel whose checked load and store
    at one past the end of a buffer were skipped (ERR_BOUNDS expected)."""
    return int(load().heat1d_checked_selftest())


class Opts(ctypes.Structure):
    _fields_ = [("segments", ctypes.c_int64), ("q", ctypes.c_int32), ("halo_steps", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("elems_per_thread", ctypes.c_int32),
                ("spin_limit_ns", ctypes.c_int64), ("stall_segment", ctypes.c_int32),
                ("sync_mode", ctypes.c_int32), ("boundary", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class RodSpec(ctypes.Structure):
    """heat1d_rod: one rod of a batch (offset into the packed state, N, K, r, c1, cN)."""
    _fields_ = [("offset", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int64), ("r", ctypes.c_double),
                ("c1", ctypes.c_double), ("cN", ctypes.c_double)]


_lib = None


def load():
    """Loads libheat1d.so (built by ``python -m paper_1510_08982_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libheat1d.so is not built (%s); run `python -m paper_1510_08982_gb300.build` "
                           "or __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "heat1d_default_opts": (None, [ctypes.POINTER(Opts)]),
        "heat1d_create": (vp, [i64, dbl, dbl, dbl, i32]),
        "heat1d_destroy": (None, [vp]),
        "heat1d_last_error": (ctypes.c_char_p, []),
        "heat1d_set_stream": (i32, [vp, vp]),
        "heat1d_set_snapshots": (i32, [vp, vp, i64, i64]),
        "heat1d_set_opts": (i32, [vp, ctypes.POINTER(Opts)]),
        "heat1d_get_opts": (i32, [vp, ctypes.POINTER(Opts)]),
        "heat1d_num_segments": (i64, [vp, vp]),
        "heat1d_set_u": (i32, [vp, vp, i32]),
        "heat1d_get_u": (i32, [vp, vp, i32]),
        "heat1d_run_sync": (i32, [vp, i64]),
        "heat1d_run_async": (i32, [vp, i64, vp, i32]),
        "heat1d_trace_bytes": (i64, [vp, i64]),
        "heat1d_replay": (i32, [vp, i64, vp, i32]),
        "heat1d_sync": (i32, [vp]),
        "heat1d_run_async_blocked": (i32, [vp, i64, vp, i32]),
        "heat1d_replay_blocked": (i32, [vp, i64, vp, i32]),
        "heat1d_blocked_trace_bytes": (i64, [vp, i64]),
        "heat1d_blocked_segments": (i64, [vp, vp, ctypes.POINTER(ctypes.c_int32)]),
        "heat1d_async_cluster": (i32, [vp, i32]),
        "heat1d_checked": (i32, []),
        "heat1d_batch_run_async": (i32, [vp, vp, vp, vp]),
        "heat1d_batch_replay": (i32, [vp, vp, vp, vp]),
        "heat1d_batch_trace_bytes": (i64, [vp]),
        "heat1d_batch_rod_parts": (i64, [vp, i64, vp, ctypes.POINTER(ctypes.c_int64)]),
        "heat1d_checked_selftest": (i32, []),
        "heat1d_state_bytes": (i64, [vp]),
        "heat1d_get_state": (i32, [vp, vp, i32]),
        "heat1d_set_state": (i32, [vp, vp, i32]),
        "heat1d_run_sync_noalloc": (i32, [vp, vp, i64, dbl, dbl, dbl, i32, i64, i64, vp, vp]),
        "heat1d_probe_fma": (i32, [i32, i32, i64, i64, i32, vp, vp, ctypes.POINTER(i64)]),
        "heat1d_batch_create": (vp, [ctypes.POINTER(RodSpec), i64, i32, ctypes.POINTER(Opts)]),
        "heat1d_batch_run": (i32, [vp, vp, vp]),
        "heat1d_batch_sync": (i32, [vp]),
        "heat1d_batch_describe": (i32, [vp, vp]),
        "heat1d_batch_destroy": (None, [vp]),
        "heat1d_run_batched": (i32, [ctypes.POINTER(RodSpec), i64, vp, i32, ctypes.POINTER(Opts), vp]),
        "heat1d_adjoint": (i32, [vp, i64, vp, i32, vp, i64, vp, vp, vp]),
        "heat1d_vjp": (i32, [vp, i64, vp, i32, vp, i64, vp, vp]),
        "heat1d_adjoint_batched": (i32, [i64, i64, i64, vp, vp, vp, i32, vp, vp, i32, i64, i32, vp, i64, vp, vp, vp,
                                          vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().heat1d_last_error().decode()


def _check(rc):
    if rc != OK:
        raise Heat1dError(rc, last_error())
    return rc


def _torch():
    import torch
    return torch


def _dtype_code(dtype):
    torch = _torch()
    if dtype in (torch.float64, np.float64, "f64", "float64"):
        return F64
    if dtype in (torch.float32, np.float32, "f32", "float32"):
        return F32
    raise ValueError("dtype must be float32 or float64")


def default_opts() -> Opts:
    o = Opts()
    load().heat1d_default_opts(ctypes.byref(o))
    return o


class Heat1d:
    """One rod of N points: state, options and scratch on the current device.

    ``opts`` keywords: segments, q, halo_steps, block_threads,
    elems_per_thread, spin_limit_ns, stall_segment, sync_mode, boundary,
    cluster (see heat1d_opts; boundary=1 is the periodic ring of Section 5.3,
    cluster the CTAs per thread-block cluster of per-step asynchronous runs)."""

    def __init__(self, N, r, c1, cN, dtype="float64", **opts):
        torch = _torch()
        self.lib = load()
        self.N = int(N)
        self.code = _dtype_code(dtype)
        self.torch_dtype = torch.float64 if self.code == F64 else torch.float32
        self.np_dtype = np.float64 if self.code == F64 else np.float32
        torch.cuda.init()
        h = self.lib.heat1d_create(self.N, float(r), float(c1), float(cN), self.code)
        if not h:
            raise Heat1dError(ERR_INVAL, last_error())
        self.h = ctypes.c_void_p(h)
        if opts:
            self.set_opts(**opts)

    def close(self):
        if getattr(self, "h", None):
            self.lib.heat1d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- config
    def _stream(self):
        torch = _torch()
        _check(self.lib.heat1d_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

    def set_opts(self, **kw):
        o = default_opts()
        for k, v in kw.items():
            if not hasattr(o, k):
                raise TypeError("unknown option %r" % k)
            setattr(o, k, int(v))
        _check(self.lib.heat1d_set_opts(self.h, ctypes.byref(o)))

    def set_snapshots(self, buf=None, every=1):
        """Record the state every `every` steps of the following runs into
        buf (CUDA tensor of shape (rows, N), the handle's dtype); None stops."""
        if buf is None:
            _check(self.lib.heat1d_set_snapshots(self.h, None, 0, 0))
            self._snap = None
            return
        if not buf.is_cuda or buf.dtype != self.torch_dtype or buf.dim() != 2 or buf.shape[1] != self.N:
            raise ValueError("snapshot buffer must be a CUDA tensor (rows, N) of the handle's dtype")
        _check(self.lib.heat1d_set_snapshots(self.h, ctypes.c_void_p(buf.data_ptr()), int(every), buf.shape[0]))
        self._snap = buf

    def get_opts(self) -> dict:
        o = Opts()
        _check(self.lib.heat1d_get_opts(self.h, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in Opts._fields_ if k != "reserved"}

    @property
    def segments(self) -> np.ndarray:
        S = self.lib.heat1d_num_segments(self.h, None)
        off = np.zeros(S + 1, dtype=np.int64)
        self.lib.heat1d_num_segments(self.h, off.ctypes.data_as(ctypes.c_void_p))
        return off

    @property
    def S(self) -> int:
        return int(self.lib.heat1d_num_segments(self.h, None))

    # ---------------------------------------------------------------- state
    def set_u(self, u):
        """u: a CUDA tensor (device copy) or a host array/tensor of N values."""
        torch = _torch()
        self._stream()
        if isinstance(u, torch.Tensor) and u.is_cuda:
            t = u.to(self.torch_dtype).contiguous()
            if t.numel() != self.N:
                raise ValueError("u has %d values, expected %d" % (t.numel(), self.N))
            _check(self.lib.heat1d_set_u(self.h, ctypes.c_void_p(t.data_ptr()), 1))
            self._keep = t  # alive until the copy is done
        else:
            a = np.ascontiguousarray(u.cpu().numpy() if isinstance(u, torch.Tensor) else u, dtype=self.np_dtype)
            if a.size != self.N:
                raise ValueError("u has %d values, expected %d" % (a.size, self.N))
            _check(self.lib.heat1d_set_u(self.h, a.ctypes.data_as(ctypes.c_void_p), 0))

    def get_u(self, out=None, device=True):
        """The current state as a CUDA tensor (device=True) or numpy array."""
        torch = _torch()
        self._stream()
        if device:
            if out is None:
                out = torch.empty(self.N, dtype=self.torch_dtype, device="cuda")
            _check(self.lib.heat1d_get_u(self.h, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        a = np.empty(self.N, dtype=self.np_dtype) if out is None else out
        _check(self.lib.heat1d_get_u(self.h, a.ctypes.data_as(ctypes.c_void_p), 0))
        return a

    # ---------------------------------------------------------------- runs
    def trace_bytes(self, K) -> int:
        return int(self.lib.heat1d_trace_bytes(self.h, int(K)))

    def new_trace(self, K, device=True):
        torch = _torch()
        periodic = self.get_opts().get("boundary", 0) == 1
        shape = (int(K), self.S if periodic else max(self.S - 1, 0), 2)
        if device:
            return torch.empty(shape, dtype=torch.uint8, device="cuda")
        return np.empty(shape, dtype=np.uint8)

    def run_sync(self, K):
        self._stream()
        _check(self.lib.heat1d_run_sync(self.h, int(K)))

    def run_async(self, K, trace_out=None):
        """trace_out: None, a CUDA uint8 tensor or a host uint8 array of
        trace_bytes(K) bytes (host arrays are complete after sync())."""
        self._stream()
        ptr, on_dev = self._trace_ptr(trace_out, K)
        _check(self.lib.heat1d_run_async(self.h, int(K), ptr, on_dev))

    def replay(self, K, trace):
        self._stream()
        ptr, on_dev = self._trace_ptr(trace, K)
        _check(self.lib.heat1d_replay(self.h, int(K), ptr, on_dev))

    def blocked_trace_bytes(self, K) -> int:
        return int(self.lib.heat1d_blocked_trace_bytes(self.h, int(K)))

    def blocked_segments(self):
        """(offsets, T): the segments of the blocked asynchronous run (the
        handle's segments on chip, the HBM tiles when streamed) and its block
        length."""
        n = int(self.lib.heat1d_blocked_segments(self.h, None, None))
        if n < 0:
            raise Heat1dError(n, last_error())
        off = np.zeros(n + 1, dtype=np.int64)
        T = ctypes.c_int32(0)
        self.lib.heat1d_blocked_segments(self.h, off.ctypes.data_as(ctypes.c_void_p), ctypes.byref(T))
        return off, int(T.value)

    def async_cluster(self, blocked=False) -> int:
        """CTAs per thread-block cluster of the per-step (or, blocked=True,
        the blocked) asynchronous run (1: every exchange through global
        memory)."""
        c = int(self.lib.heat1d_async_cluster(self.h, 1 if blocked else 0))
        if c < 0:
            raise Heat1dError(c, last_error())
        return c

    def new_blocked_trace(self, K, device=True):
        """A trace buffer for a blocked run of K steps: (ceil(K/T), S-1, 2)
        uint8 (S segments of blocked_segments(); S on the periodic ring)."""
        torch = _torch()
        o = self.get_opts()
        off, T = self.blocked_segments()
        S = off.size - 1
        shape = ((int(K) + T - 1) // T, S if o.get("boundary", 0) == 1 else max(S - 1, 0), 2)
        if device:
            return torch.empty(shape, dtype=torch.uint8, device="cuda")
        return np.empty(shape, dtype=np.uint8)

    def run_async_blocked(self, K, trace_out=None):
        """Asynchronous run with temporal blocking (blocks of halo_steps steps);
        trace_out as for run_async, blocked_trace_bytes(K) bytes."""
        self._stream()
        ptr, on_dev = self._trace_ptr(trace_out, K, self.blocked_trace_bytes(K))
        _check(self.lib.heat1d_run_async_blocked(self.h, int(K), ptr, on_dev))

    def replay_blocked(self, K, trace):
        self._stream()
        ptr, on_dev = self._trace_ptr(trace, K, self.blocked_trace_bytes(K))
        _check(self.lib.heat1d_replay_blocked(self.h, int(K), ptr, on_dev))

    def state_bytes(self) -> int:
        return int(self.lib.heat1d_state_bytes(self.h))

    def get_state(self, device=False):
        """heat1d_get_state: the state (u and the edge history of the last q
        steps of an asynchronous run) as a uint8 numpy array, or a CUDA
        tensor with device=True."""
        torch = _torch()
        self._stream()
        n = self.state_bytes()
        if device:
            buf = torch.empty(n, dtype=torch.uint8, device="cuda")
            _check(self.lib.heat1d_get_state(self.h, ctypes.c_void_p(buf.data_ptr()), 1))
            return buf
        buf = np.empty(n, dtype=np.uint8)
        _check(self.lib.heat1d_get_state(self.h, buf.ctypes.data_as(ctypes.c_void_p), 0))
        return buf

    def set_state(self, state):
        """heat1d_set_state from a state of get_state (numpy or CUDA tensor)."""
        torch = _torch()
        self._stream()
        if isinstance(state, torch.Tensor) and state.is_cuda:
            _check(self.lib.heat1d_set_state(self.h, ctypes.c_void_p(state.contiguous().data_ptr()), 1))
        else:
            st = np.ascontiguousarray(state if not isinstance(state, torch.Tensor) else state.numpy(), dtype=np.uint8)
            _check(self.lib.heat1d_set_state(self.h, st.ctypes.data_as(ctypes.c_void_p), 0))

    def sync(self):
        """Waits for the stream; raises on a device-side failure."""
        _check(self.lib.heat1d_sync(self.h))

    def adjoint(self, K, u_obs, trace=None, ckpt_every=0):
        """heat1d_adjoint from the current state: returns (loss, grad_u0 as a
        CUDA float64 tensor, grad_r).  Afterwards the state is u(K)."""
        torch = _torch()
        self._stream()
        uo = u_obs.to(device="cuda", dtype=torch.float64).contiguous()
        g = torch.empty(self.N, dtype=torch.float64, device="cuda")
        gr = ctypes.c_double(0.0)
        ls = ctypes.c_double(0.0)
        tp, on_dev = self._trace_ptr(trace, K) if trace is not None else (None, 0)
        _check(self.lib.heat1d_adjoint(self.h, int(K), tp, on_dev, ctypes.c_void_p(uo.data_ptr()), int(ckpt_every),
                                       ctypes.c_void_p(g.data_ptr()), ctypes.byref(gr), ctypes.byref(ls)))
        return ls.value, g, gr.value

    def vjp(self, K, grad_uK, trace=None, ckpt_every=0):
        """heat1d_vjp from the current state: (grad_u0 float64 tensor, grad_r)."""
        torch = _torch()
        self._stream()
        gk = grad_uK.to(device="cuda", dtype=torch.float64).contiguous()
        g = torch.empty(self.N, dtype=torch.float64, device="cuda")
        gr = ctypes.c_double(0.0)
        tp, on_dev = self._trace_ptr(trace, K) if trace is not None else (None, 0)
        _check(self.lib.heat1d_vjp(self.h, int(K), tp, on_dev, ctypes.c_void_p(gk.data_ptr()), int(ckpt_every),
                                   ctypes.c_void_p(g.data_ptr()), ctypes.byref(gr)))
        return g, gr.value

    def _trace_ptr(self, t, K, n=None):
        torch = _torch()
        if t is None:
            return None, 0
        if n is None:
            n = self.trace_bytes(K)
        if isinstance(t, torch.Tensor):
            if t.dtype != torch.uint8 or not t.is_contiguous() or t.numel() != n:
                raise ValueError("trace must be a contiguous uint8 tensor of %d bytes" % n)
            if t.is_cuda:
                return ctypes.c_void_p(t.data_ptr()), 1
            t = t.numpy()
        if not isinstance(t, np.ndarray) or t.dtype != np.uint8 or not t.flags.c_contiguous or t.size != n:
            raise ValueError("trace must be a contiguous uint8 array of %d bytes" % n)
        return t.ctypes.data_as(ctypes.c_void_p), 0


def run_sync_noalloc(u_in, u_out, r, c1, cN, K, segments=0, status_out=None):
    """heat1d_run_sync_noalloc on CUDA tensors u_in -> u_out (same dtype, N
    values each) on the current stream; allocates nothing.  status_out: an
    optional CUDA int32 tensor that receives the device status."""
    torch = _torch()
    lib = load()
    if not (u_in.is_cuda and u_out.is_cuda) or u_in.dtype != u_out.dtype or u_in.numel() != u_out.numel():
        raise ValueError("u_in and u_out must be CUDA tensors of the same dtype and size")
    if not (u_in.is_contiguous() and u_out.is_contiguous()):
        raise ValueError("u_in and u_out must be contiguous")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sp = None if status_out is None else ctypes.c_void_p(status_out.data_ptr())
    _check(lib.heat1d_run_sync_noalloc(ctypes.c_void_p(u_in.data_ptr()), ctypes.c_void_p(u_out.data_ptr()),
                                       u_in.numel(), float(r), float(c1), float(cN), _dtype_code(u_in.dtype),
                                       int(K), int(segments), st, sp))


def probe_fma(dtype="float64", iters=None, shapes=None, repeats=3):
    """heat1d_probe_fma: the fused multiply-add rate of the device (FMA per
    second).  Each launch shape (chains per thread, CTAs per SM, threads per
    CTA) is launched once untimed and `repeats` times timed with CUDA events
    on the current stream; returns (best rate, {shape: best rate})."""
    torch = _torch()
    lib = load()
    dev = torch.cuda.current_device()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    f64 = dtype in ("float64", torch.float64)
    tdt = torch.float64 if f64 else torch.float32
    if shapes is None:  # (chains, CTAs per SM, threads); chains < 0: the stencil's pattern on -chains points
        shapes = [(8, 4, 256), (16, 2, 512), (4, 8, 256), (16, 1, 1024), (-8, 4, 256), (-16, 2, 256)]
    if iters is None:
        iters = 40_000 if f64 else 400_000
    st = torch.cuda.current_stream()
    n = ctypes.c_int64(0)
    rates = {}
    for chains, per_sm, threads in shapes:
        blocks = nsm * per_sm
        out = torch.empty(blocks * threads, dtype=tdt, device="cuda")
        best = 0.0
        for i in range(repeats + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            per_iter = chains if chains > 0 else -chains * 6
            _check(lib.heat1d_probe_fma(_dtype_code(tdt), chains, int(max(1, iters * 8 // per_iter)), blocks, threads,
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream),
                                        ctypes.byref(n)))
            e1.record(st)
            e1.synchronize()
            if i > 0:  # the first launch is a warm-up
                best = max(best, n.value / (e0.elapsed_time(e1) * 1e-3))
        key = ("chains=%d" % chains) if chains > 0 else ("stencil points=%d" % -chains)
        rates["%s ctas_per_sm=%d threads=%d" % (key, per_sm, threads)] = best
    return max(rates.values()), rates


# ---------------------------------------------------------------------------- batched rods


def pack_offsets(Ns):
    """Offsets of rods of lengths Ns laid out back to back (int64 array) and
    the total length."""
    Ns = np.asarray(Ns, dtype=np.int64)
    off = np.zeros(Ns.size, dtype=np.int64)
    if Ns.size:
        off[1:] = np.cumsum(Ns)[:-1]
    return off, int(Ns.sum())


def _rod_array(specs):
    arr = (RodSpec * len(specs))()
    for i, sp in enumerate(specs):
        off, N, K, r, c1, cN = sp
        arr[i] = RodSpec(int(off), int(N), int(K), float(r), float(c1), float(cN))
    return arr


def _opts(kw):
    o = default_opts()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError("unknown option %r" % k)
        setattr(o, k, int(v))
    return o


class Batch:
    """A planned batch of rods (heat1d_batch_*).  specs: sequence of
    (offset, N, K, r, c1, cN).  run(u) advances every rod in the packed CUDA
    tensor u in place on the current stream (capturable in a CUDA graph)."""

    def __init__(self, specs, dtype="float64", **opts):
        self.lib = load()
        self.code = _dtype_code(dtype)
        arr = _rod_array(specs)
        o = _opts(opts)
        b = self.lib.heat1d_batch_create(arr, len(specs), self.code, ctypes.byref(o))
        if not b:
            raise Heat1dError(ERR_INVAL, last_error())
        self.b = ctypes.c_void_p(b)

    def run(self, u):
        torch = _torch()
        if not u.is_cuda or not u.is_contiguous():
            raise ValueError("u must be a contiguous CUDA tensor")
        if _dtype_code(u.dtype) != self.code:
            raise ValueError("u has the wrong dtype for this batch")
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        _check(self.lib.heat1d_batch_run(self.b, ctypes.c_void_p(u.data_ptr()), st))

    def run_async(self, u, trace=None):
        """Asynchronous run: the parts of split rods exchange strips with
        bounded block delays (heat1d_batch_run_async); trace: a CUDA uint8
        tensor of trace_bytes() entries (or None)."""
        torch = _torch()
        self._check_u(u)
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        tp = None if trace is None else ctypes.c_void_p(self._trace_ptr(trace))
        _check(self.lib.heat1d_batch_run_async(self.b, ctypes.c_void_p(u.data_ptr()), st, tp))

    def replay(self, u, trace):
        """Replay of an asynchronous run with the delays of `trace` (CUDA
        uint8 tensor of trace_bytes() entries)."""
        torch = _torch()
        self._check_u(u)
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        _check(self.lib.heat1d_batch_replay(self.b, ctypes.c_void_p(u.data_ptr()), st,
                                            ctypes.c_void_p(self._trace_ptr(trace))))

    def trace_bytes(self) -> int:
        return int(self.lib.heat1d_batch_trace_bytes(self.b))

    def new_trace(self):
        torch = _torch()
        return torch.zeros(max(self.trace_bytes(), 1), dtype=torch.uint8, device="cuda")

    def rod_parts(self, rod):
        """(offsets, trace_offset) of a rod's parts: offsets has P+1 entries
        (rod-relative part starts, then N); trace_offset is -1 for a rod that
        is not split."""
        n = int(self.lib.heat1d_batch_rod_parts(self.b, int(rod), None, None))
        if n < 0:
            raise Heat1dError(n, last_error())
        off = np.zeros(n + 1, dtype=np.int64)
        toff = ctypes.c_int64(0)
        self.lib.heat1d_batch_rod_parts(self.b, int(rod), off.ctypes.data_as(ctypes.c_void_p), ctypes.byref(toff))
        return off, int(toff.value)

    def _check_u(self, u):
        if not u.is_cuda or not u.is_contiguous():
            raise ValueError("u must be a contiguous CUDA tensor")
        if _dtype_code(u.dtype) != self.code:
            raise ValueError("u has the wrong dtype for this batch")

    def _trace_ptr(self, trace):
        torch = _torch()
        if not (isinstance(trace, torch.Tensor) and trace.is_cuda and trace.dtype == torch.uint8 and trace.is_contiguous()
                and trace.numel() >= self.trace_bytes()):
            raise ValueError("trace must be a contiguous CUDA uint8 tensor of trace_bytes() entries")
        return trace.data_ptr()

    def sync(self):
        _check(self.lib.heat1d_batch_sync(self.b))

    def describe(self) -> dict:
        info = np.zeros(8, dtype=np.int64)
        _check(self.lib.heat1d_batch_describe(self.b, info.ctypes.data_as(ctypes.c_void_p)))
        keys = ["warp_batches", "cta_rods", "rod_parts", "ctas", "threads", "elems_per_thread", "halo_steps",
                "points_per_cta"]
        return dict(zip(keys, (int(x) for x in info)))

    def close(self):
        if getattr(self, "b", None):
            self.lib.heat1d_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_batched(specs, u, dtype="float64", **opts):
    """heat1d_run_batched: plan, run on the current stream, wait, free."""
    torch = _torch()
    arr = _rod_array(specs)
    o = _opts(opts)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(load().heat1d_run_batched(arr, len(specs), ctypes.c_void_p(u.data_ptr()), _dtype_code(dtype),
                                     ctypes.byref(o), st))


def adjoint_batched(u0, u_obs, r, c1, cN, K, trace=None, segments=0, q=3, ckpt_every=0, cotangent=False):
    """heat1d_adjoint_batched for u0 of shape (nrods, N) (CUDA, float32 or
    float64).  Returns (uK, grad_u0 (float64), grad_r (numpy), loss (numpy))."""
    torch = _torch()
    nrods, N = u0.shape
    u0 = u0.contiguous()
    uo = u_obs.to(device="cuda", dtype=torch.float64).contiguous()
    uK = torch.empty_like(u0)
    g = torch.empty((nrods, N), dtype=torch.float64, device="cuda")
    rr = np.ascontiguousarray(r, dtype=np.float64)
    cc1 = np.ascontiguousarray(c1, dtype=np.float64)
    ccN = np.ascontiguousarray(cN, dtype=np.float64)
    gr = np.zeros(nrods)
    ls = np.zeros(nrods)
    tp = None
    if trace is not None:
        if not (isinstance(trace, torch.Tensor) and trace.is_cuda and trace.dtype == torch.uint8):
            raise ValueError("trace must be a CUDA uint8 tensor of shape (nrods, K, segments-1, 2)")
        tp = ctypes.c_void_p(trace.contiguous().data_ptr())
    vp = ctypes.c_void_p
    st = vp(torch.cuda.current_stream().cuda_stream)
    _check(load().heat1d_adjoint_batched(nrods, N, int(K), rr.ctypes.data_as(vp), cc1.ctypes.data_as(vp),
                                         ccN.ctypes.data_as(vp), _dtype_code(u0.dtype), vp(u0.data_ptr()),
                                         vp(uo.data_ptr()), int(bool(cotangent)), int(segments), int(q), tp,
                                         int(ckpt_every), vp(uK.data_ptr()), vp(g.data_ptr()),
                                         gr.ctypes.data_as(vp), ls.ctypes.data_as(vp), st))
    return uK, g, gr, ls
