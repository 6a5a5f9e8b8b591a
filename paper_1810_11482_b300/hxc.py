"""ctypes binding of libhxc.so (include/hxc.h), same names as the C ABI.

Argument marshalling only: every step of the stencil path runs in the
library's CUDA kernels.  Loading fails loudly when libhxc.so is missing; there
is no fallback implementation.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhxc.so")

# Streams are multiplexed onto hardware queues; allow more concurrent queues
# than the default (effective only before the CUDA context is created).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

HXC_OK = 0
HXC_E_INVALID = 1
HXC_E_NOMEM = 2
HXC_E_CUDA = 3
HXC_E_TIMEOUT = 4
HXC_E_DEP_FAILED = 5
HXC_E_CALLBACK = 6
HXC_E_UNSUPPORTED = 7
HXC_E_NODEV = 8

HXC_MAX_SLOTS = 256

HXC_K_SUM_U32 = 1
HXC_K_PRK_STENCIL = 2
HXC_K_HEAT1D = 3
HXC_K_HEAT2D = 4
HXC_K_TILE_NORM2 = 5
HXC_K_HEAT3D = 6
HXC_K_VARCOEF2D = 7
HXC_K_ADJOINT2D = 8
HXC_K_PARTITION = 9
HXC_K_MANDELBROT = 10

HXC_PIPE_F64_FMA = 0
HXC_PIPE_F64_ADD = 1
HXC_PIPE_F32_FMA = 2

HXC_MODE_PLAIN = 0
HXC_MODE_GRAPH = 1
HXC_MODE_FUSED = 2
MODES = {"plain": HXC_MODE_PLAIN, "graph": HXC_MODE_GRAPH, "fused": HXC_MODE_FUSED}

c_dev = ctypes.c_void_p
c_buf = ctypes.c_void_p
c_fut = ctypes.c_void_p
c_graph = ctypes.c_void_p
c_st = ctypes.c_int
i64 = ctypes.c_int64
HOST_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p)
# argument structs beyond the core set, checked against the header by the tests
EXTRA_STRUCTS = ["hxc_heat3d_args", "hxc_varcoef2d_args", "hxc_adjoint2d_args", "hxc_kernel_arg",
                 "hxc_mandelbrot_args"]


class hxc_launch_cfg(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_uint32 * 3), ("block", ctypes.c_uint32 * 3)]


class hxc_sum_args(ctypes.Structure):
    _fields_ = [("input", c_buf), ("result", c_buf), ("n", i64)]


class hxc_prk_args(ctypes.Structure):
    _fields_ = [("in_", c_buf), ("out", c_buf), ("n", i64)]


class hxc_heat1d_args(ctypes.Structure):
    _fields_ = [("src", c_buf), ("dst", c_buf), ("n", i64), ("lo", i64), ("count", i64),
                ("r", ctypes.c_double), ("steps", ctypes.c_int32)]


class hxc_heat2d_args(ctypes.Structure):
    _fields_ = [("src", c_buf), ("dst", c_buf), ("ny", i64), ("nx", i64), ("y0", i64),
                ("x0", i64), ("ty", i64), ("tx", i64), ("r", ctypes.c_double)]


class hxc_tile_norm2_args(ctypes.Structure):
    _fields_ = [("src", c_buf), ("snap", c_buf), ("sums", c_buf), ("ny", i64), ("nx", i64),
                ("y0", i64), ("x0", i64), ("ty", i64), ("tx", i64), ("sum_index", i64)]


class hxc_heat3d_args(ctypes.Structure):
    _fields_ = [("src", c_buf), ("dst", c_buf), ("nz", i64), ("ny", i64), ("nx", i64),
                ("r", ctypes.c_float), ("steps", ctypes.c_int32)]


class hxc_varcoef2d_args(ctypes.Structure):
    _fields_ = [("src", c_buf), ("dst", c_buf), ("kappa", c_buf), ("ny", i64), ("nx", i64),
                ("c", ctypes.c_double)]


class hxc_adjoint2d_args(ctypes.Structure):
    _fields_ = [("lam_in", c_buf), ("lam_out", c_buf), ("u", c_buf), ("kappa", c_buf),
                ("grad_kappa", c_buf), ("ny", i64), ("nx", i64), ("c", ctypes.c_double)]


class hxc_partition_args(ctypes.Structure):
    _fields_ = [("x", c_buf), ("n", i64), ("offset", i64)]


class hxc_mandelbrot_args(ctypes.Structure):
    _fields_ = [("rgb", c_buf), ("counts", c_buf), ("width", i64), ("height", i64),
                ("x0", ctypes.c_float), ("y0", ctypes.c_float), ("dx", ctypes.c_float),
                ("dy", ctypes.c_float), ("max_iter", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class hxc_kernel_arg(ctypes.Structure):
    _fields_ = [("buf", c_buf), ("value", ctypes.c_void_p), ("size", ctypes.c_size_t)]


class hxc_run_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", i64), ("graph_launches", i64), ("copies", i64),
                ("host_tasks", i64), ("h2d_bytes", i64), ("d2h_bytes", i64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class hxc_heat2d_cfg(ctypes.Structure):
    _fields_ = [("ny", i64), ("nx", i64), ("tiles_y", i64), ("tiles_x", i64),
                ("r", ctypes.c_double), ("steps", ctypes.c_int32),
                ("snapshot_every", ctypes.c_int32), ("mode", ctypes.c_int),
                ("host_norms", ctypes.POINTER(ctypes.c_double)),
                ("gpu_norms", ctypes.POINTER(ctypes.c_double))]


_SIGS = {
    "hxc_status_string": (ctypes.c_char_p, [c_st]),
    "hxc_last_error": (ctypes.c_char_p, []),
    "hxc_abi_version": (ctypes.c_int, []),
    "hxc_shutdown": (c_st, []),
    "hxc_get_all_devices": (c_st, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(c_dev),
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "hxc_device_info": (c_st, [c_dev, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)]),
    "hxc_device_synchronize": (c_st, [c_dev]),
    "hxc_device_stream": (c_st, [c_dev, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "hxc_device_retain": (c_st, [c_dev]),
    "hxc_device_release": (c_st, [c_dev]),
    "hxc_host_alloc": (c_st, [ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "hxc_host_free": (c_st, [ctypes.c_void_p]),
    "hxc_device_create_buffer": (c_st, [c_dev, ctypes.c_size_t, ctypes.POINTER(c_buf)]),
    "hxc_buffer_wrap": (c_st, [c_dev, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(c_buf)]),
    "hxc_buffer_device_ptr": (c_st, [c_buf, ctypes.POINTER(ctypes.c_void_p),
                                     ctypes.POINTER(ctypes.c_size_t)]),
    "hxc_buffer_retain": (c_st, [c_buf]),
    "hxc_buffer_release": (c_st, [c_buf]),
    "hxc_buffer_enqueue_write": (c_st, [c_buf, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.POINTER(c_fut), ctypes.c_int,
                                        ctypes.POINTER(c_fut)]),
    "hxc_buffer_enqueue_read": (c_st, [c_buf, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.POINTER(c_fut), ctypes.c_int,
                                       ctypes.POINTER(c_fut)]),
    "hxc_buffer_enqueue_read_sync": (c_st, [c_buf, ctypes.c_size_t, ctypes.c_size_t,
                                            ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(c_fut),
                                            ctypes.c_int]),
    "hxc_buffer_enqueue_copy": (c_st, [c_buf, ctypes.c_size_t, c_buf, ctypes.c_size_t,
                                       ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(c_fut),
                                       ctypes.c_int, ctypes.POINTER(c_fut)]),
    "hxc_buffer_enqueue_write_2d": (c_st, [c_buf, ctypes.c_size_t, ctypes.c_size_t,
                                           ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                           ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(c_fut),
                                           ctypes.c_int, ctypes.POINTER(c_fut)]),
    "hxc_buffer_enqueue_read_2d": (c_st, [c_buf, ctypes.c_size_t, ctypes.c_size_t,
                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                          ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(c_fut),
                                          ctypes.c_int, ctypes.POINTER(c_fut)]),
    "hxc_future_is_ready": (c_st, [c_fut, ctypes.POINTER(ctypes.c_int)]),
    "hxc_future_wait": (c_st, [c_fut, ctypes.c_int64]),
    "hxc_wait_all": (c_st, [ctypes.POINTER(c_fut), ctypes.c_int, ctypes.c_int64]),
    "hxc_future_then": (c_st, [c_fut, HOST_FN, ctypes.c_void_p, ctypes.POINTER(c_fut)]),
    "hxc_when_all": (c_st, [ctypes.POINTER(c_fut), ctypes.c_int, ctypes.POINTER(c_fut)]),
    "hxc_make_ready_future": (c_st, [c_st, ctypes.POINTER(c_fut)]),
    "hxc_promise_create": (c_st, [ctypes.POINTER(c_fut)]),
    "hxc_promise_set": (c_st, [c_fut, c_st]),
    "hxc_debug_inject": (c_st, [i64, c_st]),
    "hxc_future_from_stream": (c_st, [c_dev, ctypes.c_void_p, ctypes.POINTER(c_fut)]),
    "hxc_future_stream_wait": (c_st, [c_fut, ctypes.c_void_p]),
    "hxc_future_retain": (c_st, [c_fut]),
    "hxc_future_release": (c_st, [c_fut]),
    "hxc_launch": (c_st, [c_dev, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                          ctypes.POINTER(hxc_launch_cfg), ctypes.c_int, ctypes.POINTER(c_fut),
                          ctypes.c_int, ctypes.POINTER(c_fut)]),
    "hxc_graph_begin": (c_st, [c_dev]),
    "hxc_graph_end": (c_st, [c_dev, ctypes.POINTER(c_graph)]),
    "hxc_graph_launch": (c_st, [c_graph, ctypes.c_int, ctypes.POINTER(c_fut), ctypes.c_int,
                                ctypes.POINTER(c_fut)]),
    "hxc_graph_node_count": (c_st, [c_graph, ctypes.POINTER(ctypes.c_size_t)]),
    "hxc_graph_release": (c_st, [c_graph]),
    "hxc_heat1d_run": (c_st, [c_dev, c_buf, c_buf, i64, ctypes.c_int, ctypes.c_double,
                              ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(c_fut),
                              ctypes.c_int, ctypes.POINTER(c_fut), ctypes.POINTER(hxc_run_stats)]),
    "hxc_heat2d_run": (c_st, [c_dev, c_buf, c_buf, ctypes.POINTER(hxc_heat2d_cfg),
                              ctypes.POINTER(c_fut), ctypes.c_int, ctypes.POINTER(c_fut),
                              ctypes.POINTER(c_fut), ctypes.POINTER(hxc_run_stats)]),
    "hxc_heat3d_run": (c_st, [c_dev, c_buf, c_buf, i64, i64, i64, ctypes.c_float, ctypes.c_int,
                              ctypes.c_int, ctypes.c_int, ctypes.POINTER(c_fut), ctypes.c_int,
                              ctypes.POINTER(c_fut), ctypes.POINTER(hxc_run_stats)]),
    "hxc_varcoef_batch_run": (c_st, [c_dev, c_buf, c_buf, ctypes.POINTER(i64),
                                     ctypes.POINTER(ctypes.c_double), i64, ctypes.c_int,
                                     ctypes.c_int, ctypes.POINTER(c_fut), ctypes.c_int,
                                     ctypes.POINTER(c_fut), ctypes.POINTER(hxc_run_stats)]),
    "hxc_sqerr_seed": (c_st, [c_dev, c_buf, c_buf, c_buf, c_buf, i64, ctypes.c_int,
                              ctypes.POINTER(c_fut), ctypes.c_int, ctypes.POINTER(c_fut)]),
    "hxc_varcoef_adjoint_run": (c_st, [c_dev, c_buf, c_buf, c_buf, i64, i64, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, c_buf, c_buf,
                                       c_buf, ctypes.POINTER(c_fut), ctypes.c_int,
                                       ctypes.POINTER(c_fut), ctypes.POINTER(hxc_run_stats)]),
    "hxc_varcoef_forward_run": (c_st, [c_dev, c_buf, c_buf, i64, i64, ctypes.c_double,
                                       ctypes.c_int, c_buf, ctypes.POINTER(c_fut), ctypes.c_int,
                                       ctypes.POINTER(c_fut), ctypes.POINTER(hxc_run_stats)]),
    "hxc_varcoef_tape_states": (c_st, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(i64)]),
    "hxc_varcoef_forward_tape": (c_st, [c_dev, c_buf, c_buf, i64, i64, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, c_buf, c_buf, ctypes.POINTER(c_fut),
                                        ctypes.c_int, ctypes.POINTER(c_fut),
                                        ctypes.POINTER(hxc_run_stats)]),
    "hxc_varcoef_adjoint_tape": (c_st, [c_dev, c_buf, c_buf, c_buf, i64, i64, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, c_buf, c_buf,
                                        ctypes.POINTER(c_fut), ctypes.c_int, ctypes.POINTER(c_fut),
                                        ctypes.POINTER(hxc_run_stats)]),
    "hxc_heat2d_step_kinds": (c_st, [ctypes.c_void_p, ctypes.POINTER(i64)]),
    "hxc_heat1d_step_kinds": (c_st, [ctypes.c_double, ctypes.c_int, ctypes.POINTER(i64)]),
    "hxc_host_norms": (c_st, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(i64), ctypes.c_int,
                              ctypes.c_void_p]),
    "hxc_heat2d_stream_run": (c_st, [c_dev, ctypes.c_void_p, ctypes.c_void_p, i64, i64, i64, i64,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(c_fut), ctypes.c_int, ctypes.POINTER(c_fut),
                                     ctypes.POINTER(hxc_run_stats)]),
    "hxc_partition_run": (c_st, [c_dev, ctypes.c_void_p, ctypes.c_void_p, i64, ctypes.c_int, c_buf,
                                 ctypes.POINTER(c_fut), ctypes.c_int, ctypes.POINTER(c_fut)]),
    "hxc_partition_run_native": (c_st, [c_dev, ctypes.c_void_p, ctypes.c_void_p, i64, ctypes.c_int,
                                        c_buf]),
    "hxc_png_write": (c_st, [ctypes.c_void_p, i64, i64, ctypes.c_int, ctypes.c_char_p]),
    "hxc_mandelbrot_png": (c_st, [c_dev, ctypes.POINTER(hxc_mandelbrot_args), ctypes.c_void_p,
                                  ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(c_fut), ctypes.c_int, ctypes.POINTER(c_fut)]),
    "hxc_program_create_with_source": (c_st, [c_dev, ctypes.c_char_p, ctypes.c_char_p,
                                              ctypes.POINTER(ctypes.c_void_p)]),
    "hxc_program_create_with_file": (c_st, [c_dev, ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]),
    "hxc_program_build": (c_st, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_char_p,
                                 ctypes.POINTER(c_fut), ctypes.c_int, ctypes.POINTER(c_fut)]),
    "hxc_program_build_log": (c_st, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t,
                                     ctypes.POINTER(ctypes.c_size_t)]),
    "hxc_program_run": (c_st, [ctypes.c_void_p, ctypes.c_char_p, ctypes.POINTER(hxc_kernel_arg),
                               ctypes.c_int, ctypes.POINTER(hxc_launch_cfg), ctypes.c_int,
                               ctypes.POINTER(c_fut), ctypes.c_int, ctypes.POINTER(c_fut)]),
    "hxc_program_release": (c_st, [ctypes.c_void_p]),
    "hxc_tune_set": (c_st, [ctypes.c_char_p, i64]),
    "hxc_tune_get": (c_st, [ctypes.c_char_p, ctypes.POINTER(i64)]),
    "hxc_tune_load": (c_st, [ctypes.c_char_p, ctypes.c_int, ctypes.c_int]),
    "hxc_tile_norms_noalloc": (c_st, [ctypes.c_void_p, i64, i64, i64, i64, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "hxc_debug_wait_errors": (c_st, [c_dev, ctypes.POINTER(ctypes.c_uint32)]),
    "hxc_pipe_rate": (c_st, [c_dev, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)]),
    "hxc_heat2d_run_host": (c_st, [c_dev, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(hxc_heat2d_cfg), ctypes.POINTER(hxc_run_stats)]),
    "hxc_heat2d_run_host_async": (c_st, [c_dev, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.POINTER(hxc_heat2d_cfg), ctypes.POINTER(c_fut),
                                         ctypes.c_int, ctypes.POINTER(c_fut),
                                         ctypes.POINTER(hxc_run_stats)]),
}

_lib = None


class HxcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


def lib():
    """The loaded libhxc.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libhxc.so not found at %s: build it with "
                "`python -m paper_1810_11482_b300.build` (there is no fallback)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(st, what=""):
    if st != HXC_OK:
        L = lib()
        raise HxcError(st, "%s: %s (%s)" % (what, L.hxc_status_string(st).decode(),
                                            L.hxc_last_error().decode()))
    return st


def _futs(deps):
    deps = list(deps or [])
    arr = (c_fut * max(1, len(deps)))(*[d.h if isinstance(d, Future) else d for d in deps])
    return arr, len(deps)


class Future:
    """Owning wrapper of an hxc_future handle (released on close/GC)."""

    def __init__(self, h):
        self.h = h

    def wait(self, timeout_ns=-1):
        return lib().hxc_future_wait(self.h, timeout_ns)

    def get(self, timeout_ns=-1):
        check(self.wait(timeout_ns), "future")

    def is_ready(self):
        r = ctypes.c_int(0)
        check(lib().hxc_future_is_ready(self.h, ctypes.byref(r)))
        return bool(r.value)

    def then(self, fn):
        """Host continuation: fn() -> None (raising -> HXC_E_CALLBACK)."""
        def tramp(_user):
            try:
                fn()
                return HXC_OK
            except Exception:
                return HXC_E_CALLBACK
        cb = HOST_FN(tramp)
        out = c_fut()
        check(lib().hxc_future_then(self.h, cb, None, ctypes.byref(out)), "then")
        f = Future(out.value)
        f._cb = cb  # keep the trampoline alive
        f._parent_cb = getattr(self, "_cb", None)
        return f

    def close(self):
        if self.h:
            lib().hxc_future_release(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def when_all(futs):
    arr, n = _futs(futs)
    out = c_fut()
    check(lib().hxc_when_all(arr, n, ctypes.byref(out)), "when_all")
    return Future(out.value)


class Graph:
    """Owning wrapper of an hxc_graph handle (released on close/GC)."""

    def __init__(self, h):
        self.h = h

    def launch(self, slot=0, deps=()):
        arr, n = _futs(deps)
        out = c_fut()
        check(lib().hxc_graph_launch(self.h, slot, arr, n, ctypes.byref(out)), "graph_launch")
        return Future(out.value)

    def node_count(self):
        n = ctypes.c_size_t()
        check(lib().hxc_graph_node_count(self.h, ctypes.byref(n)), "graph_node_count")
        return n.value

    def close(self):
        if self.h:
            lib().hxc_graph_release(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def graph_begin(dev):
    check(lib().hxc_graph_begin(dev.h), "graph_begin")


def graph_end(dev):
    out = c_graph()
    check(lib().hxc_graph_end(dev.h, ctypes.byref(out)), "graph_end")
    return Graph(out.value)


def wait_all(futs, timeout_ns=-1):
    arr, n = _futs(futs)
    return lib().hxc_wait_all(arr, n, timeout_ns)


def make_ready_future(status=HXC_OK):
    out = c_fut()
    check(lib().hxc_make_ready_future(status, ctypes.byref(out)))
    return Future(out.value)


def promise():
    out = c_fut()
    check(lib().hxc_promise_create(ctypes.byref(out)))
    return Future(out.value)


def promise_set(f, status=HXC_OK):
    check(lib().hxc_promise_set(f.h, status), "promise_set")


def debug_inject(after_ops, status=None):
    """Arms the host-side fault injection (hxc_debug_inject); after_ops < 0
    disarms."""
    check(lib().hxc_debug_inject(after_ops, HXC_E_CUDA if status is None else status),
          "debug_inject")


class Device:
    def __init__(self, h):
        self.h = h
        a, b, c, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        check(lib().hxc_device_info(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                    ctypes.byref(m)))
        self.major, self.minor, self.sm_count, self.global_mem = a.value, b.value, c.value, m.value

    def buffer(self, nbytes):
        out = c_buf()
        check(lib().hxc_device_create_buffer(self.h, nbytes, ctypes.byref(out)), "create_buffer")
        return Buffer(out.value, nbytes)

    def wrap(self, ptr, nbytes):
        out = c_buf()
        check(lib().hxc_buffer_wrap(self.h, ptr, nbytes, ctypes.byref(out)), "wrap")
        return Buffer(out.value, nbytes)

    def launch(self, kid, args, slot=0, deps=(), cfg=None):
        arr, n = _futs(deps)
        out = c_fut()
        pc = ctypes.byref(cfg) if cfg is not None else None
        check(lib().hxc_launch(self.h, kid, ctypes.byref(args), ctypes.sizeof(args), pc, slot,
                               arr, n, ctypes.byref(out)), "launch")
        return Future(out.value)

    def synchronize(self):
        check(lib().hxc_device_synchronize(self.h), "synchronize")

    def stream(self, slot):
        out = ctypes.c_void_p()
        check(lib().hxc_device_stream(self.h, slot, ctypes.byref(out)))
        return out.value


def get_all_devices(major=0, minor=0):
    L = lib()
    n = ctypes.c_int(0)
    arr = (c_dev * 16)()
    st = L.hxc_get_all_devices(major, minor, arr, 16, ctypes.byref(n))
    if st == HXC_E_NODEV:
        return []
    check(st, "get_all_devices")
    return [Device(arr[i]) for i in range(min(n.value, 16))]


class Buffer:
    def __init__(self, h, nbytes):
        self.h = h
        self.nbytes = nbytes

    @property
    def ptr(self):
        p = ctypes.c_void_p()
        check(lib().hxc_buffer_device_ptr(self.h, ctypes.byref(p), None))
        return p.value

    def write(self, host, off=0, slot=0, deps=()):
        """Async host->device copy of a C-contiguous numpy array."""
        host = np.ascontiguousarray(host)
        arr, n = _futs(deps)
        out = c_fut()
        check(lib().hxc_buffer_enqueue_write(self.h, off, host.nbytes, host.ctypes.data, slot,
                                             arr, n, ctypes.byref(out)), "enqueue_write")
        f = Future(out.value)
        f._host = host
        return f

    def read(self, host, off=0, slot=0, deps=()):
        arr, n = _futs(deps)
        out = c_fut()
        check(lib().hxc_buffer_enqueue_read(self.h, off, host.nbytes, host.ctypes.data, slot,
                                            arr, n, ctypes.byref(out)), "enqueue_read")
        f = Future(out.value)
        f._host = host
        return f

    def read_sync(self, host, off=0, slot=0, deps=()):
        arr, n = _futs(deps)
        check(lib().hxc_buffer_enqueue_read_sync(self.h, off, host.nbytes, host.ctypes.data,
                                                 slot, arr, n), "enqueue_read_sync")
        return host

    def close(self):
        if self.h:
            lib().hxc_buffer_release(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def heat1d_run(dev, u, tmp, n, parts, r, steps, mode="plain", steps_per_launch=0, deps=()):
    arr, nd = _futs(deps)
    out = c_fut()
    st = hxc_run_stats()
    check(lib().hxc_heat1d_run(dev.h, u.h, tmp.h, n, parts, r, steps, MODES[mode],
                               steps_per_launch, arr, nd, ctypes.byref(out), ctypes.byref(st)),
          "heat1d_run")
    return Future(out.value), st


def heat3d_run(dev, u, tmp, shape, r, steps, mode="fused", steps_per_launch=0, deps=()):
    arr, nd = _futs(deps)
    out = c_fut()
    st = hxc_run_stats()
    nz, ny, nx = shape
    check(lib().hxc_heat3d_run(dev.h, u.h, tmp.h, nz, ny, nx, r, steps, MODES[mode],
                               steps_per_launch, arr, nd, ctypes.byref(out), ctypes.byref(st)),
          "heat3d_run")
    return Future(out.value), st


def varcoef_batch_run(dev, u, kappa, sides, cs, steps, mode="fused", deps=()):
    sides = np.ascontiguousarray(sides, dtype=np.int64)
    cs = np.ascontiguousarray(cs, dtype=np.float64)
    arr, nd = _futs(deps)
    out = c_fut()
    st = hxc_run_stats()
    check(lib().hxc_varcoef_batch_run(dev.h, u.h, kappa.h, sides.ctypes.data_as(ctypes.POINTER(i64)),
                                      cs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      sides.size, steps, MODES[mode], arr, nd, ctypes.byref(out),
                                      ctypes.byref(st)), "varcoef_batch_run")
    return Future(out.value), st


def sqerr_seed(dev, u, t, lam, loss, n, slot=0, deps=()):
    arr, nd = _futs(deps)
    out = c_fut()
    check(lib().hxc_sqerr_seed(dev.h, u.h, t.h, lam.h if lam is not None else None, loss.h, n,
                               slot, arr, nd, ctypes.byref(out)), "sqerr_seed")
    return Future(out.value)


def varcoef_forward_run(dev, u0, kappa, ny, nx, c, steps, uT, deps=()):
    arr, nd = _futs(deps)
    out = c_fut()
    st = hxc_run_stats()
    check(lib().hxc_varcoef_forward_run(dev.h, u0.h, kappa.h, ny, nx, c, steps, uT.h, arr, nd,
                                        ctypes.byref(out), ctypes.byref(st)), "varcoef_forward_run")
    return Future(out.value), st


def varcoef_adjoint_run(dev, u0, kappa, lamT, ny, nx, c, steps, gk, gu0, uT=None, every=0,
                        mode="fused", deps=()):
    arr, nd = _futs(deps)
    out = c_fut()
    st = hxc_run_stats()
    check(lib().hxc_varcoef_adjoint_run(dev.h, u0.h, kappa.h, lamT.h, ny, nx, c, steps, every,
                                        MODES[mode], gk.h, gu0.h, uT.h if uT is not None else None,
                                        arr, nd, ctypes.byref(out), ctypes.byref(st)),
          "varcoef_adjoint_run")
    return Future(out.value), st


def varcoef_tape_states(steps, every=0):
    v = i64()
    check(lib().hxc_varcoef_tape_states(steps, every, ctypes.byref(v)), "varcoef_tape_states")
    return int(v.value)


def varcoef_forward_tape(dev, u0, kappa, ny, nx, c, steps, uT, tape, every=0, deps=()):
    arr, nd = _futs(deps)
    out = c_fut()
    st = hxc_run_stats()
    check(lib().hxc_varcoef_forward_tape(dev.h, u0.h, kappa.h, ny, nx, c, steps, every, uT.h,
                                         tape.h, arr, nd, ctypes.byref(out), ctypes.byref(st)),
          "varcoef_forward_tape")
    return Future(out.value), st


def varcoef_adjoint_tape(dev, tape, kappa, lamT, ny, nx, c, steps, gk, gu0, every=0,
                         mode="fused", deps=()):
    arr, nd = _futs(deps)
    out = c_fut()
    st = hxc_run_stats()
    check(lib().hxc_varcoef_adjoint_tape(dev.h, tape.h, kappa.h, lamT.h, ny, nx, c, steps, every,
                                         MODES[mode], gk.h, gu0.h, arr, nd, ctypes.byref(out),
                                         ctypes.byref(st)), "varcoef_adjoint_tape")
    return Future(out.value), st


def heat2d_cfg(ny, nx, tiles_y, tiles_x, r, steps, snapshot_every=0, mode="plain",
               host_norms=None, gpu_norms=None):
    c = hxc_heat2d_cfg()
    c.ny, c.nx, c.tiles_y, c.tiles_x = ny, nx, tiles_y, tiles_x
    c.r, c.steps, c.snapshot_every, c.mode = r, steps, snapshot_every, MODES[mode]
    dp = ctypes.POINTER(ctypes.c_double)
    c.host_norms = host_norms.ctypes.data_as(dp) if host_norms is not None else dp()
    c.gpu_norms = gpu_norms.ctypes.data_as(dp) if gpu_norms is not None else dp()
    c._keep = (host_norms, gpu_norms)
    return c


def heat2d_run(dev, u, tmp, cfg, deps=(), field_ready=False):
    """Returns (all-done future, stats), or (all-done, field-ready, stats)."""
    arr, nd = _futs(deps)
    out, fr = c_fut(), c_fut()
    st = hxc_run_stats()
    check(lib().hxc_heat2d_run(dev.h, u.h, tmp.h, ctypes.byref(cfg), arr, nd, ctypes.byref(out),
                               ctypes.byref(fr), ctypes.byref(st)), "heat2d_run")
    if field_ready:
        return Future(out.value), Future(fr.value), st
    lib().hxc_future_release(fr.value)
    return Future(out.value), st


def heat2d_run_host(dev, host_u0, host_uT, cfg):
    st = hxc_run_stats()
    check(lib().hxc_heat2d_run_host(dev.h, host_u0, host_uT, ctypes.byref(cfg),
                                    ctypes.byref(st)), "heat2d_run_host")
    return st


def heat2d_run_host_async(dev, host_u0, host_uT, cfg, deps=()):
    """Returns (future of the result in host_uT and the norms, stats).  The
    host arrays and cfg (with its norm arrays) must outlive the future."""
    arr, nd = _futs(deps)
    out = c_fut()
    st = hxc_run_stats()
    check(lib().hxc_heat2d_run_host_async(dev.h, host_u0, host_uT, ctypes.byref(cfg), arr, nd,
                                          ctypes.byref(out), ctypes.byref(st)),
          "heat2d_run_host_async")
    return Future(out.value), st


class _Pinned:
    """Owner of a page-locked host allocation, exposed to numpy."""

    def __init__(self, shape, dtype):
        nbytes = int(np.prod(shape)) * dtype.itemsize
        p = ctypes.c_void_p()
        check(lib().hxc_host_alloc(nbytes, ctypes.byref(p)), "host_alloc")
        self.ptr = p.value
        self.__array_interface__ = {"shape": tuple(shape), "typestr": dtype.str,
                                    "data": (self.ptr, False), "version": 3}

    def __del__(self):
        try:
            lib().hxc_host_free(self.ptr)
        except Exception:
            pass


def host_empty(shape, dtype=np.float64):
    """A numpy array over page-locked memory from hxc_host_alloc; the memory is
    freed when the array and all its views are gone."""
    if isinstance(shape, int):
        shape = (shape,)
    return np.asarray(_Pinned(shape, np.dtype(dtype)))


def debug_wait_errors(dev):
    """Reads and clears the record of device-side bounded waits that ran out
    (0: none)."""
    v = ctypes.c_uint32()
    check(lib().hxc_debug_wait_errors(dev.h, ctypes.byref(v)), "debug_wait_errors")
    return int(v.value)


def pipe_rate(dev, kind):
    """Measured throughput of one arithmetic pipe (HXC_PIPE_*): (operations
    per second, SM clock in MHz during the measurement)."""
    ops, mhz = ctypes.c_double(), ctypes.c_double()
    check(lib().hxc_pipe_rate(dev.h, kind, ctypes.byref(ops), ctypes.byref(mhz)), "pipe_rate")
    return ops.value, mhz.value


def tune_set(key, value):
    check(lib().hxc_tune_set(key.encode(), int(value)), "tune_set")


def tune_get(key):
    v = i64()
    check(lib().hxc_tune_get(key.encode(), ctypes.byref(v)), "tune_get")
    return int(v.value)


def tune_load(path, major=10, minor=3):
    check(lib().hxc_tune_load(str(path).encode(), major, minor), "tune_load")


def _f64_host(a, what):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError(what + " must be a C-contiguous float64 array")
    return a.ctypes.data


def heat1d_step_kinds(r, steps):
    """(canonical, scaled, closing) step counts of a 1D run."""
    out = (i64 * 3)()
    check(lib().hxc_heat1d_step_kinds(r, steps, out), "heat1d_step_kinds")
    return tuple(int(v) for v in out)


def heat2d_step_kinds(cfg):
    """(canonical, scaled, closing) step counts of a 2D run with this cfg."""
    out = (i64 * 3)()
    check(lib().hxc_heat2d_step_kinds(ctypes.byref(cfg), out), "heat2d_step_kinds")
    return tuple(int(v) for v in out)


def host_norms(arrays):
    """sqrt(sum v^2) of each float64 array on the host worker pool."""
    arrays = [np.ascontiguousarray(a, dtype=np.float64) for a in arrays]
    ptrs = (ctypes.c_void_p * max(1, len(arrays)))(*[a.ctypes.data for a in arrays])
    counts = (i64 * max(1, len(arrays)))(*[a.size for a in arrays])
    out = np.empty(len(arrays))
    check(lib().hxc_host_norms(ptrs, counts, len(arrays), out.ctypes.data), "host_norms")
    return out


def heat2d_stream_run(dev, host_a, host_b, tiles, r, steps, sequential=False, deps=()):
    """hxc_heat2d_stream_run on two (ny, nx) float64 host arrays; returns
    (future, stats, result array) -- the result is host_a after an even
    number of steps, host_b after an odd one."""
    if host_a.shape != host_b.shape or host_a.ndim != 2:
        raise ValueError("host_a and host_b must be (ny, nx) arrays of the same shape")
    ny, nx = host_a.shape
    arr, n = _futs(deps)
    out = c_fut()
    st = hxc_run_stats()
    check(lib().hxc_heat2d_stream_run(dev.h, _f64_host(host_a, "host_a"), _f64_host(host_b, "host_b"),
                                      ny, nx, tiles[0], tiles[1], r, steps, int(bool(sequential)),
                                      arr, n, ctypes.byref(out), ctypes.byref(st)),
          "heat2d_stream_run")
    f = Future(out.value)
    f._host = (host_a, host_b)
    return f, st, (host_a if steps % 2 == 0 else host_b)


def partition_run(dev, host_x, host_r, parts, work, deps=()):
    """Algorithm 1 on the futures layer (hxc_partition_run); returns the
    future of the last copy back.  host_x/host_r: float64 arrays (pinned
    ones from host_empty overlap)."""
    if host_r.size != host_x.size:
        raise ValueError("host_x and host_r differ in size")
    arr, n = _futs(deps)
    out = c_fut()
    check(lib().hxc_partition_run(dev.h, _f64_host(host_x, "host_x"), _f64_host(host_r, "host_r"),
                                  host_x.size, parts, work.h, arr, n, ctypes.byref(out)),
          "partition_run")
    f = Future(out.value)
    f._host = (host_x, host_r)
    return f


def partition_run_native(dev, host_x, host_r, parts, work):
    """The same loops as plain CUDA calls on the same streams; blocks."""
    if host_r.size != host_x.size:
        raise ValueError("host_x and host_r differ in size")
    check(lib().hxc_partition_run_native(dev.h, _f64_host(host_x, "host_x"),
                                         _f64_host(host_r, "host_r"), host_x.size, parts, work.h),
          "partition_run_native")


def mandelbrot_args(rgb, width, height, x0, y0, dx, dy, max_iter, counts=None):
    return hxc_mandelbrot_args(rgb.h, counts.h if counts is not None else None, width, height,
                               x0, y0, dx, dy, max_iter, 0)


def png_write(rgb, path, level=-1):
    """rgb: uint8 array (height, width, 3), C-contiguous."""
    if not (isinstance(rgb, np.ndarray) and rgb.dtype == np.uint8 and rgb.ndim == 3
            and rgb.shape[2] == 3 and rgb.flags.c_contiguous):
        raise ValueError("rgb must be a C-contiguous uint8 array of shape (h, w, 3)")
    check(lib().hxc_png_write(rgb.ctypes.data, rgb.shape[1], rgb.shape[0], level,
                              str(path).encode()), "png_write")


def mandelbrot_png(dev, args, host_rgb, path, level=-1, async_write=True, slot=0, deps=()):
    """One image to a PNG file (hxc_mandelbrot_png); returns the future of
    the file write.  host_rgb: uint8 array of width*height*3 bytes."""
    if host_rgb.dtype != np.uint8 or host_rgb.size < args.width * args.height * 3:
        raise ValueError("host_rgb must be a uint8 array of width*height*3 bytes")
    arr, n = _futs(deps)
    out = c_fut()
    check(lib().hxc_mandelbrot_png(dev.h, ctypes.byref(args), host_rgb.ctypes.data,
                                   str(path).encode(), level, int(bool(async_write)), slot, arr, n,
                                   ctypes.byref(out)), "mandelbrot_png")
    f = Future(out.value)
    f._host = host_rgb
    return f


class Program:
    """A run-time compiled program (the paper's `program`)."""

    def __init__(self, h):
        self.h = h

    @staticmethod
    def from_file(dev, path):
        out = ctypes.c_void_p()
        check(lib().hxc_program_create_with_file(dev.h, str(path).encode(), ctypes.byref(out)),
              "create_program_with_file")
        return Program(out.value)

    @staticmethod
    def from_source(dev, source, name="program.cu"):
        out = ctypes.c_void_p()
        check(lib().hxc_program_create_with_source(dev.h, source.encode(), name.encode(),
                                                   ctypes.byref(out)), "create_program")
        return Program(out.value)

    def build(self, kernel_names, options=None, deps=()):
        arr, n = _futs(deps)
        out = c_fut()
        check(lib().hxc_program_build(self.h, kernel_names.encode(),
                                      options.encode() if options else None, arr, n,
                                      ctypes.byref(out)), "build")
        return Future(out.value)

    def log(self):
        n = ctypes.c_size_t()
        check(lib().hxc_program_build_log(self.h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value + 1)
        check(lib().hxc_program_build_log(self.h, buf, n.value + 1, None))
        return buf.value.decode(errors="replace")

    def run(self, name, args, grid, block, slot=0, deps=()):
        """args: Buffer objects or (ctypes scalar) values."""
        arr = (hxc_kernel_arg * max(1, len(args)))()
        keep = []
        for i, a in enumerate(args):
            if isinstance(a, Buffer):
                arr[i].buf = a.h
            else:
                keep.append(a)
                arr[i].value = ctypes.cast(ctypes.pointer(a), ctypes.c_void_p)
                arr[i].size = ctypes.sizeof(a)
        cfg = hxc_launch_cfg(tuple(grid), tuple(block))
        darr, n = _futs(deps)
        out = c_fut()
        check(lib().hxc_program_run(self.h, name.encode(), arr, len(args), ctypes.byref(cfg), slot,
                                    darr, n, ctypes.byref(out)), "run")
        return Future(out.value)

    def close(self):
        if self.h:
            lib().hxc_program_release(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
