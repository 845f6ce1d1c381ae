"""ctypes binding of libgdag (include/gdag.h): the same calls, argument
marshalling only.  Every step of the hot path runs in the library's C++ runtime
and CUDA kernels; nothing here computes.

Module-level functions carry the C names and raise :class:`GdagError` on a
negative status.  :class:`Context` is a thin convenience layer over them that
accepts torch tensors (device memory) and Python scalars.
"""
from __future__ import annotations

import ctypes
import numbers
import os
import struct

# The scheduler runs independent nodes on up to max_streams (default 16)
# streams.  CUDA maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware work
# queues, 8 unless set: streams sharing a queue are serialised behind each
# other's cross-stream waits once the host issues ahead of the device, which
# turns a multi-stream DAG back into a partly serial one.  32 (the maximum)
# gives every pool stream its own queue; it must be set before the process
# creates its CUDA context, so it is set here, at import, unless the caller
# chose a value.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgdag.so")

# ---------------------------------------------------------------- constants
GDAG_OK = 0
GDAG_ERR_INVALID = -1
GDAG_ERR_CUDA = -2
GDAG_ERR_TIMEOUT = -3
GDAG_ERR_OOM = -4
GDAG_ERR_POISONED = -5
GDAG_ERR_BUSY = -6
GDAG_ERR_NOT_FOUND = -7
ERR_NAMES = {0: "OK", -1: "INVALID", -2: "CUDA", -3: "TIMEOUT", -4: "OOM", -5: "POISONED",
             -6: "BUSY", -7: "NOT_FOUND"}

GDAG_POLICY_SERIAL_SYNC = 0
GDAG_POLICY_SERIAL_ASYNC = 1
GDAG_POLICY_PARALLEL = 2
GDAG_BACKEND_CUDA = 0
GDAG_BACKEND_FAKE = 1

GDAG_MODE_DEFAULT = 0
GDAG_MODE_IN = 1
GDAG_MODE_CONST = 2
GDAG_MODE_OUT = 3
GDAG_MODE_INOUT = 4
GDAG_MODE_SIGNATURE = -1

GDAG_EDGE_RAW, GDAG_EDGE_WAR, GDAG_EDGE_WAW = 0, 1, 2
GDAG_NODE_KERNEL, GDAG_NODE_HOST_WRITE, GDAG_NODE_HOST_READ, GDAG_NODE_EXTERNAL, GDAG_NODE_HOST_PREFETCH = 0, 1, 2, 3, 4
GDAG_NODE_GRAPH = 5
GDAG_ARG_ARRAY, GDAG_ARG_SCALAR = 0, 1
GDAG_ELEM_LAUNCH, GDAG_ELEM_LAUNCH_FUSED, GDAG_ELEM_WRITE, GDAG_ELEM_PREFETCH_HOST = 0, 1, 2, 3
GDAG_FUSED_MAX = 4096     # members per gdag_launch_fused call
GDAG_FUSED_TABLE = 128    # members per persistent launch of a fused element
GDAG_AUTO_GRAPH_SEQS = 64 # sequences the automatic capture keeps (options.auto_graph)
(GDAG_OP_LAUNCH, GDAG_OP_COPY_H2D, GDAG_OP_COPY_D2H, GDAG_OP_EXTERNAL, GDAG_OP_RECORD, GDAG_OP_WAIT,
 GDAG_OP_HOST_WAIT, GDAG_OP_STREAM_SYNC, GDAG_OP_HOST_NODE, GDAG_OP_QUERY_DONE) = range(10)


# ---------------------------------------------------------------- structs
class gdag_dim3(ctypes.Structure):
    _fields_ = [("x", ctypes.c_uint32), ("y", ctypes.c_uint32), ("z", ctypes.c_uint32)]


class gdag_options(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int32), ("backend", ctypes.c_int32), ("device", ctypes.c_int32),
                ("max_streams", ctypes.c_int32), ("prefetch", ctypes.c_int32),
                ("retire_by_query", ctypes.c_int32), ("record_log", ctypes.c_int32),
                ("trace", ctypes.c_int32), ("timeout_ms", ctypes.c_int32), ("trim_nodes", ctypes.c_int32),
                ("fake_complete", ctypes.c_int32), ("fake_fail_sticky", ctypes.c_int32),
                ("fake_fail_op", ctypes.c_int64), ("stream_priority", ctypes.c_int32), ("auto_graph", ctypes.c_int32)]


class gdag_arg(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("mode", ctypes.c_int32), ("array", ctypes.c_int32),
                ("size", ctypes.c_int32), ("value", ctypes.c_uint64)]


class gdag_argspec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("mode", ctypes.c_int32), ("size", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class gdag_edge(ctypes.Structure):
    _fields_ = [("src", ctypes.c_int64), ("dst", ctypes.c_int64), ("array", ctypes.c_int32),
                ("kind", ctypes.c_int32)]


class gdag_node_info(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("kind", ctypes.c_int32), ("stream", ctypes.c_int32)]


class gdag_op(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("stream", ctypes.c_int32), ("event", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("node", ctypes.c_int64)]


class gdag_trace_rec(ctypes.Structure):
    _fields_ = [("node", ctypes.c_int64), ("kind", ctypes.c_int32), ("stream", ctypes.c_int32),
                ("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double)]


class gdag_stats(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_int64), ("edges", ctypes.c_int64), ("waits", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("copies", ctypes.c_int64), ("host_waits", ctypes.c_int64),
                ("streams", ctypes.c_int32), ("active", ctypes.c_int32), ("fused_members", ctypes.c_int64),
                ("held_nodes", ctypes.c_int64), ("held_readers", ctypes.c_int64)]


class gdag_elem(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("kernel", ctypes.c_int32), ("array", ctypes.c_int32),
                ("nargs", ctypes.c_int32), ("count", ctypes.c_int32), ("smem", ctypes.c_uint32),
                ("arg0", ctypes.c_int64), ("off", ctypes.c_uint64), ("bytes", ctypes.c_uint64),
                ("grid", gdag_dim3), ("block", gdag_dim3)]


EXTERNAL_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_P = ctypes.POINTER
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_ctx = ctypes.c_void_p

# name -> (restype, argtypes)
SIGNATURES = {
    "gdag_options_default": (None, [_P(gdag_options)]),
    "gdag_create": (ctypes.c_int, [_P(_ctx), _P(gdag_options)]),
    "gdag_destroy": (ctypes.c_int, [_ctx]),
    "gdag_last_error": (ctypes.c_char_p, [_ctx]),
    "gdag_add_stream": (ctypes.c_int, [_ctx, _vp]),
    "gdag_array_register": (ctypes.c_int, [_ctx, _vp, _sz, _vp, _P(_i32)]),
    "gdag_array_unregister": (ctypes.c_int, [_ctx, _i32]),
    "gdag_array_host": (ctypes.c_int, [_ctx, _i32, _i32, _P(_vp)]),
    "gdag_array_write": (ctypes.c_int, [_ctx, _i32, _vp, _sz, _sz]),
    "gdag_array_read": (ctypes.c_int, [_ctx, _i32, _vp, _sz, _sz]),
    "gdag_array_prefetch_host": (ctypes.c_int, [_ctx, _i32, _sz, _sz]),
    "gdag_kernel_lookup": (ctypes.c_int, [_ctx, ctypes.c_char_p, _P(_i32)]),
    "gdag_kernel_signature": (ctypes.c_int, [_ctx, _i32, _P(_i32), _P(gdag_argspec), _i32]),
    "gdag_kernel_register": (ctypes.c_int, [_ctx, ctypes.c_char_p, _vp, _i32, _P(gdag_argspec), _P(_i32)]),
    "gdag_launch": (ctypes.c_int, [_ctx, _i32, gdag_dim3, gdag_dim3, _sz, _P(gdag_arg), _i32, _P(_i64)]),
    "gdag_launch_raw": (ctypes.c_int, [_ctx, _i32, gdag_dim3, gdag_dim3, _sz, _P(gdag_arg), _i32, _vp]),
    "gdag_launch_fused": (ctypes.c_int, [_ctx, _i32, _P(gdag_arg), _i32, _i32, _P(_i64)]),
    "gdag_launch_external": (ctypes.c_int, [_ctx, EXTERNAL_FN, _vp, _P(_i32), _P(_i32), _i32, _P(_i64)]),
    "gdag_sync": (ctypes.c_int, [_ctx]),
    "gdag_stream_wait_all": (ctypes.c_int, [_ctx, _vp]),
    "gdag_stream_fork": (ctypes.c_int, [_ctx, _vp]),
    "gdag_dag_export": (ctypes.c_int, [_ctx, _P(gdag_edge), _sz, _P(_sz)]),
    "gdag_nodes_export": (ctypes.c_int, [_ctx, _P(gdag_node_info), _sz, _P(_sz)]),
    "gdag_ops_export": (ctypes.c_int, [_ctx, _P(gdag_op), _sz, _P(_sz)]),
    "gdag_trace_export": (ctypes.c_int, [_ctx, _P(gdag_trace_rec), _sz, _P(_sz)]),
    "gdag_stats_get": (ctypes.c_int, [_ctx, _P(gdag_stats)]),
    "gdag_trace_write": (ctypes.c_int, [_ctx, ctypes.c_char_p]),
    "gdag_node_query": (ctypes.c_int, [_ctx, _i64, _P(_i32)]),
    "gdag_nodes_query": (ctypes.c_int, [_ctx, _vp, _i32, _vp]),
    "gdag_issue": (ctypes.c_int, [_ctx, _vp, _i32, _vp, _i64, _vp, _P(_i32)]),
    "gdag_capture_begin": (ctypes.c_int, [_ctx]),
    "gdag_capture_end": (ctypes.c_int, [_ctx, _P(_i32)]),
    "gdag_graph_launch": (ctypes.c_int, [_ctx, _i32, _P(_i64)]),
    "gdag_graph_destroy": (ctypes.c_int, [_ctx, _i32]),
    "gdag_scratch_bytes": (_sz, [ctypes.c_char_p, _i64]),
    "gdag_vec_reduce_diff_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp]),
}

_lib = None
_LAUNCH = [None]  # gdag_launch, bound once by lib()


class GdagError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gdag error %d (%s): %s" % (code, ERR_NAMES.get(code, "?"), msg))
        self.code = code


def lib():
    """Load libgdag.so (built in-tree by __graft_entry__.build()).  There is
    no fallback: a missing library is an error."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libgdag.so not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LAUNCH[0] = L.gdag_launch
        _lib = L
    return _lib


def _check(ctx, code):
    if code < 0:
        msg = lib().gdag_last_error(ctx) if ctx else b""
        raise GdagError(code, (msg or b"").decode(errors="replace"))
    return code


# ---------------------------------------------------------- C-named calls
def gdag_options_default():
    o = gdag_options()
    lib().gdag_options_default(ctypes.byref(o))
    return o


def gdag_create(opts=None):
    h = _ctx()
    code = lib().gdag_create(ctypes.byref(h), ctypes.byref(opts) if opts is not None else None)
    if code < 0:
        raise GdagError(code, "gdag_create failed")
    return h


def gdag_destroy(ctx):
    return _check(None, lib().gdag_destroy(ctx))


def gdag_add_stream(ctx, stream):
    return _check(ctx, lib().gdag_add_stream(ctx, stream))


def gdag_array_register(ctx, dev, nbytes, host=None):
    a = _i32()
    _check(ctx, lib().gdag_array_register(ctx, dev, nbytes, host, ctypes.byref(a)))
    return a.value


def gdag_array_unregister(ctx, a):
    return _check(ctx, lib().gdag_array_unregister(ctx, a))


def gdag_array_host(ctx, a, mode):
    p = _vp()
    _check(ctx, lib().gdag_array_host(ctx, a, mode, ctypes.byref(p)))
    return p.value


def gdag_array_write(ctx, a, src, off, nbytes):
    return _check(ctx, lib().gdag_array_write(ctx, a, src, off, nbytes))


def gdag_array_read(ctx, a, dst, off, nbytes):
    return _check(ctx, lib().gdag_array_read(ctx, a, dst, off, nbytes))


def gdag_array_prefetch_host(ctx, a, off, nbytes):
    return _check(ctx, lib().gdag_array_prefetch_host(ctx, a, off, nbytes))


def gdag_kernel_lookup(ctx, name):
    k = _i32()
    _check(ctx, lib().gdag_kernel_lookup(ctx, name.encode(), ctypes.byref(k)))
    return k.value


def gdag_kernel_signature(ctx, k):
    n = _i32()
    spec = (gdag_argspec * 16)()
    _check(ctx, lib().gdag_kernel_signature(ctx, k, ctypes.byref(n), spec, 16))
    return [spec[i] for i in range(n.value)]


def gdag_kernel_register(ctx, name, fn, specs):
    k = _i32()
    arr = (gdag_argspec * max(1, len(specs)))(*specs)
    _check(ctx, lib().gdag_kernel_register(ctx, name.encode(), fn, len(specs), arr, ctypes.byref(k)))
    return k.value


def gdag_launch(ctx, k, grid, block, smem, args):
    node = _i64()
    arr = (gdag_arg * max(1, len(args)))(*args)
    _check(ctx, lib().gdag_launch(ctx, k, grid, block, smem, arr, len(args), ctypes.byref(node)))
    return node.value


def gdag_launch_fused(ctx, k, args, nargs, count):
    """args: count * nargs gdag_arg values, member after member."""
    node = _i64()
    arr = (gdag_arg * max(1, len(args)))(*args)
    _check(ctx, lib().gdag_launch_fused(ctx, k, arr, nargs, count, ctypes.byref(node)))
    return node.value


def gdag_launch_raw(ctx, k, grid, block, smem, args, stream):
    arr = (gdag_arg * max(1, len(args)))(*args)
    return _check(ctx, lib().gdag_launch_raw(ctx, k, grid, block, smem, arr, len(args), stream))


def gdag_launch_external(ctx, fn, user, arrays, modes):
    node = _i64()
    n = len(arrays)
    a = (_i32 * max(1, n))(*arrays)
    m = (_i32 * max(1, n))(*modes)
    _check(ctx, lib().gdag_launch_external(ctx, fn, user, a, m, n, ctypes.byref(node)))
    return node.value


def gdag_sync(ctx):
    return _check(ctx, lib().gdag_sync(ctx))


def gdag_stream_wait_all(ctx, stream):
    return _check(ctx, lib().gdag_stream_wait_all(ctx, stream))


def gdag_stream_fork(ctx, stream):
    return _check(ctx, lib().gdag_stream_fork(ctx, stream))


def _export(ctx, fn, T):
    n = _sz()
    _check(ctx, fn(ctx, None, 0, ctypes.byref(n)))
    buf = (T * max(1, n.value))()
    _check(ctx, fn(ctx, buf, n.value, ctypes.byref(n)))
    return [buf[i] for i in range(n.value)]


def gdag_dag_export(ctx):
    return _export(ctx, lib().gdag_dag_export, gdag_edge)


def gdag_nodes_export(ctx):
    return _export(ctx, lib().gdag_nodes_export, gdag_node_info)


def gdag_ops_export(ctx):
    return _export(ctx, lib().gdag_ops_export, gdag_op)


def gdag_trace_export(ctx):
    return _export(ctx, lib().gdag_trace_export, gdag_trace_rec)


def gdag_trace_write(ctx, path):
    return _check(ctx, lib().gdag_trace_write(ctx, os.fsencode(path)))


def gdag_stats_get(ctx):
    s = gdag_stats()
    _check(ctx, lib().gdag_stats_get(ctx, ctypes.byref(s)))
    return s


def gdag_node_query(ctx, node):
    d = _i32()
    _check(ctx, lib().gdag_node_query(ctx, node, ctypes.byref(d)))
    return bool(d.value)


def gdag_nodes_query(ctx, nodes):
    """Completion flags of a sequence of node ids (one C call)."""
    import numpy as np
    nd = np.ascontiguousarray(nodes, dtype=np.int64)
    done = np.zeros(nd.size, dtype=np.int32)
    _check(ctx, lib().gdag_nodes_query(ctx, nd.ctypes.data, nd.size, done.ctypes.data))
    return done


def gdag_issue(ctx, elems, args):
    """Issue a ctypes array of gdag_elem against a ctypes array of gdag_arg;
    returns the node ids (-1 where an element made none)."""
    n = len(elems)
    nodes = (_i64 * max(1, n))()
    issued = _i32()
    r = lib().gdag_issue(ctx, ctypes.addressof(elems) if n else None, n,
                         ctypes.addressof(args) if len(args) else None, len(args), ctypes.addressof(nodes),
                         ctypes.byref(issued))
    if r < 0:
        e = GdagError(r, (lib().gdag_last_error(ctx) or b"").decode(errors="replace"))
        e.issued = issued.value
        e.nodes = [nodes[i] for i in range(n)]
        raise e
    return [nodes[i] for i in range(n)]


def gdag_capture_begin(ctx):
    return _check(ctx, lib().gdag_capture_begin(ctx))


def gdag_capture_end(ctx):
    g = _i32()
    _check(ctx, lib().gdag_capture_end(ctx, ctypes.byref(g)))
    return g.value


def gdag_graph_launch(ctx, g):
    node = _i64()
    _check(ctx, lib().gdag_graph_launch(ctx, g, ctypes.byref(node)))
    return node.value


def gdag_graph_destroy(ctx, g):
    return _check(ctx, lib().gdag_graph_destroy(ctx, g))


def gdag_scratch_bytes(kernel, n):
    return lib().gdag_scratch_bytes(kernel.encode(), n)


def gdag_vec_reduce_diff_noalloc(dev_x, dev_y, dev_z, n, stream):
    """The allocation-free VEC reduction (no context; caller's stream)."""
    return _check(None, lib().gdag_vec_reduce_diff_noalloc(dev_x, dev_y, dev_z, n, stream))


# ------------------------------------------------------------ convenience
def array_arg(a, mode=GDAG_MODE_SIGNATURE):
    return gdag_arg(GDAG_ARG_ARRAY, mode, a, 0, 0)


def scalar_arg(value, size):
    return gdag_arg(GDAG_ARG_SCALAR, 0, 0, size, _scalar_bits(value, size))


_F32 = struct.Struct("<f")
_U32 = struct.Struct("<I")
_F64 = struct.Struct("<d")
_U64 = struct.Struct("<Q")
_ARG = struct.Struct("<iiiiQ")  # gdag_arg: kind, mode, array, size, value
assert _ARG.size == ctypes.sizeof(gdag_arg)


def _scalar_bits(value, size):
    """The value field of a scalar argument (as scalar_arg builds it):
    integers (Python or numpy, and bool) as two's complement, anything else
    (Python or numpy floats) as an IEEE float of `size` bytes."""
    if isinstance(value, numbers.Integral):
        return int(value) & ((1 << (8 * size)) - 1)
    value = float(value)
    return _U32.unpack(_F32.pack(value))[0] if size == 4 else _U64.unpack(_F64.pack(value))[0]


def _scalar_key(a):
    """Cache key of a scalar argument that is not an int or a nonzero float:
    equal keys give equal argument bits.  Value equality alone would not do
    (-0.0 == 0.0), so these keys add the value's bits as a double.  (A
    nonzero Python float is its own key: equal nonzero floats have equal
    bits, and a NaN, never equal, only misses the cache.)"""
    c = a.__class__
    if c is int:
        return (c, a)
    try:
        return (c, a, _F64.pack(a))
    except (struct.error, TypeError):  # not convertible to a double
        return (c, a)


class Array:
    """A registered array: a handle plus what it was registered with."""

    __slots__ = ("handle", "nbytes", "tensor", "host", "name")

    def __init__(self, handle, nbytes, tensor=None, host=None, name=None):
        self.handle, self.nbytes, self.tensor, self.host, self.name = handle, nbytes, tensor, host, name

    def __repr__(self):
        return "Array(%d, %s, %d B)" % (self.handle, self.name, self.nbytes)


class Mode:
    """Per-call access-mode override: ``ctx.launch(k, Mode(a, GDAG_MODE_IN), ...)``."""

    __slots__ = ("array", "mode")

    def __init__(self, array, mode):
        self.array, self.mode = array, mode


class Context:
    """One gdag context.  ``backend='fake'`` records operations only."""

    def __init__(self, policy=GDAG_POLICY_PARALLEL, backend="cuda", device=0, max_streams=16, prefetch=True,
                 retire_by_query=False, record_log=False, trace=False, timeout_ms=60000, trim_nodes=0,
                 fake_complete=False, fake_fail_op=-1, fake_fail_sticky=False, stream_priority=0, auto_graph=0):
        o = gdag_options_default()
        o.policy = policy
        o.backend = GDAG_BACKEND_FAKE if backend == "fake" else GDAG_BACKEND_CUDA
        o.device = device
        o.max_streams = max_streams
        o.prefetch = int(prefetch)
        o.retire_by_query = int(retire_by_query)
        o.record_log = int(record_log)
        o.trace = int(trace)
        o.timeout_ms = timeout_ms
        o.trim_nodes = trim_nodes
        o.fake_complete = int(fake_complete)
        o.fake_fail_op = fake_fail_op
        o.fake_fail_sticky = int(fake_fail_sticky)
        o.stream_priority = stream_priority
        o.auto_graph = auto_graph
        self.options = o
        self.h = gdag_create(o)
        self._kernels = {}
        self._prepared = {}  # marshalled argument arrays of repeated launches
        self._packed = {}    # packed argument bytes of repeated fused-launch members

    # lifetime
    def close(self):
        if self.h:
            h, self.h = self.h, None
            gdag_destroy(h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def last_error(self):
        return (lib().gdag_last_error(self.h) or b"").decode()

    # arrays
    def array(self, tensor=None, *, dev=None, nbytes=None, host=None, name=None):
        """Register a torch tensor (device memory) or a raw (dev, nbytes)."""
        if tensor is not None:
            dev = tensor.data_ptr()
            nbytes = tensor.numel() * tensor.element_size()
        hptr = host.data_ptr() if host is not None and hasattr(host, "data_ptr") else host
        h = gdag_array_register(self.h, dev, nbytes, hptr)
        return Array(h, nbytes, tensor, host, name)

    def unregister(self, a):
        gdag_array_unregister(self.h, a.handle)

    def host_view(self, a, mode):
        return gdag_array_host(self.h, a.handle, mode)

    def write(self, a, src=None, off=0, nbytes=None):
        """Host write; src is a host pointer (int), a numpy array or None."""
        nbytes = a.nbytes - off if nbytes is None else nbytes
        ptr = _host_ptr(src)
        gdag_array_write(self.h, a.handle, ptr, off, nbytes)

    def read(self, a, dst=None, off=0, nbytes=None):
        nbytes = a.nbytes - off if nbytes is None else nbytes
        gdag_array_read(self.h, a.handle, _host_ptr(dst), off, nbytes)

    def prefetch_host(self, a, off=0, nbytes=None):
        nbytes = a.nbytes - off if nbytes is None else nbytes
        gdag_array_prefetch_host(self.h, a.handle, off, nbytes)

    # kernels
    def kernel(self, name):
        k = self._kernels.get(name)
        if k is None:
            kid = gdag_kernel_lookup(self.h, name)
            k = (kid, gdag_kernel_signature(self.h, kid))
            self._kernels[name] = k
        return k

    def _pack(self, name, args, out):
        """Append the gdag_arg bytes of one launch of `name` to the bytearray
        `out` (the same values _args builds, one struct.pack per argument
        instead of one ctypes structure); returns the kernel handle.  The
        bytes of a member seen before (same kernel, handles, modes and typed
        scalars) come from a cache."""
        key = (name,) + tuple(
            a.handle if a.__class__ is Array else
            (Mode, a.array.handle, a.mode) if a.__class__ is Mode else
            (int, a) if a.__class__ is int else
            (float, a) if a.__class__ is float and a else _scalar_key(a) for a in args)
        hit = self._packed.get(key)
        if hit is not None:
            out += hit[1]
            return hit[0]
        start = len(out)
        kid = self._pack_new(name, args, out)
        if len(self._packed) >= 4096:
            self._packed.clear()
        self._packed[key] = (kid, bytes(out[start:]))
        return kid

    def _pack_new(self, name, args, out):
        kid, spec = self.kernel(name)
        if len(args) != len(spec):
            raise GdagError(GDAG_ERR_INVALID, "%s takes %d arguments, got %d" % (name, len(spec), len(args)))
        pack = _ARG.pack
        for sp, v in zip(spec, args):
            if sp.kind == GDAG_ARG_ARRAY:
                if v.__class__ is Mode:
                    out += pack(GDAG_ARG_ARRAY, v.mode, v.array.handle, 0, 0)
                else:
                    out += pack(GDAG_ARG_ARRAY, GDAG_MODE_SIGNATURE, v.handle, 0, 0)
            else:
                out += pack(GDAG_ARG_SCALAR, 0, 0, sp.size, _scalar_bits(v, sp.size))
        return kid

    def _args(self, name, args):
        kid, spec = self.kernel(name)
        if len(args) != len(spec):
            raise GdagError(GDAG_ERR_INVALID, "%s takes %d arguments, got %d" % (name, len(spec), len(args)))
        out = []
        for s, v in zip(spec, args):
            if s.kind == GDAG_ARG_ARRAY:
                if isinstance(v, Mode):
                    out.append(array_arg(v.array.handle, v.mode))
                else:
                    out.append(array_arg(v.handle))
            else:
                out.append(scalar_arg(v, s.size))
        return kid, out

    def launch(self, name, *args, grid=None, block=None, smem=0):
        # A program issues the same launches step after step: their ctypes
        # argument arrays are built once and reused (keyed by kernel, launch
        # shape, array handles, access-mode overrides and typed scalars), so a
        # repeated launch costs one C call.  The dependency inference, stream
        # choice and event waits still run on every launch, in the library.
        key = (name, tuple(grid) if grid else None, tuple(block) if block else None, smem) + tuple(
            a.handle if a.__class__ is Array else
            (Mode, a.array.handle, a.mode) if a.__class__ is Mode else
            (int, a) if a.__class__ is int else
            (float, a) if a.__class__ is float and a else _scalar_key(a) for a in args)
        p = self._prepared.get(key)
        if p is None:
            buf = bytearray()
            kid = self._pack(name, args, buf)
            n = len(args)
            g = gdag_dim3(*grid) if grid else gdag_dim3(0, 0, 0)
            b = gdag_dim3(*block) if block else gdag_dim3(0, 0, 0)
            arr = (gdag_arg * max(1, n)).from_buffer_copy(buf) if n else (gdag_arg * 1)()
            p = (kid, g, b, smem, arr, n, _i64())
            if len(self._prepared) >= 4096:
                self._prepared.clear()
            self._prepared[key] = p
        kid, g, b, sm, arr, n, node = p
        r = _LAUNCH[0](self.h, kid, g, b, sm, arr, n, ctypes.byref(node))
        if r:
            _check(self.h, r)
        return node.value

    def launch_fused(self, name, members):
        """One DAG element and one persistent launch for several launches of
        built-in kernel `name`; `members` is a list of argument tuples, each
        as `launch` would take it."""
        if not members:
            raise GdagError(GDAG_ERR_INVALID, "fused launch of no members")
        buf = bytearray()
        kid = None
        for m in members:
            kid = self._pack(name, m, buf)
        nargs = len(members[0])
        arr = (gdag_arg * (len(buf) // _ARG.size)).from_buffer_copy(buf)
        node = _i64()
        _check(self.h, lib().gdag_launch_fused(self.h, kid, arr, nargs, len(members), ctypes.byref(node)))
        return node.value

    def program(self):
        """A new :class:`Program` recording elements for this context."""
        return Program(self)

    def done_many(self, nodes):
        """Non-blocking: completion flags of several nodes (one C call)."""
        return gdag_nodes_query(self.h, nodes)

    def launch_raw(self, name, *args, stream, grid=None, block=None, smem=0):
        kid, a = self._args(name, args)
        g = gdag_dim3(*grid) if grid else gdag_dim3(0, 0, 0)
        b = gdag_dim3(*block) if block else gdag_dim3(0, 0, 0)
        gdag_launch_raw(self.h, kid, g, b, smem, a, stream)

    def external(self, fn, arrays_modes, user=None):
        # the library calls fn before gdag_launch_external returns and keeps
        # no reference to it, so the ctypes thunk only has to outlive the call
        cb = EXTERNAL_FN(fn)
        return gdag_launch_external(self.h, cb, user, [a.handle for a, _ in arrays_modes],
                                    [m for _, m in arrays_modes])

    # captured DAG shapes
    def capture(self, fn):
        """Record fn() (which issues elements on this context) as a graph;
        returns its handle."""
        gdag_capture_begin(self.h)
        try:
            fn()
        except BaseException:
            gdag_capture_end(self.h)
            raise
        return gdag_capture_end(self.h)

    def done(self, node):
        """Non-blocking: has this node completed?"""
        return gdag_node_query(self.h, node)

    def replay(self, g):
        return gdag_graph_launch(self.h, g)

    def drop_graph(self, g):
        gdag_graph_destroy(self.h, g)

    # sync and inspection
    def sync(self):
        gdag_sync(self.h)

    def wait_all(self, stream):
        gdag_stream_wait_all(self.h, stream)

    def fork(self, stream):
        gdag_stream_fork(self.h, stream)

    def edges(self):
        return [(e.src, e.dst, e.array, e.kind) for e in gdag_dag_export(self.h)]

    def nodes(self):
        return [(n.id, n.kind, n.stream) for n in gdag_nodes_export(self.h)]

    def ops(self):
        return [(o.type, o.stream, o.event, o.node) for o in gdag_ops_export(self.h)]

    def trace(self):
        return [(t.node, t.kind, t.stream, t.start_ms, t.end_ms) for t in gdag_trace_export(self.h)]

    def chrome_trace(self, path, names=None):
        """Write the timed nodes of a traced context (options.trace = 1) as a
        Chrome trace (JSON for chrome://tracing or Perfetto): one track per
        pool stream, one complete event per node, microseconds from context
        creation.  ``names``: optional {node id: label} (e.g. kernel names);
        other nodes are labelled by kind.  Returns the number of events."""
        import json
        kinds = {GDAG_NODE_KERNEL: "kernel", GDAG_NODE_HOST_WRITE: "h2d", GDAG_NODE_HOST_READ: "read",
                 GDAG_NODE_EXTERNAL: "external", GDAG_NODE_HOST_PREFETCH: "d2h", GDAG_NODE_GRAPH: "graph"}
        names = names or {}
        ev = []
        for node, kind, stream, t0, t1 in self.trace():
            cat = kinds.get(kind, "node")
            ev.append({"name": names.get(node, "%s %d" % (cat, node)), "cat": cat, "ph": "X",
                       "ts": t0 * 1e3, "dur": max(0.0, t1 - t0) * 1e3, "pid": 0,
                       "tid": "stream %d" % stream if stream >= 0 else "host",
                       "args": {"node": node}})
        with open(path, "w") as f:
            json.dump({"traceEvents": ev, "displayTimeUnit": "ms"}, f)
        return len(ev)

    def trace_write(self, path):
        """The library's Chrome trace of a traced context (gdag_trace_write)."""
        gdag_trace_write(self.h, path)

    def stats(self):
        s = gdag_stats_get(self.h)
        return {f: getattr(s, f) for f, _ in gdag_stats._fields_}


class Param:
    """A scalar of a :class:`Program` (a kernel's scalar argument, or the
    offset or byte count of a write or prefetch) whose value is given at each
    issue."""

    __slots__ = ("name",)

    def __init__(self, name):
        self.name = name

    def __repr__(self):
        return "Param(%r)" % self.name


_ELEM_WORDS = ctypes.sizeof(gdag_elem) // 8   # gdag_elem as 64-bit words
_ELEM_OFF_WORD = gdag_elem.off.offset // 8
_ELEM_BYTES_WORD = gdag_elem.bytes.offset // 8
_ARG_WORDS = ctypes.sizeof(gdag_arg) // 8
_ARG_VALUE_WORD = gdag_arg.value.offset // 8


class Program:
    """A recorded sequence of non-blocking elements of a program -- kernel
    launches, fused launches, host writes from the array's host view, and
    prefetches to the host -- issued by ONE gdag_issue call.  This is
    argument marshalling only: the library infers, places and issues each
    element exactly as its single call would.  Scalars may be :class:`Param`
    objects whose values are bound at each :meth:`issue`, so one recording
    serves every size of a request shape; the arrays are fixed at recording.
    """

    def __init__(self, ctx):
        self.ctx = ctx
        self._elems = []           # gdag_elem field tuples
        self._args = bytearray()   # packed gdag_arg entries
        self._nargs = 0
        self._arg_params = []      # (name, arg index, scalar size)
        self._elem_params = []     # (name, element index, word of the element)
        self._ready = None

    def __len__(self):
        return len(self._elems)

    def _pack_args(self, name, args):
        kid, spec = self.ctx.kernel(name)
        if len(args) != len(spec):
            raise GdagError(GDAG_ERR_INVALID, "%s takes %d arguments, got %d" % (name, len(spec), len(args)))
        first = self._nargs
        for i, (sp, v) in enumerate(zip(spec, args)):
            if sp.kind == GDAG_ARG_ARRAY:
                if v.__class__ is Mode:
                    self._args += _ARG.pack(GDAG_ARG_ARRAY, v.mode, v.array.handle, 0, 0)
                else:
                    self._args += _ARG.pack(GDAG_ARG_ARRAY, GDAG_MODE_SIGNATURE, v.handle, 0, 0)
            elif v.__class__ is Param:
                self._arg_params.append((v.name, first + i, sp.size))
                self._args += _ARG.pack(GDAG_ARG_SCALAR, 0, 0, sp.size, 0)
            else:
                self._args += _ARG.pack(GDAG_ARG_SCALAR, 0, 0, sp.size, _scalar_bits(v, sp.size))
        self._nargs += len(args)
        return kid, first

    def _sized(self, value, word):
        if value.__class__ is Param:
            self._elem_params.append((value.name, len(self._elems), word))
            return 0
        return int(value)

    def launch(self, name, *args, grid=None, block=None, smem=0):
        self._ready = None
        kid, first = self._pack_args(name, args)
        g = tuple(grid) if grid else (0, 0, 0)
        b = tuple(block) if block else (0, 0, 0)
        self._elems.append((GDAG_ELEM_LAUNCH, kid, 0, len(args), 1, smem, first, 0, 0, g, b))
        return len(self._elems) - 1

    def launch_fused(self, name, members):
        """One fused element (gdag_launch_fused) of the member argument lists."""
        self._ready = None
        if not members:
            raise GdagError(GDAG_ERR_INVALID, "fused launch of no members")
        first = None
        for m in members:
            kid, f = self._pack_args(name, m)
            first = f if first is None else first
        self._elems.append((GDAG_ELEM_LAUNCH_FUSED, kid, 0, len(members[0]), len(members), 0, first, 0, 0,
                            (0, 0, 0), (0, 0, 0)))
        return len(self._elems) - 1

    def _copy(self, kind, a, off, nbytes):
        self._ready = None
        nbytes = a.nbytes - off if nbytes is None else nbytes
        o = self._sized(off, _ELEM_OFF_WORD)
        nb = self._sized(nbytes, _ELEM_BYTES_WORD)
        self._elems.append((kind, 0, a.handle, 0, 0, 0, 0, o, nb, (0, 0, 0), (0, 0, 0)))
        return len(self._elems) - 1

    def write(self, a, off=0, nbytes=None):
        """Host write of [off, off + nbytes) from the array's host view."""
        return self._copy(GDAG_ELEM_WRITE, a, off, nbytes)

    def prefetch_host(self, a, off=0, nbytes=None):
        return self._copy(GDAG_ELEM_PREFETCH_HOST, a, off, nbytes)

    def _prepare(self):
        import numpy as np
        n = len(self._elems)
        elems = (gdag_elem * max(1, n))()
        for i, (t, k, a, na, cnt, sm, a0, off, nb, g, b) in enumerate(self._elems):
            e = elems[i]
            e.type, e.kernel, e.array, e.nargs, e.count, e.smem, e.arg0 = t, k, a, na, cnt, sm, a0
            e.off, e.bytes = off, nb
            e.grid = gdag_dim3(*g)
            e.block = gdag_dim3(*b)
        args = (gdag_arg * max(1, self._nargs)).from_buffer_copy(bytes(self._args) or bytes(_ARG.size))
        ew = np.frombuffer(elems, dtype=np.uint64)
        aw = np.frombuffer(args, dtype=np.uint64)
        groups = {}
        for name, idx, size in self._arg_params:
            groups.setdefault(name, {}).setdefault(("a", size), []).append(idx * _ARG_WORDS + _ARG_VALUE_WORD)
        for name, idx, word in self._elem_params:
            groups.setdefault(name, {}).setdefault(("e", 8), []).append(idx * _ELEM_WORDS + word)
        plan = {name: [(ew if w == "e" else aw, size, np.asarray(ix, dtype=np.intp))
                       for (w, size), ix in g.items()] for name, g in groups.items()}
        nodes = (_i64 * max(1, n))()
        self._ready = (elems, args, plan, nodes, _i32(), n, self._nargs)

    def params(self):
        return sorted({p[0] for p in self._arg_params} | {p[0] for p in self._elem_params})

    def issue(self, **values):
        """Bind every Param and issue all elements in one call; returns the
        node id of each element (-1 where it made none).  A failure raises
        GdagError with ``issued`` (elements issued before the failing one)
        and ``nodes``."""
        if self._ready is None:
            self._prepare()
        elems, args, plan, nodes, issued, n, nargs = self._ready
        if len(values) != len(plan) or any(k not in values for k in plan):
            raise GdagError(GDAG_ERR_INVALID, "program parameters %s, given %s"
                            % (sorted(plan), sorted(values)))
        for name, targets in plan.items():
            v = values[name]
            for words, size, ix in targets:
                words[ix] = _scalar_bits(v, size)
        r = lib().gdag_issue(self.ctx.h, ctypes.addressof(elems), n, ctypes.addressof(args), nargs,
                             ctypes.addressof(nodes), ctypes.byref(issued))
        out = nodes[:n]
        if r < 0:
            e = GdagError(r, self.ctx.last_error)
            e.issued, e.nodes = issued.value, out
            raise e
        return out


def _host_ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "ctypes"):  # numpy
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffer must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):  # torch CPU tensor
        return x.data_ptr()
    raise TypeError("unsupported host buffer %r" % type(x))
