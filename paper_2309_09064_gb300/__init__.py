"""Python binding of libtc (exact triangle counting on one GB300).

A thin ctypes layer over the C ABI declared in ``include/tc.h``: every
function here has the name of the C entry point it calls and only marshals
arguments (numpy arrays for host buffers, torch CUDA tensors or raw integers
for device buffers and streams).  All counting runs in the CUDA kernels of
``csrc/``; there is no CPU fallback: importing this package without the
compiled library (and nvcc to build it) raises ImportError.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = [
    "TcError", "TC_OK", "TC_NOT_READY", "TC_HOST", "TC_DEVICE", "TC_COPY", "TC_BORROW", "TC_VALIDATE",
    "TC_ORDER_DEGREE", "TC_ORDER_ID", "tc_create", "tc_destroy", "tc_last_error", "tc_set_stream",
    "tc_arena_bytes", "tc_build_csr", "tc_graph_from_csr", "tc_graph_info", "tc_graph_copy_out",
    "tc_validate", "tc_graph_free", "tc_count", "tc_count_levels", "tc_count_with_levels", "tc_count_vertices",
    "tc_list_triangles", "tc_count_alg3", "tc_count_batch",
    "tc_submit", "tc_poll",
    "tc_get_tuning", "tc_set_tuning", "tc_count_noalloc", "tc_poll_ex", "tc_count_shard", "tc_selftest_barrier",
    "library_path",
    "EXPORTED",
]

TC_OK, TC_ERR_INVALID, TC_ERR_OOM, TC_ERR_CUDA, TC_ERR_TIMEOUT, TC_ERR_BUSY, TC_NOT_READY, TC_ERR_CAPACITY = range(8)
TC_HOST, TC_DEVICE = 0, 1
TC_COPY, TC_BORROW, TC_VALIDATE = 0, 1, 2
TC_ORDER_DEGREE, TC_ORDER_ID = 0, 1
_STATUS = {0: "TC_OK", 1: "TC_ERR_INVALID", 2: "TC_ERR_OOM", 3: "TC_ERR_CUDA", 4: "TC_ERR_TIMEOUT",
           5: "TC_ERR_BUSY", 6: "TC_NOT_READY", 7: "TC_ERR_CAPACITY"}

# every entry point tc.h declares
EXPORTED = ["tc_create", "tc_destroy", "tc_last_error", "tc_set_stream", "tc_get_tuning", "tc_set_tuning",
            "tc_selftest_barrier",
            "tc_arena_bytes", "tc_build_csr",
            "tc_graph_from_csr", "tc_graph_info", "tc_graph_copy_out", "tc_validate", "tc_graph_free",
            "tc_count", "tc_count_levels", "tc_count_with_levels", "tc_count_vertices", "tc_list_triangles",
            "tc_count_alg3", "tc_count_shard",
            "tc_count_batch", "tc_submit",
            "tc_poll", "tc_poll_ex",
            "tc_count_noalloc"]


class TcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class tc_options(ctypes.Structure):
    _fields_ = [("order", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("stream", ctypes.c_void_p),
                ("max_queue", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 7)]


class tc_tuning(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint32) for k in (
        "warp_cap", "block_cap", "task_work", "warps_per_block", "block_threads", "warp_task_work",
        "hub_task_work", "max_v", "hub_group", "hub_filter_log2", "hub_threads", "tiny_cap",
        "table_kind", "flat_cap", "block_bits_log2", "batch_small_slots")] + [("reserved", ctypes.c_uint32 * 2)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class tc_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "n", "m", "triangles", "t_same", "t_cross", "horizontal_edges", "levels", "components", "probes",
        "row2_slots", "alg_bytes", "isect_bytes")] + [(k, ctypes.c_float) for k in (
            "ms_total", "ms_levels", "ms_mark", "ms_isect")] + [
        ("class_rows", ctypes.c_uint64 * 4), ("class_probes", ctypes.c_uint64 * 4),
        ("class_bytes", ctypes.c_uint64 * 4), ("ms_class", ctypes.c_float * 4),
        ("class_inserts", ctypes.c_uint64 * 4),
        ("launches", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def to_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if isinstance(v, ctypes.Array) else v
        return out


def _load():
    try:
        path = _build.build()
    except FileNotFoundError as e:  # no nvcc here: a library built from these sources is still fine
        if not os.path.exists(_build.LIB) or os.path.getmtime(_build.LIB) < _build._deps():
            raise ImportError(f"libtc.so is missing or older than its sources, and nvcc is not available: {e}") from e
        path = _build.LIB
    except Exception as e:  # compile error: fail loudly, never load a stale library
        raise ImportError(f"libtc.so could not be built: {e}") from e
    lib = ctypes.CDLL(path)
    P, V, U32, U64, I = ctypes.POINTER, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sig = {
        "tc_create": ([P(V), I, P(tc_options)], I),
        "tc_destroy": ([V], I),
        "tc_last_error": ([V], ctypes.c_char_p),
        "tc_set_stream": ([V, V], I),
        "tc_get_tuning": ([V, P(tc_tuning)], I),
        "tc_set_tuning": ([V, P(tc_tuning)], I),
        "tc_arena_bytes": ([V, P(U64)], I),
        "tc_selftest_barrier": ([V, U32], I),
        "tc_build_csr": ([V, U32, U64, V, V, I, P(V)], I),
        "tc_graph_from_csr": ([V, U32, V, V, I, I, P(V)], I),
        "tc_graph_info": ([V, P(U32), P(U64), P(V), P(V)], I),
        "tc_graph_copy_out": ([V, V, V, V, I], I),
        "tc_validate": ([V, V, P(I)], I),
        "tc_graph_free": ([V], I),
        "tc_count": ([V, V, P(U64), P(tc_stats)], I),
        "tc_count_levels": ([V, V, V, P(U64), P(tc_stats)], I),
        "tc_count_with_levels": ([V, V, V, P(U64), P(tc_stats)], I),
        "tc_count_vertices": ([V, V, V, P(U64), P(tc_stats)], I),
        "tc_list_triangles": ([V, V, V, U64, P(U64), P(tc_stats)], I),
        "tc_count_alg3": ([V, V, P(U64), P(tc_stats)], I),
        "tc_count_shard": ([V, V, U32, U32, P(U64), P(tc_stats)], I),
        "tc_count_batch": ([V, U32, P(V), P(U64)], I),
        "tc_submit": ([V, V, P(U64)], I),
        "tc_poll": ([V, U64, P(U64)], I),
        "tc_poll_ex": ([V, U64, P(U64), P(U64)], I),
        "tc_count_noalloc": ([V, V, U32, U64, U32, V, V], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def library_path() -> str:
    return _lib._name


def _check(ctx, st):
    if st != TC_OK:
        msg = _lib.tc_last_error(ctx).decode() if ctx else ""
        raise TcError(st, msg)


def _ptr(x):
    """(address, where) of a numpy array (host), a torch tensor (host/device) or an int (device)."""
    if x is None:
        return None, TC_HOST
    if isinstance(x, int):
        return x, TC_DEVICE
    if isinstance(x, np.ndarray):
        return x.ctypes.data, TC_HOST
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        return x.data_ptr(), (TC_DEVICE if x.is_cuda else TC_HOST)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


# ----------------------------------------------------------------------------- context

def tc_create(device: int = 0, order: int = TC_ORDER_DEGREE, stream=None, max_queue: int = 0):
    opt = tc_options()
    opt.order = order
    opt.stream = _stream_handle(stream)
    opt.max_queue = max_queue
    h = ctypes.c_void_p()
    _check(None, _lib.tc_create(ctypes.byref(h), device, ctypes.byref(opt)))
    return h


def tc_destroy(ctx):
    _check(None, _lib.tc_destroy(ctx))


def tc_last_error(ctx) -> str:
    return _lib.tc_last_error(ctx).decode()


def tc_set_stream(ctx, stream):
    _check(ctx, _lib.tc_set_stream(ctx, _stream_handle(stream)))


def tc_get_tuning(ctx) -> dict:
    t = tc_tuning()
    _check(ctx, _lib.tc_get_tuning(ctx, ctypes.byref(t)))
    return t.to_dict()


def tc_set_tuning(ctx, **kw):
    """Change some knobs of the context's tuning (keys of tc_tuning)."""
    t = tc_tuning()
    _check(ctx, _lib.tc_get_tuning(ctx, ctypes.byref(t)))
    for k, v in kw.items():
        if k not in t.to_dict():
            raise KeyError(k)
        setattr(t, k, int(v))
    _check(ctx, _lib.tc_set_tuning(ctx, ctypes.byref(t)))


def tc_selftest_barrier(ctx, timeout_ms: int = 200) -> int:
    """Run the bounded-wait self-test; returns its status (TC_ERR_TIMEOUT when the wait ended as designed)."""
    return _lib.tc_selftest_barrier(ctx, timeout_ms)


def tc_arena_bytes(ctx) -> int:
    b = ctypes.c_uint64()
    _check(ctx, _lib.tc_arena_bytes(ctx, ctypes.byref(b)))
    return b.value


# ----------------------------------------------------------------------------- graphs

def tc_build_csr(ctx, n: int, src, dst):
    """Tuples -> device CSR (symmetrised, loops dropped, de-duplicated, rows sorted)."""
    if isinstance(src, np.ndarray):
        src = np.ascontiguousarray(src, dtype=np.uint32)
        dst = np.ascontiguousarray(dst, dtype=np.uint32)
    ps, ws = _ptr(src)
    pd, wd = _ptr(dst)
    if ws != wd:
        raise ValueError("src and dst must live in the same place")
    t = len(src)
    g = ctypes.c_void_p()
    _check(ctx, _lib.tc_build_csr(ctx, n, t, ps, pd, ws, ctypes.byref(g)))
    return g


def tc_graph_from_csr(ctx, row_ptr, col, flags: int = TC_COPY, n: int | None = None):
    if isinstance(row_ptr, np.ndarray):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint64)
        col = np.ascontiguousarray(col, dtype=np.uint32)
    n = len(row_ptr) - 1 if n is None else n
    pr, wr = _ptr(row_ptr)
    pc, wc = _ptr(col)
    if wr != wc:
        raise ValueError("row_ptr and col must live in the same place")
    g = ctypes.c_void_p()
    _check(ctx, _lib.tc_graph_from_csr(ctx, n, pr, pc, wr, flags, ctypes.byref(g)))
    return g


def tc_graph_info(g):
    n, s = ctypes.c_uint32(), ctypes.c_uint64()
    rp, col = ctypes.c_void_p(), ctypes.c_void_p()
    _check(None, _lib.tc_graph_info(g, ctypes.byref(n), ctypes.byref(s), ctypes.byref(rp), ctypes.byref(col)))
    return n.value, s.value, rp.value, col.value


def tc_graph_copy_out(ctx, g):
    """Host copy of the graph's CSR: (row_ptr uint64[n+1], col uint32[slots])."""
    n, s, _, _ = tc_graph_info(g)
    rp = np.zeros(n + 1, dtype=np.uint64)
    col = np.zeros(max(s, 1), dtype=np.uint32)
    _check(ctx, _lib.tc_graph_copy_out(ctx, g, rp.ctypes.data, col.ctypes.data, TC_HOST))
    return rp, col[:s]


def tc_validate(ctx, g) -> bool:
    ok = ctypes.c_int()
    _check(ctx, _lib.tc_validate(ctx, g, ctypes.byref(ok)))
    return bool(ok.value)


def tc_graph_free(g):
    _check(None, _lib.tc_graph_free(g))


# ----------------------------------------------------------------------------- counting

def tc_count(ctx, g):
    """(T, stats dict)."""
    T = ctypes.c_uint64()
    st = tc_stats()
    _check(ctx, _lib.tc_count(ctx, g, ctypes.byref(T), ctypes.byref(st)))
    return T.value, st.to_dict()


def tc_count_levels(ctx, g, levels):
    """Count and write BFS levels into `levels` (a CUDA tensor of n 4-byte ints, or a device address)."""
    p, where = _ptr(levels)
    if where != TC_DEVICE:
        raise ValueError("levels must be a device buffer")
    T = ctypes.c_uint64()
    st = tc_stats()
    _check(ctx, _lib.tc_count_levels(ctx, g, p, ctypes.byref(T), ctypes.byref(st)))
    return T.value, st.to_dict()


def tc_count_with_levels(ctx, g, levels):
    """Count with caller-supplied levels (a CUDA tensor of n 4-byte ints, or a device address)."""
    p, where = _ptr(levels)
    if where != TC_DEVICE:
        raise ValueError("levels must be a device buffer")
    T = ctypes.c_uint64()
    st = tc_stats()
    _check(ctx, _lib.tc_count_with_levels(ctx, g, p, ctypes.byref(T), ctypes.byref(st)))
    return T.value, st.to_dict()


def tc_count_vertices(ctx, g, counts):
    """Triangles through every vertex into `counts` (a CUDA tensor of n 8-byte ints, or a device address)."""
    p, where = _ptr(counts)
    if where != TC_DEVICE:
        raise ValueError("counts must be a device buffer")
    T = ctypes.c_uint64()
    st = tc_stats()
    _check(ctx, _lib.tc_count_vertices(ctx, g, p, ctypes.byref(T), ctypes.byref(st)))
    return T.value, st.to_dict()


def tc_count_alg3(ctx, g):
    """Algorithm 3 (full neighbourhoods with the level rule) as a comparison kernel: (T, stats)."""
    T = ctypes.c_uint64()
    st = tc_stats()
    _check(ctx, _lib.tc_count_alg3(ctx, g, ctypes.byref(T), ctypes.byref(st)))
    return T.value, st.to_dict()


def tc_list_triangles(ctx, g, triples, capacity: int):
    """Every triangle once into `triples` (a CUDA tensor of 3 * capacity 4-byte ints, or a device address;
    None with capacity 0): returns (T, stats).  More than `capacity` triangles raise TcError with status
    TC_ERR_CAPACITY and the count in its `triangles` attribute."""
    p, where = _ptr(triples)
    if p is not None and where != TC_DEVICE:
        raise ValueError("triples must be a device buffer")
    if hasattr(triples, "numel") and triples.numel() * triples.element_size() < 12 * capacity:
        raise ValueError("triples holds fewer than 3 * capacity 4-byte ints")
    T = ctypes.c_uint64()
    st = tc_stats()
    status = _lib.tc_list_triangles(ctx, g, p, capacity, ctypes.byref(T), ctypes.byref(st))
    if status == TC_ERR_CAPACITY:
        e = TcError(status, _lib.tc_last_error(ctx).decode())
        e.triangles = T.value
        raise e
    _check(ctx, status)
    return T.value, st.to_dict()


def tc_count_shard(ctx, g, shard: int, nshards: int):
    """(partial T of shard `shard` of `nshards`, stats); the partials of all shards sum to T."""
    T = ctypes.c_uint64()
    st = tc_stats()
    _check(ctx, _lib.tc_count_shard(ctx, g, shard, nshards, ctypes.byref(T), ctypes.byref(st)))
    return T.value, st.to_dict()


def tc_count_batch(ctx, graphs):
    G = len(graphs)
    arr = (ctypes.c_void_p * max(G, 1))(*[g.value for g in graphs])
    out = np.zeros(max(G, 1), dtype=np.uint64)
    _check(ctx, _lib.tc_count_batch(ctx, G, arr, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
    return out[:G]


def tc_poll_ex(ctx, ticket: int):
    """(T, latency_ns) when done, None while not ready; raises on failure."""
    T, lat = ctypes.c_uint64(), ctypes.c_uint64()
    st = _lib.tc_poll_ex(ctx, ticket, ctypes.byref(T), ctypes.byref(lat))
    if st == TC_NOT_READY:
        return None
    _check(ctx, st)
    return T.value, lat.value


def tc_count_noalloc(row_ptr, col, n: int, slots: int, out, order: int = TC_ORDER_DEGREE, stream=None):
    """Count a small device CSR without any allocation by the library.

    For callers that cannot allocate device memory at the point of the count.
    row_ptr / col / out are device buffers (CUDA tensors or addresses); out
    receives [T, T inside G0, T cross-level, limit flag] as uint64 when the
    stream reaches the kernel.  Asynchronous; raises TcError on bad sizes.
    """
    pr, wr = _ptr(row_ptr)
    pc, wc = _ptr(col)
    po, wo = _ptr(out)
    if TC_HOST in (wr, wc, wo):
        raise ValueError("tc_count_noalloc takes device buffers only")
    _check(None, _lib.tc_count_noalloc(pr, pc, n, slots, order, po, _stream_handle(stream)))


def tc_submit(ctx, g) -> int:
    t = ctypes.c_uint64()
    _check(ctx, _lib.tc_submit(ctx, g, ctypes.byref(t)))
    return t.value


def tc_poll(ctx, ticket: int):
    """T when done, None while not ready; raises on failure."""
    T = ctypes.c_uint64()
    st = _lib.tc_poll(ctx, ticket, ctypes.byref(T))
    if st == TC_NOT_READY:
        return None
    _check(ctx, st)
    return T.value
