"""Thin Python binding of libgbx.so (the C ABI declared in include/gbx.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Functions keep the C names without the ``gbx_`` prefix.  Device
buffers are CUDA tensors (PyTorch provides device memory and streams; it does
no compute here).  Failing calls raise ``GbxError`` with the library's status
and message.  If libgbx.so has not been built the import of a function raises
instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

OK = 0
ERR_INVALID_VALUE = 1
ERR_INVALID_INDEX = 2
ERR_DIMENSION_MISMATCH = 3
ERR_OUT_OF_MEMORY = 4
ERR_NOT_SUPPORTED = 5
ERR_TIMEOUT = 6
ERR_CUDA = 7
ERR_OVERFLOW = 8
ERR_BUSY = 9
ERR_NULL_POINTER = 10

SYMMETRIZE = 0x1
DROP_SELF_LOOPS = 0x2
DEVICE_EDGES = 0x4
DENSE = 0
SPARSE = 1
DENSE_F32 = 2
DIR_AUTO = 0
DIR_PUSH = 1
DIR_PULL = 2
HEUR_RATIO = 0
HEUR_BEAMER = 1
LOR_LAND = 0
MIN_PLUS_F32 = 1
DEPTH_I32 = 0
DEPTH_I16 = 1
TUNE_BFS = 0
TUNE_BATCH = 1
TUNE_SSSP = 2

EXPORTED = [
    "gbx_last_error", "gbx_status_string", "gbx_version", "gbx_graph_build", "gbx_graph_free", "gbx_graph_info",
    "gbx_graph_csr", "gbx_graph_copy_csr", "gbx_graph_sync", "gbx_desc_init", "gbx_mxv", "gbx_mxv_stats",
    "gbx_bfs", "gbx_bfs_host", "gbx_bfs_trace", "gbx_set_wait_timeout_ns", "gbx_selftest_barrier_timeout",
    "gbx_mxv_pull_noalloc", "gbx_bfs_batch", "gbx_bfs_batch_trace",
    "gbx_server_config_init", "gbx_server_create", "gbx_server_add_graph", "gbx_server_graph_lanes",
    "gbx_server_submit", "gbx_server_poll", "gbx_server_stats", "gbx_server_destroy", "gbx_autotune",
    "gbx_graph_set_weights", "gbx_graph_copy_weights", "gbx_sssp", "gbx_sssp_trace", "gbx_server_set_graph_desc",
    "gbx_tune_thresholds",
]


class GbxError(RuntimeError):
    def __init__(self, status: int, fn: str, message: str):
        super().__init__(f"{fn}: status {status} ({message})")
        self.status = status


class Vector(ctypes.Structure):
    _fields_ = [("format", ctypes.c_int32), ("size", ctypes.c_int32), ("data", ctypes.c_void_p),
                ("nnz", ctypes.c_void_p), ("capacity", ctypes.c_int32)]


class Desc(ctypes.Structure):
    _fields_ = [("transpose", ctypes.c_int32), ("mask_complement", ctypes.c_int32), ("early_exit", ctypes.c_int32),
                ("accum", ctypes.c_int32), ("direction", ctypes.c_int32), ("heuristic", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float), ("masking", ctypes.c_int32),
                ("operand_reuse", ctypes.c_int32), ("trace", ctypes.c_int32), ("pull_probe", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("push_sort", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class Level(ctypes.Structure):
    _fields_ = [("direction", ctypes.c_int32), ("level", ctypes.c_int32), ("nf", ctypes.c_int64),
                ("mf", ctypes.c_int64), ("nu", ctypes.c_int64), ("nu_nz", ctypes.c_int64), ("mu", ctypes.c_int64),
                ("e_exam", ctypes.c_int64), ("n_new", ctypes.c_int64), ("mf_new", ctypes.c_int64),
                ("time_ns", ctypes.c_int64)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("slots", ctypes.c_int32), ("depth_type", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("max_pending", ctypes.c_int64), ("memory_budget", ctypes.c_int64),
                ("reserved", ctypes.c_int32 * 4)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("graph_id", ctypes.c_int32), ("source", ctypes.c_int32),
                ("status", ctypes.c_int32), ("levels", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("t_submit", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double)]


LEVEL_FIELDS = ["direction", "level", "nf", "mf", "nu", "nu_nz", "mu", "e_exam", "n_new", "mf_new", "time_ns"]


def lib_path() -> str:
    return _build.LIB_PATH


def load():
    """Load libgbx.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                                   "or python -m paper_1804_03327_gb300.build")
            L = ctypes.CDLL(path)
            p, i32, i64, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
            sigs = {
                "gbx_last_error": (ctypes.c_char_p, []),
                "gbx_status_string": (ctypes.c_char_p, [ctypes.c_int]),
                "gbx_version": (i32, []),
                "gbx_graph_build": (ctypes.c_int, [ctypes.POINTER(p), i32, i64, p, p, u32, p]),
                "gbx_graph_free": (ctypes.c_int, [p]),
                "gbx_graph_info": (ctypes.c_int, [p, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)]),
                "gbx_graph_csr": (ctypes.c_int, [p, i32, ctypes.POINTER(p), ctypes.POINTER(p)]),
                "gbx_graph_copy_csr": (ctypes.c_int, [p, i32, p, p]),
                "gbx_graph_sync": (ctypes.c_int, [p, p]),
                "gbx_desc_init": (None, [ctypes.POINTER(Desc)]),
                "gbx_mxv": (ctypes.c_int, [ctypes.POINTER(Vector), ctypes.POINTER(Vector), i32, p,
                                           ctypes.POINTER(Vector), ctypes.POINTER(Desc), p]),
                "gbx_mxv_stats": (ctypes.c_int, [p] + [ctypes.POINTER(i64)] * 4),
                "gbx_bfs": (ctypes.c_int, [p, i32, p, p, ctypes.POINTER(Desc), p]),
                "gbx_bfs_host": (ctypes.c_int, [p, p, i32, p, p, ctypes.POINTER(Desc), p]),
                "gbx_bfs_trace": (ctypes.c_int, [p, ctypes.POINTER(Level), i32, ctypes.POINTER(i32)]),
                "gbx_set_wait_timeout_ns": (ctypes.c_int, [u64]),
                "gbx_selftest_barrier_timeout": (ctypes.c_int, [p, u64, p]),
                "gbx_mxv_pull_noalloc": (ctypes.c_int, [i32, p, p, p, p, i32, i32, p, p]),
                "gbx_bfs_batch": (ctypes.c_int, [p, p, i32, p, i32, ctypes.POINTER(Desc), p]),
                "gbx_bfs_batch_trace": (ctypes.c_int, [p, ctypes.POINTER(Level), i32, ctypes.POINTER(i32)]),
                "gbx_server_config_init": (None, [ctypes.POINTER(ServerConfig)]),
                "gbx_server_create": (ctypes.c_int, [ctypes.POINTER(p), ctypes.POINTER(ServerConfig)]),
                "gbx_server_add_graph": (ctypes.c_int, [p, p, ctypes.POINTER(i32)]),
                "gbx_server_graph_lanes": (ctypes.c_int, [p, i32, ctypes.POINTER(i32)]),
                "gbx_server_set_graph_desc": (ctypes.c_int, [p, i32, ctypes.POINTER(Desc)]),
                "gbx_server_submit": (ctypes.c_int, [p, i32, i32, p, u64]),
                "gbx_server_poll": (ctypes.c_int, [p, ctypes.POINTER(Completion), i32, ctypes.POINTER(i32)]),
                "gbx_server_stats": (ctypes.c_int, [p, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                                    ctypes.POINTER(i64), ctypes.POINTER(i64)]),
                "gbx_server_destroy": (ctypes.c_int, [p]),
                "gbx_autotune": (ctypes.c_int, [p, i32, p, i32, ctypes.POINTER(Desc), ctypes.POINTER(ctypes.c_double),
                                                ctypes.c_char_p, p]),
                "gbx_graph_set_weights": (ctypes.c_int, [p, i64, p, p, p, u32, p]),
                "gbx_graph_copy_weights": (ctypes.c_int, [p, i32, p]),
                "gbx_sssp": (ctypes.c_int, [p, i32, p, ctypes.POINTER(Desc), p]),
                "gbx_sssp_trace": (ctypes.c_int, [p, ctypes.POINTER(Level), i32, ctypes.POINTER(i32)]),
                "gbx_tune_thresholds": (ctypes.c_int, [ctypes.POINTER(Level), ctypes.POINTER(Level), i32, i32,
                                                       ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                                       ctypes.POINTER(i32)]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, fn: str):
    if status != OK:
        msg = load().gbx_last_error().decode(errors="replace")
        raise GbxError(status, fn, msg)


def _stream_ptr(stream):
    """cudaStream_t of a torch stream (None: the current torch stream)."""
    if isinstance(stream, int):
        return stream
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def status_string(status: int) -> str:
    return load().gbx_status_string(status).decode()


def version() -> int:
    return int(load().gbx_version())


def desc_init(**fields) -> Desc:
    d = Desc()
    load().gbx_desc_init(ctypes.byref(d))
    for k, v in fields.items():
        if not hasattr(d, k):
            raise AttributeError(k)
        setattr(d, k, v)
    return d


def selftest_barrier_timeout(g: "Graph", timeout_ns: int, stream=None):
    _check(load().gbx_selftest_barrier_timeout(g.handle, int(timeout_ns), _stream_ptr(stream)),
           "gbx_selftest_barrier_timeout")


def set_wait_timeout_ns(ns: int):
    _check(load().gbx_set_wait_timeout_ns(int(ns)), "gbx_set_wait_timeout_ns")


class Graph:
    """Owning handle of a gbx_graph."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            _check(load().gbx_graph_free(self._h), "gbx_graph_free")
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self):
        n, nnz, sym = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
        _check(load().gbx_graph_info(self._h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(sym)),
               "gbx_graph_info")
        return n.value, nnz.value, bool(sym.value)


def graph_build(n: int, src, dst, symmetrize: bool = True, drop_self_loops: bool = True, stream=None) -> Graph:
    """Build from host numpy int32 arrays or CUDA int32 tensors (src[e] -> dst[e])."""
    flags = (SYMMETRIZE if symmetrize else 0) | (DROP_SELF_LOOPS if drop_self_loops else 0)
    if isinstance(src, np.ndarray):
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        sp, dp = src.ctypes.data, dst.ctypes.data
        m = len(src)
        sptr = None
    else:
        if src.dtype != dst.dtype or str(src.dtype) != "torch.int32" or not src.is_cuda:
            raise TypeError("device edges must be CUDA int32 tensors")
        src, dst = src.contiguous(), dst.contiguous()
        sp, dp = src.data_ptr(), dst.data_ptr()
        m = src.numel()
        flags |= DEVICE_EDGES
        sptr = _stream_ptr(stream)
    h = ctypes.c_void_p()
    st = load().gbx_graph_build(ctypes.byref(h), int(n), int(m), sp, dp, flags,
                                sptr if sptr is not None else (_stream_ptr(stream) if _torch_cuda() else None))
    _check(st, "gbx_graph_build")
    return Graph(h.value)


def _torch_cuda() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def graph_copy_csr(g: Graph, transpose: bool = False):
    """(row_ptr, col) of A (or A^T) as host numpy int32 arrays."""
    n, nnz, _ = g.info()
    row_ptr = np.empty(n + 1, dtype=np.int32)
    col = np.empty(max(nnz, 1), dtype=np.int32)
    _check(load().gbx_graph_copy_csr(g.handle, int(transpose), row_ptr.ctypes.data, col.ctypes.data),
           "gbx_graph_copy_csr")
    return row_ptr, col[:nnz]


def graph_sync(g: Graph, stream=None):
    _check(load().gbx_graph_sync(g.handle, _stream_ptr(stream)), "gbx_graph_sync")


def dense(t) -> Vector:
    """View of a CUDA uint8 tensor as a GBX_DENSE vector."""
    assert t.is_cuda and str(t.dtype) == "torch.uint8" and t.is_contiguous()
    return Vector(DENSE, t.numel(), t.data_ptr(), None, 0)


def dense_f32(t) -> Vector:
    """View of a CUDA float32 tensor as a GBX_DENSE_F32 vector (+inf = no entry)."""
    assert t.is_cuda and str(t.dtype) == "torch.float32" and t.is_contiguous()
    return Vector(DENSE_F32, t.numel(), t.data_ptr(), None, 0)


def graph_set_weights(g: "Graph", src, dst, w, stream=None):
    """Attach float32 weights: host numpy arrays or CUDA tensors, the edge list g was built from."""
    if isinstance(src, np.ndarray):
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.float32)
        ptrs, flags, m = (src.ctypes.data, dst.ctypes.data, w.ctypes.data), 0, len(src)
    else:
        src, dst, w = src.contiguous(), dst.contiguous(), w.contiguous()
        ptrs, flags, m = (src.data_ptr(), dst.data_ptr(), w.data_ptr()), DEVICE_EDGES, src.numel()
    _check(load().gbx_graph_set_weights(g.handle, int(m), *ptrs, flags, _stream_ptr(stream) if _torch_cuda() else None),
           "gbx_graph_set_weights")


def graph_weights(g: "Graph", transpose: bool = False) -> np.ndarray:
    _, nnz, _ = g.info()
    out = np.empty(max(1, nnz), dtype=np.float32)
    _check(load().gbx_graph_copy_weights(g.handle, int(transpose), out.ctypes.data), "gbx_graph_copy_weights")
    return out[:nnz]


def sssp(g: "Graph", source: int, dist, desc: Desc | None = None, stream=None):
    """Shortest-path distances from `source` into a CUDA float32 tensor dist[n]."""
    assert dist.is_cuda and str(dist.dtype) == "torch.float32"
    _check(load().gbx_sssp(g.handle, int(source), dist.data_ptr(), ctypes.byref(desc) if desc is not None else None,
                           _stream_ptr(stream)), "gbx_sssp")


def sssp_trace(g: "Graph", cap: int = 1 << 16) -> np.ndarray:
    return _levels(g, cap, "gbx_sssp_trace")


def sparse(indices, nnz, size: int) -> Vector:
    """View of CUDA int32 tensors (indices[capacity], nnz[1]) as a GBX_SPARSE vector."""
    assert indices.is_cuda and str(indices.dtype) == "torch.int32" and indices.is_contiguous()
    assert nnz.is_cuda and str(nnz.dtype) == "torch.int32"
    return Vector(SPARSE, int(size), indices.data_ptr(), nnz.data_ptr(), indices.numel())


def mxv(w: Vector, mask, semiring: int, A: Graph, u: Vector, desc: Desc | None = None, stream=None):
    st = load().gbx_mxv(ctypes.byref(w), ctypes.byref(mask) if mask is not None else None, int(semiring), A.handle,
                        ctypes.byref(u), ctypes.byref(desc) if desc is not None else None, _stream_ptr(stream))
    _check(st, "gbx_mxv")


def mxv_stats(A: Graph):
    vals = [ctypes.c_int64() for _ in range(4)]
    _check(load().gbx_mxv_stats(A.handle, *[ctypes.byref(v) for v in vals]), "gbx_mxv_stats")
    return dict(zip(["rows", "examined", "u_nnz", "edges"], [v.value for v in vals]))


def graph_csr(g: Graph, transpose: bool = False):
    """Device pointers (row_ptr, col) of A (or A^T), owned by the graph."""
    rp, col = ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().gbx_graph_csr(g.handle, int(transpose), ctypes.byref(rp), ctypes.byref(col)), "gbx_graph_csr")
    return rp.value, col.value


def mxv_pull_noalloc(n: int, row_ptr: int, col: int, u, mask, w, mask_complement: bool = False,
                     early_exit: bool = True, stream=None):
    """Allocation-free pull matvec on caller-owned CSR (device addresses) and
    CUDA uint8 tensors u, mask (or None) and w."""
    _check(load().gbx_mxv_pull_noalloc(int(n), row_ptr, col, u.data_ptr(),
                                       mask.data_ptr() if mask is not None else None, int(mask_complement),
                                       int(early_exit), w.data_ptr(), _stream_ptr(stream)), "gbx_mxv_pull_noalloc")


def bfs(g: Graph, source: int, depth, parent=None, desc: Desc | None = None, stream=None):
    """BFS into CUDA int32 tensors depth[n] and (optionally) parent[n]."""
    st = load().gbx_bfs(g.handle, int(source), depth.data_ptr(), parent.data_ptr() if parent is not None else None,
                        ctypes.byref(desc) if desc is not None else None, _stream_ptr(stream))
    _check(st, "gbx_bfs")


def bfs_host(g: Graph, sources, depth_host: np.ndarray, parent_host: np.ndarray | None = None,
             desc: Desc | None = None, stream=None):
    """BFS for every source into host arrays depth_host[count, n] (and parent_host)."""
    srcs = np.ascontiguousarray(sources, dtype=np.int32)
    dptr = depth_host.data_ptr() if hasattr(depth_host, "data_ptr") else depth_host.ctypes.data
    pptr = None
    if parent_host is not None:
        pptr = parent_host.data_ptr() if hasattr(parent_host, "data_ptr") else parent_host.ctypes.data
    st = load().gbx_bfs_host(g.handle, srcs.ctypes.data, len(srcs), dptr, pptr,
                             ctypes.byref(desc) if desc is not None else None, _stream_ptr(stream))
    _check(st, "gbx_bfs_host")


def autotune(g: Graph, kind: int, sources, cache_path: str | None = None, stream=None):
    """Fastest descriptor for g on these sources: (Desc, ms)."""
    srcs = np.ascontiguousarray(sources, dtype=np.int32)
    d = Desc()
    ms = ctypes.c_double()
    _check(load().gbx_autotune(g.handle, int(kind), srcs.ctypes.data, len(srcs), ctypes.byref(d), ctypes.byref(ms),
                               cache_path.encode() if cache_path else None, _stream_ptr(stream)), "gbx_autotune")
    return d, ms.value


def tune_thresholds(push_trace: np.ndarray, pull_trace: np.ndarray, n: int):
    """Ratio-rule (alpha, beta) reproducing the per-level best schedule of one BFS
    traced both ways (gbx_tune_thresholds), and that schedule."""
    k = len(push_trace)
    bufs = []
    for tr in (push_trace, pull_trace):
        b = (Level * max(k, 1))()
        for i in range(min(k, len(tr))):
            for f in LEVEL_FIELDS:
                setattr(b[i], f, int(tr[i][f]))
        bufs.append(b)
    a, bt = ctypes.c_float(), ctypes.c_float()
    sched = (ctypes.c_int32 * max(k, 1))()
    _check(load().gbx_tune_thresholds(bufs[0], bufs[1], k if len(pull_trace) == k else -1, int(n), ctypes.byref(a),
                                      ctypes.byref(bt), sched), "gbx_tune_thresholds")
    return a.value, bt.value, [int(x) for x in sched[:k]]


def desc_dict(d: Desc) -> dict:
    return {f: (list(getattr(d, f)) if f == "reserved" else getattr(d, f)) for f, _ in d._fields_ if f != "reserved"}


def bfs_batch(g: Graph, sources, depth, desc: Desc | None = None, stream=None):
    """Multi-source BFS into a CUDA tensor depth[S, n] (int32 or int16)."""
    srcs = np.ascontiguousarray(sources, dtype=np.int32)
    dt = DEPTH_I16 if str(depth.dtype) == "torch.int16" else DEPTH_I32
    _check(load().gbx_bfs_batch(g.handle, srcs.ctypes.data, len(srcs), depth.data_ptr(), dt,
                                ctypes.byref(desc) if desc is not None else None, _stream_ptr(stream)),
           "gbx_bfs_batch")


def bfs_batch_trace(g: Graph, cap: int = 1 << 16) -> np.ndarray:
    return _levels(g, cap, "gbx_bfs_batch_trace")


def bfs_trace(g: Graph, cap: int = 1 << 16) -> np.ndarray:
    """Per-level records of the last traced BFS as a numpy structured array."""
    return _levels(g, cap, "gbx_bfs_trace")


def _levels(g: Graph, cap: int, fn: str) -> np.ndarray:
    buf = (Level * cap)()
    nl = ctypes.c_int32()
    _check(getattr(load(), fn)(g.handle, buf, cap, ctypes.byref(nl)), fn)
    k = min(nl.value, cap)
    dt = np.dtype([(f, np.int64) for f in LEVEL_FIELDS])
    out = np.zeros(k, dtype=dt)
    for i in range(k):
        for f in LEVEL_FIELDS:
            out[i][f] = getattr(buf[i], f)
    return out


class Server:
    """Continuous-batching BFS server (gbx_server_*)."""

    def __init__(self, **cfg):
        c = ServerConfig()
        load().gbx_server_config_init(ctypes.byref(c))
        for k, v in cfg.items():
            setattr(c, k, v)
        h = ctypes.c_void_p()
        _check(load().gbx_server_create(ctypes.byref(h), ctypes.byref(c)), "gbx_server_create")
        self._h = h.value
        self._buf = (Completion * 4096)()

    def add_graph(self, g: Graph) -> int:
        gid = ctypes.c_int32()
        _check(load().gbx_server_add_graph(self._h, g.handle, ctypes.byref(gid)), "gbx_server_add_graph")
        return gid.value

    def lanes(self, gid: int) -> int:
        x = ctypes.c_int32()
        _check(load().gbx_server_graph_lanes(self._h, gid, ctypes.byref(x)), "gbx_server_graph_lanes")
        return x.value

    def set_graph_desc(self, gid: int, desc: Desc):
        """Descriptor of this graph's batches (e.g. from autotune(..., TUNE_BATCH, ...))."""
        _check(load().gbx_server_set_graph_desc(self._h, gid, ctypes.byref(desc)), "gbx_server_set_graph_desc")

    def submit(self, gid: int, source: int, out, tag: int) -> bool:
        """Queue a query; False if the server refused it (queue full).  The server's
        streams do not wait on torch's: work queued on `out` must have finished."""
        st = load().gbx_server_submit(self._h, int(gid), int(source), out.data_ptr(), int(tag))
        if st == ERR_BUSY:
            return False
        _check(st, "gbx_server_submit")
        return True

    def poll(self) -> list:
        n = ctypes.c_int32()
        _check(load().gbx_server_poll(self._h, self._buf, len(self._buf), ctypes.byref(n)), "gbx_server_poll")
        return [self._buf[i] for i in range(n.value)]

    def stats(self) -> dict:
        q, f, r, b = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().gbx_server_stats(self._h, ctypes.byref(q), ctypes.byref(f), ctypes.byref(r), ctypes.byref(b)),
               "gbx_server_stats")
        return {"queued": q.value, "in_flight": f.value, "rejected": r.value, "scratch_bytes": b.value}

    def destroy(self):
        if self._h:
            _check(load().gbx_server_destroy(self._h), "gbx_server_destroy")
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
