"""Weighted betweenness centrality on one GB300: thin Python binding.

Every function below marshals arguments to the C ABI of libbcgpu
(include/bcgpu.h) and nothing else: all work runs in the library's CUDA
kernels.  The library is built in-tree by ``paper_1701_05975_gb300.build``;
when it is missing or fails to load, every call raises (there is no CPU
fallback).

Method: arxiv 1701.05975 (Brandes' algorithm per source with a parallel,
strict-criterion Dijkstra; Sec. 2-3).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbcgpu.so")

BC_OK = 0
BC_ERR_INVALID = 1
BC_ERR_NOMEM = 2
BC_ERR_CUDA = 3
BC_ERR_TIMEOUT = 4
BC_ERR_BUSY = 5
BC_ERR_CANCELLED = 6
BC_UNDIRECTED_CHECK = 1
BC_RELABEL_DEGREE = 2
BC_KEEP_ORDER = 4
BC_DIRECTED = 8
BC_MODE_BATCHED = 0
BC_MODE_PLAIN = 1
BC_ALGO_AUTO, BC_ALGO_STRICT, BC_ALGO_DELTA = 0, 1, 2
BC_REQ_QUEUED, BC_REQ_RUNNING, BC_REQ_DONE, BC_REQ_FAILED, BC_REQ_CANCELLED = range(5)

_ERR_NAMES = {1: "BC_ERR_INVALID", 2: "BC_ERR_NOMEM", 3: "BC_ERR_CUDA", 4: "BC_ERR_TIMEOUT", 5: "BC_ERR_BUSY",
              6: "BC_ERR_CANCELLED"}


class BCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class bc_config(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("team_threads", ctypes.c_uint32), ("max_slots", ctypes.c_uint32),
                ("settle_in", ctypes.c_uint32), ("bucket_width", ctypes.c_uint64), ("phase_cap", ctypes.c_uint64),
                ("mem_fraction", ctypes.c_double), ("warp_degree", ctypes.c_uint32), ("team_degree", ctypes.c_uint32),
                ("algorithm", ctypes.c_uint32), ("hot_vertices", ctypes.c_uint32)]


class bc_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("nnz", ctypes.c_uint64), ("max_weight", ctypes.c_uint32),
                ("dist_bits", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64), ("slab_bytes", ctypes.c_uint64),
                ("relabeled", ctypes.c_uint32), ("directed", ctypes.c_uint32)]


class bc_run_stats(ctypes.Structure):
    _fields_ = [("sources", ctypes.c_uint64), ("phases", ctypes.c_uint64), ("refills", ctypes.c_uint64),
                ("reached", ctypes.c_uint64), ("relax_atomics", ctypes.c_uint64),
                ("entries_scanned", ctypes.c_uint64), ("team_threads", ctypes.c_uint32),
                ("slots", ctypes.c_uint32), ("bucket_width", ctypes.c_uint64), ("dag_edges", ctypes.c_uint64),
                ("pair_overflows", ctypes.c_uint64), ("cycles_expand", ctypes.c_uint64),
                ("cycles_refill", ctypes.c_uint64), ("cycles_settle", ctypes.c_uint64),
                ("cycles_backward", ctypes.c_uint64), ("near_scanned", ctypes.c_uint64),
                ("far_scanned", ctypes.c_uint64), ("levels", ctypes.c_uint64), ("algorithm", ctypes.c_uint32),
                ("warp_degree", ctypes.c_uint32), ("team_degree", ctypes.c_uint32),
                ("settle_in", ctypes.c_uint32)]


class bc_serving_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("edges_traversed", ctypes.c_uint64),
                ("max_concurrent", ctypes.c_uint32)]


_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_f64 = ctypes.c_double
_int = ctypes.c_int

_SIGNATURES = {
    "bc_get_config": [ctypes.POINTER(bc_config)],
    "bc_set_config": [ctypes.POINTER(bc_config)],
    "bc_graph_create": [_vp, _vp, _vp, _u32, _u64, _u32, ctypes.POINTER(_vp)],
    "bc_graph_destroy": [_vp],
    "bc_graph_get_info": [_vp, ctypes.POINTER(bc_graph_info)],
    "bc_compute": [_vp, _vp, _u32, _f64, _vp],
    "bc_compute_async": [_vp, _vp, _u32, _f64, _vp, _vp],
    "bc_sync_status": [_vp, _vp],
    "bc_edge_compute": [_vp, _vp, _u32, _f64, _vp, _vp],
    "bc_request_submit": [_vp, _vp, _u32, _f64, _vp, ctypes.POINTER(_u64)],
    "bc_request_poll": [_u64, ctypes.POINTER(_int)],
    "bc_request_wait": [_u64, _int],
    "bc_request_cancel": [_u64],
    "bc_serving_stats_get": [ctypes.POINTER(bc_serving_stats)],
    "bc_serving_reset": [],
    "bc_sssp_debug": [_vp, _u32, _vp, _vp, _vp],
    "bc_last_run_stats": [_vp, ctypes.POINTER(bc_run_stats)],
    "bc_autotune": [_vp, _vp, _u32],
    "bc_compute_noalloc": [_vp, _vp, _vp, _u32, _u64, _vp, _u32, _f64, _vp, _vp, _vp],
    "bc_compute_paper_variant": [_vp, _vp, _u32, _f64, _vp, _int, _int],
    "bc_edge_compute_async": [_vp, _vp, _u32, _f64, _vp, _vp, _vp],
    "bc_step_create": [_vp, _vp, _u32, _f64, _vp, ctypes.POINTER(_vp)],
    "bc_step_launch": [_vp, _vp],
    "bc_step_sync": [_vp, _vp],
    "bc_step_destroy": [_vp],
}

_lib = None


def lib(path: str | None = None):
    """Load libbcgpu.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libbcgpu.so not built ({p}); run paper_1701_05975_gb300.build.build()")
    L = ctypes.CDLL(p)
    for name, args in _SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.bc_last_error.argtypes = []
    L.bc_last_error.restype = ctypes.c_char_p
    if path is None:
        _lib = L
    return L


def _check(rc: int):
    if rc != BC_OK:
        raise BCError(rc, lib().bc_last_error().decode(errors="replace"))


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


# --------------------------------------------------------------- C-ABI names


def bc_get_config() -> bc_config:
    c = bc_config()
    _check(lib().bc_get_config(ctypes.byref(c)))
    return c


def bc_set_config(cfg: bc_config | None = None, **fields):
    c = cfg if cfg is not None else bc_get_config()
    for k, v in fields.items():
        setattr(c, k, v)
    _check(lib().bc_set_config(ctypes.byref(c)))


def bc_graph_create(row_ptr, col_idx, w, n: int, flags: int = 0):
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    col = np.ascontiguousarray(col_idx, dtype=np.uint32)
    ww = np.ascontiguousarray(w, dtype=np.uint32)
    nnz = int(rp[-1]) if len(rp) else 0
    h = ctypes.c_void_p()
    _check(lib().bc_graph_create(_ptr(rp), _ptr(col) if len(col) else None, _ptr(ww) if len(ww) else None, n,
                                 len(col), flags, ctypes.byref(h)))
    del nnz
    return h


def bc_graph_destroy(h):
    _check(lib().bc_graph_destroy(h))


def bc_graph_get_info(h) -> bc_graph_info:
    i = bc_graph_info()
    _check(lib().bc_graph_get_info(h, ctypes.byref(i)))
    return i


def bc_compute(h, sources, scale: float, out_bc: np.ndarray):
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    assert out_bc.dtype == np.float64 and out_bc.flags.c_contiguous
    _check(lib().bc_compute(h, _ptr(src) if len(src) else None, len(src), scale, _ptr(out_bc)))
    return out_bc


def bc_compute_async(h, d_sources_ptr: int, k: int, scale: float, d_out_ptr: int, stream_ptr: int):
    _check(lib().bc_compute_async(h, ctypes.c_void_p(d_sources_ptr), k, scale, ctypes.c_void_p(d_out_ptr),
                                  ctypes.c_void_p(stream_ptr)))


def bc_compute_paper_variant(h, sources, scale: float, out_bc: np.ndarray, node_parallel: bool, vwarp: int):
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    _check(lib().bc_compute_paper_variant(h, _ptr(src) if len(src) else None, len(src), scale, _ptr(out_bc),
                                          int(node_parallel), vwarp))
    return out_bc


def bc_sync_status(h, stream_ptr: int):
    _check(lib().bc_sync_status(h, ctypes.c_void_p(stream_ptr)))


def bc_edge_compute_async(h, d_sources_ptr: int, k: int, scale: float, d_ebc_ptr: int, d_bc_ptr: int,
                          stream_ptr: int):
    _check(lib().bc_edge_compute_async(h, ctypes.c_void_p(d_sources_ptr), k, scale, ctypes.c_void_p(d_ebc_ptr),
                                       ctypes.c_void_p(d_bc_ptr), ctypes.c_void_p(stream_ptr)))


def bc_step_create(h, d_sources_ptr: int, k: int, scale: float, d_out_ptr: int):
    out = ctypes.c_void_p()
    _check(lib().bc_step_create(h, ctypes.c_void_p(d_sources_ptr), k, scale, ctypes.c_void_p(d_out_ptr),
                                ctypes.byref(out)))
    return out


def bc_step_launch(step, stream_ptr: int):
    _check(lib().bc_step_launch(step, ctypes.c_void_p(stream_ptr)))


def bc_step_sync(step, stream_ptr: int):
    _check(lib().bc_step_sync(step, ctypes.c_void_p(stream_ptr)))


def bc_step_destroy(step):
    _check(lib().bc_step_destroy(step))


def bc_edge_compute(h, sources, scale: float, out_ebc: np.ndarray, out_bc: np.ndarray | None = None):
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    _check(lib().bc_edge_compute(h, _ptr(src) if len(src) else None, len(src), scale, _ptr(out_ebc),
                                 _ptr(out_bc) if out_bc is not None else None))
    return out_ebc


def bc_request_submit(h, sources, scale: float, out_bc: np.ndarray) -> int:
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    rid = ctypes.c_uint64()
    _check(lib().bc_request_submit(h, _ptr(src) if len(src) else None, len(src), scale, _ptr(out_bc),
                                   ctypes.byref(rid)))
    return rid.value


def bc_request_poll(rid: int) -> int:
    st = ctypes.c_int()
    _check(lib().bc_request_poll(rid, ctypes.byref(st)))
    return st.value


def bc_request_wait(rid: int, timeout_ms: int = -1):
    _check(lib().bc_request_wait(rid, timeout_ms))


def bc_request_cancel(rid: int):
    _check(lib().bc_request_cancel(rid))


def bc_serving_stats_get() -> bc_serving_stats:
    s = bc_serving_stats()
    _check(lib().bc_serving_stats_get(ctypes.byref(s)))
    return s


def bc_serving_reset():
    _check(lib().bc_serving_reset())


def bc_sssp_debug(h, s: int, n: int):
    d = np.empty(n, np.uint64)
    sg = np.empty(n, np.float64)
    lev = np.empty(n, np.uint32)
    _check(lib().bc_sssp_debug(h, s, _ptr(d), _ptr(sg), _ptr(lev)))
    return d, sg, lev


def bc_last_run_stats(h) -> bc_run_stats:
    s = bc_run_stats()
    _check(lib().bc_last_run_stats(h, ctypes.byref(s)))
    return s


def bc_autotune(h, sources):
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    _check(lib().bc_autotune(h, _ptr(src), len(src)))


def bc_compute_noalloc(d_row_ptr: int, d_col_idx: int, d_w: int, n: int, nnz: int, d_sources: int, k: int,
                       scale: float, d_out_bc: int, d_status: int, stream_ptr: int):
    """All pointers are device addresses owned by the caller (see bcgpu.h)."""
    _check(lib().bc_compute_noalloc(ctypes.c_void_p(d_row_ptr), ctypes.c_void_p(d_col_idx), ctypes.c_void_p(d_w), n,
                                    nnz, ctypes.c_void_p(d_sources), k, scale, ctypes.c_void_p(d_out_bc),
                                    ctypes.c_void_p(d_status), ctypes.c_void_p(stream_ptr)))


# ------------------------------------------------------------ convenience


def _dptr(x) -> int:
    return 0 if x is None else int(x.data_ptr() if hasattr(x, "data_ptr") else x)


def _numel(x) -> int:
    return 0 if x is None else int(x.numel() if hasattr(x, "numel") else len(x))


def _sptr(stream) -> int:
    if stream is None:
        return 0
    return int(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)


class Graph:
    """Owns a device-resident graph (bc_graph_create / bc_graph_destroy)."""

    def __init__(self, csr, flags: int = 0):
        self.n = int(csr.n)
        self.nnz = int(csr.row_ptr[-1])
        self.handle = bc_graph_create(csr.row_ptr, csr.col, csr.w, self.n, flags)

    def compute(self, sources, scale: float = 1.0) -> np.ndarray:
        out = np.empty(self.n, np.float64)
        return bc_compute(self.handle, sources, scale, out)

    def edge_compute(self, sources, scale: float = 1.0):
        ebc = np.empty(max(self.nnz, 1), np.float64)
        bc = np.empty(self.n, np.float64)
        bc_edge_compute(self.handle, sources, scale, ebc, bc)
        return ebc[: self.nnz], bc

    def compute_paper_variant(self, sources, scale: float = 1.0, node_parallel: bool = False, vwarp: int = 32):
        out = np.empty(self.n, np.float64)
        return bc_compute_paper_variant(self.handle, sources, scale, out, node_parallel, vwarp)

    def sssp_debug(self, s: int):
        return bc_sssp_debug(self.handle, s, self.n)

    def info(self) -> bc_graph_info:
        return bc_graph_get_info(self.handle)

    def stats(self) -> bc_run_stats:
        return bc_last_run_stats(self.handle)

    def autotune(self, sources):
        bc_autotune(self.handle, sources)

    # ---- device buffers (torch tensors or anything with data_ptr()) ---------
    # Argument marshalling only: every step runs in the library's kernels.

    def compute_async(self, d_sources, d_out, scale: float = 1.0, stream=None):
        """BC into the device array d_out[n] for the device uint32/int32 ids
        d_sources[k], enqueued on `stream` (a torch.cuda.Stream, a raw
        cudaStream_t integer, or None for the legacy default stream)."""
        bc_compute_async(self.handle, _dptr(d_sources), _numel(d_sources), scale, _dptr(d_out), _sptr(stream))

    def edge_compute_async(self, d_sources, d_out_ebc, d_out_bc, scale: float = 1.0, stream=None):
        bc_edge_compute_async(self.handle, _dptr(d_sources), _numel(d_sources), scale, _dptr(d_out_ebc),
                              _dptr(d_out_bc), _sptr(stream))

    def sync(self, stream=None):
        """Wait for `stream` and raise BCError for a device-side failure of the last async run on it."""
        bc_sync_status(self.handle, _sptr(stream))

    def step(self, d_sources, d_out, scale: float = 1.0) -> "Step":
        """One batched run over d_sources captured as a CUDA graph (see Step)."""
        return Step(self, d_sources, d_out, scale)

    def submit(self, sources, scale: float = 1.0) -> "Request":
        """Queue a request on the serving loop; the result is a host array."""
        return Request(self, sources, scale)

    def close(self):
        if self.handle is not None:
            bc_graph_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Step:
    """A batched run captured once as a CUDA graph (bc_step_create) over the
    device buffers given at creation; launch() replays it, sync() waits and
    raises on a device-side failure.  The buffers must outlive the step."""

    def __init__(self, graph: Graph, d_sources, d_out, scale: float = 1.0):
        self._keep = (graph, d_sources, d_out)
        self.handle = bc_step_create(graph.handle, _dptr(d_sources), _numel(d_sources), scale, _dptr(d_out))

    def launch(self, stream=None):
        bc_step_launch(self.handle, _sptr(stream))

    def sync(self, stream=None):
        bc_step_sync(self.handle, _sptr(stream))

    def close(self):
        if self.handle is not None:
            bc_step_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Request:
    """A request on the serving loop (bc_request_submit); result() waits and
    returns the host BC array."""

    def __init__(self, graph: Graph, sources, scale: float = 1.0):
        self.out = np.empty(graph.n, np.float64)
        self._graph = graph
        self._done = False
        self.id = bc_request_submit(graph.handle, sources, scale, self.out)

    def poll(self) -> int:
        return bc_request_poll(self.id)

    def cancel(self):
        bc_request_cancel(self.id)

    def result(self, timeout_ms: int = -1) -> np.ndarray:
        if not self._done:  # the library forgets a request once it has been waited for
            bc_request_wait(self.id, timeout_ms)
            self._done = True
        return self.out
