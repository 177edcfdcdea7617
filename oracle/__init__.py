"""CPU oracle for weighted betweenness centrality (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  The CUDA library never calls it, and it shares no
code with the CUDA library: the C source is ``oracle/brandes.c`` (Brandes with
a binary-heap Dijkstra, the paper's own CPU baseline, Sec. 4.1; and a
sequential replay of the paper's Algorithms 1-3).

Parity pins live in ``tests/test_oracle_*.py``: brute force (Floyd-Warshall
plus explicit path enumeration), closed forms, the ordered-pair invariant, an
independent library implementation (networkx) and the Eq. 3 vs Eq. 4 example
of Sec. 3.2.  Every function here is pinned by at least one of them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brandes.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False, extra_flags=(), out_path: str | None = None) -> str:
    """Compile brandes.c into a shared library with gcc (portable flags only:
    the same source builds on x86_64 and aarch64)."""
    out = out_path or _LIB_PATH
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and out_path is None and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC", *extra_flags, "-o", out, _SRC, "-lpthread"]
    subprocess.run(cmd, check=True)
    return out


_TIMING_LIB = None
TIMING_FLAGS: tuple = ()


def timing_lib():
    """A second build of the same brandes.c, with the optimisation flags of a
    CPU baseline (-O3 and the host's own instruction set: -mcpu=native on
    aarch64, -march=native elsewhere; -O3 alone if the compiler rejects
    that).  Only timed, never used for parity: the tests use the pinned
    portable -O2 build.  Returns the bound library; TIMING_FLAGS says what it
    was built with."""
    global _TIMING_LIB, TIMING_FLAGS
    if _TIMING_LIB is None:
        import platform

        native = "-mcpu=native" if platform.machine().lower() in ("aarch64", "arm64") else "-march=native"
        out = os.path.join(_BUILD, "liboracle_timing.so")
        for flags in (("-O3", native), ("-O3",)):
            try:
                build(force=True, extra_flags=flags, out_path=out)
            except subprocess.CalledProcessError:
                continue
            TIMING_FLAGS = flags
            _TIMING_LIB = load(out)
            break
        else:
            TIMING_FLAGS = ("-O2",)
            _TIMING_LIB = load()
    return _TIMING_LIB


def _bind(lib):
    lib.oracle_sssp.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p, ctypes.c_uint32, _u64p, _f64p, _u32p, _u32p]
    lib.oracle_delta.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p, ctypes.c_uint32, _f64p]
    lib.oracle_bc.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p, _u32p, ctypes.c_uint32, ctypes.c_double, _f64p, ctypes.c_int]
    lib.oracle_edge_bc.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p, _u32p, ctypes.c_uint32, ctypes.c_double, _f64p]
    lib.oracle_bc_pull.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p, _u32p, ctypes.c_uint32, ctypes.c_double, _f64p]
    lib.oracle_phased.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                  _u64p, _f64p, _u32p, _f64p, _u32p]
    for f in (lib.oracle_sssp, lib.oracle_delta, lib.oracle_bc, lib.oracle_edge_bc, lib.oracle_phased,
              lib.oracle_bc_pull):
        f.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building first if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


class OracleError(RuntimeError):
    pass


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint64)
    col = np.ascontiguousarray(g.col, dtype=np.uint32)
    w = np.ascontiguousarray(g.w, dtype=np.uint32)
    if len(col) == 0:  # keep non-NULL pointers for empty edge arrays
        col = np.zeros(1, np.uint32)
        w = np.ones(1, np.uint32)
    return rp, col, w


def _check(rc):
    if rc != 0:
        raise OracleError({1: "invalid input", 2: "out of memory"}.get(rc, f"error {rc}"))


def sssp(g, s: int, lib=None):
    """Exact distances (uint64, UINT64_MAX unreachable), shortest-path counts
    (float64) and settle order from source s."""
    lib = lib or load()
    rp, col, w = _csr(g)
    d = np.empty(g.n, np.uint64)
    sig = np.empty(g.n, np.float64)
    order = np.empty(g.n, np.uint32)
    reached = ctypes.c_uint32(0)
    _check(lib.oracle_sssp(g.n, _p(rp, _u64p), _p(col, _u32p), _p(w, _u32p), s, _p(d, _u64p), _p(sig, _f64p),
                           _p(order, _u32p), ctypes.byref(reached)))
    return d, sig, order[: reached.value].copy()


def delta(g, s: int, lib=None):
    """Per-source dependencies delta_s(v) (zero at s and at unreachable v)."""
    lib = lib or load()
    rp, col, w = _csr(g)
    out = np.empty(g.n, np.float64)
    _check(lib.oracle_delta(g.n, _p(rp, _u64p), _p(col, _u32p), _p(w, _u32p), s, _p(out, _f64p)))
    return out


def bc(g, sources, scale: float = 1.0, nthreads: int = 1, lib=None):
    """out[v] = scale * sum_{s in sources} delta_s(v)."""
    lib = lib or load()
    rp, col, w = _csr(g)
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    out = np.empty(g.n, np.float64)
    _check(lib.oracle_bc(g.n, _p(rp, _u64p), _p(col, _u32p), _p(w, _u32p), _p(src, _u32p) if len(src) else None,
                         len(src), scale, _p(out, _f64p), nthreads))
    return out


def bc_directed(g, sources, scale: float = 1.0, lib=None):
    """BC on a directed CSR (rows are out-edges): dependencies pulled from
    successors over out-edges (Algorithm 3's formula); also valid undirected."""
    lib = lib or load()
    rp, col, w = _csr(g)
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    out = np.empty(g.n, np.float64)
    _check(lib.oracle_bc_pull(g.n, _p(rp, _u64p), _p(col, _u32p), _p(w, _u32p), _p(src, _u32p) if len(src) else None,
                              len(src), scale, _p(out, _f64p)))
    return out


def edge_bc(g, sources, scale: float = 1.0, lib=None):
    """Per CSR entry (a -> b): scale * sum_s of the dependency share crossing
    it from a to b (zero unless a is a shortest-path predecessor of b)."""
    lib = lib or load()
    rp, col, w = _csr(g)
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    out = np.empty(max(g.nnz, 1), np.float64)
    _check(lib.oracle_edge_bc(g.n, _p(rp, _u64p), _p(col, _u32p), _p(w, _u32p), _p(src, _u32p) if len(src) else None,
                              len(src), scale, _p(out, _f64p)))
    return out[: g.nnz]


def phased(g, s: int, nonstrict: bool = False, reverse: bool = False, lib=None):
    """The paper's Algorithms 1-3 replayed sequentially (see brandes.c).
    Returns (dist, sigma, level, delta, nlevels)."""
    lib = lib or load()
    rp, col, w = _csr(g)
    d = np.empty(g.n, np.uint64)
    sig = np.empty(g.n, np.float64)
    lev = np.empty(g.n, np.uint32)
    dl = np.empty(g.n, np.float64)
    nl = ctypes.c_uint32(0)
    _check(lib.oracle_phased(g.n, _p(rp, _u64p), _p(col, _u32p), _p(w, _u32p), s, int(nonstrict), int(reverse),
                             _p(d, _u64p), _p(sig, _f64p), _p(lev, _u32p), _p(dl, _f64p), ctypes.byref(nl)))
    return d, sig, lev, dl, nl.value
