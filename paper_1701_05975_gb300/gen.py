"""Seeded synthetic graph and source-list generators.

This module serves both the oracle and the CUDA path and holds none of the
betweenness arithmetic: it only draws graphs and source lists.

Every generator returns an undirected weighted graph in CSR form: each
undirected edge {u, v, w} is stored twice, as (u -> v, w) and (v -> u, w), rows
sorted by neighbour id.  The paper stores the graph this way (Sec. 3.1: CSR plus
a parallel weight array; undirected graphs, Sec. 2.1).

Randomness: one ``numpy.random.Generator(PCG64)`` stream per generator stage
(edges, weights, removal, sources), spawned from ``SeedSequence(seed)``, so a
change in one stage never shifts the draws of another.
"""
from __future__ import annotations

import dataclasses

import numpy as np

STAGE_EDGES, STAGE_WEIGHTS, STAGE_REMOVAL, STAGE_SOURCES = range(4)


def _streams(seed: int):
    children = np.random.SeedSequence(seed).spawn(4)
    return [np.random.Generator(np.random.PCG64(c)) for c in children]


@dataclasses.dataclass
class CSRGraph:
    """Undirected weighted graph in CSR form (both directions stored)."""

    n: int
    row_ptr: np.ndarray  # uint64[n+1]
    col: np.ndarray  # uint32[nnz]
    w: np.ndarray  # uint32[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        """Undirected edge count (each stored twice; self-loops once)."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr).astype(np.int64))
        loops = int(np.count_nonzero(rows == self.col.astype(np.int64)))
        return (self.nnz - loops) // 2 + loops

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def edges(self):
        """(u, v, w) arrays of the stored directed entries."""
        rows = np.repeat(np.arange(self.n, dtype=np.uint32), np.diff(self.row_ptr).astype(np.int64))
        return rows, self.col, self.w


def csr_from_undirected(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray, name: str = "") -> CSRGraph:
    """Store each undirected edge (u, v, w) in both directions; no dedup here."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.asarray(w, dtype=np.uint32)
    loop = u == v
    src = np.concatenate([u, v[~loop]])
    dst = np.concatenate([v, u[~loop]])
    ww = np.concatenate([w, w[~loop]])
    return csr_from_directed(n, src, dst, ww, name)


def csr_from_directed(n: int, src, dst, w, name: str = "") -> CSRGraph:
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.asarray(w, dtype=np.uint32)
    order = np.argsort(src * np.int64(max(n, 1)) + dst, kind="stable")
    src, dst, w = src[order], dst[order], w[order]
    counts = np.bincount(src, minlength=n).astype(np.uint64)
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSRGraph(n=n, row_ptr=row_ptr, col=dst.astype(np.uint32), w=w.astype(np.uint32), name=name)


def _unique_pairs_sorted(u: np.ndarray, v: np.ndarray, n: int):
    """Canonical (min, max) pairs, self-loops and duplicates dropped, sorted."""
    a = np.minimum(u, v).astype(np.int64)
    b = np.maximum(u, v).astype(np.int64)
    keep = a != b
    key = a[keep] * n + b[keep]
    del a, b, keep
    key.sort()
    first = np.ones(len(key), dtype=bool)
    first[1:] = key[1:] != key[:-1]
    key = key[first]
    return key // n, key % n


def _dedup_pairs(u: np.ndarray, v: np.ndarray, n: int):
    """Canonical (min, max) pairs, self-loops dropped, duplicates dropped keeping
    the first occurrence in draw order."""
    a = np.minimum(u, v).astype(np.int64)
    b = np.maximum(u, v).astype(np.int64)
    keep = a != b
    a, b = a[keep], b[keep]
    key = a * n + b
    _, first = np.unique(key, return_index=True)
    first.sort()
    return a[first], b[first]


def er_graph(n: int, m: int, wmin: int = 1, wmax: int = 100, seed: int = 0) -> CSRGraph:
    """Erdos-Renyi G(n, m): m distinct unordered pairs u != v drawn uniformly;
    one weight per undirected edge, uniform integer in [wmin, wmax]."""
    rng_e, rng_w, _, _ = _streams(seed)
    if m > n * (n - 1) // 2:
        raise ValueError("m exceeds the number of vertex pairs")
    draw = max(2 * m, 64)
    au = np.empty(0, np.int64)
    bu = np.empty(0, np.int64)
    while True:
        u = rng_e.integers(0, n, size=draw)
        v = rng_e.integers(0, n, size=draw)
        au = np.concatenate([au, u])
        bu = np.concatenate([bu, v])
        a, b = _dedup_pairs(au, bu, n)
        if len(a) >= m:
            a, b = a[:m], b[:m]
            break
        draw *= 2
    w = rng_w.integers(wmin, wmax + 1, size=m, dtype=np.int64)
    return csr_from_undirected(n, a, b, w, name=f"er_n{n}_m{m}")


def ba_graph(n: int, m_attach: int = 4, wmin: int = 1, wmax: int = 1000, seed: int = 0) -> CSRGraph:
    """Barabasi-Albert preferential attachment.

    Seed graph: a clique on m_attach + 1 vertices.  Each later vertex attaches
    to m_attach distinct earlier vertices, each drawn with probability
    proportional to its current degree (uniform draw from the list of edge
    endpoints); no multi-edges.  Edge count = C(m0, 2) + m_attach (n - m0).
    """
    rng_e, rng_w, _, _ = _streams(seed)
    m0 = m_attach + 1
    if n < m0:
        raise ValueError("n must be at least m_attach + 1")
    n_edges = m0 * (m0 - 1) // 2 + m_attach * (n - m0)
    eu = np.empty(n_edges, dtype=np.int64)
    ev = np.empty(n_edges, dtype=np.int64)
    ends = np.empty(2 * n_edges, dtype=np.int64)  # repeated-endpoint list
    k = 0
    for i in range(m0):
        for j in range(i + 1, m0):
            eu[k], ev[k] = i, j
            ends[2 * k], ends[2 * k + 1] = i, j
            k += 1
    # pre-draw random indices in blocks to keep the Python loop light
    pool = rng_e.random(8 * m_attach * n)
    pi = 0
    for v in range(m0, n):
        chosen = []
        span = 2 * k
        while len(chosen) < m_attach:
            if pi >= len(pool):
                pool = rng_e.random(8 * m_attach * n)
                pi = 0
            t = int(ends[int(pool[pi] * span)])
            pi += 1
            if t not in chosen:
                chosen.append(t)
        for t in chosen:
            eu[k], ev[k] = v, t
            ends[2 * k], ends[2 * k + 1] = v, t
            k += 1
    w = rng_w.integers(wmin, wmax + 1, size=n_edges, dtype=np.int64)
    return csr_from_undirected(n, eu, ev, w, name=f"ba_n{n}_k{m_attach}")


def rmat_graph(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               wmin: int = 1, wmax: int = 255, seed: int = 0, permute: bool = True) -> CSRGraph:
    """R-MAT / Kronecker generator (Graph500 style, no noise).

    2^scale vertices, edge_factor * 2^scale generated edges; at each of the
    `scale` bit levels an edge picks quadrant (0,0), (0,1), (1,0), (1,1) with
    probabilities a, b, c, 1-a-b-c.  Vertex labels are then permuted at random,
    the edge set symmetrised, self-loops and duplicate pairs removed; one weight
    per remaining undirected edge, uniform integer in [wmin, wmax].
    """
    rng_e, rng_w, _, _ = _streams(seed)
    n = 1 << scale
    ne = edge_factor * n
    src = np.zeros(ne, dtype=np.uint32)
    dst = np.zeros(ne, dtype=np.uint32)
    fa, fab, fabc = np.float32(a), np.float32(a + b), np.float32(a + b + c)
    for bit in range(scale):
        r = rng_e.random(ne, dtype=np.float32)
        go_down = r >= fab  # quadrants (1,0), (1,1): source bit set
        go_right = (r >= fa) ^ go_down ^ (r >= fabc)  # quadrants (0,1), (1,1): target bit set
        src |= go_down.view(np.uint8).astype(np.uint32) << np.uint32(bit)
        dst |= go_right.view(np.uint8).astype(np.uint32) << np.uint32(bit)
        del r, go_down, go_right
    src = src.astype(np.int64)
    dst = dst.astype(np.int64)
    if permute:
        perm = rng_e.permutation(n).astype(np.int64)
        src = perm[src]
        dst = perm[dst]
    u, v = _unique_pairs_sorted(src, dst, n)
    del src, dst
    w = rng_w.integers(wmin, wmax + 1, size=len(u), dtype=np.int64)
    return csr_from_undirected(n, u, v, w, name=f"rmat_s{scale}_ef{edge_factor}")


def rmat_digraph(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
                 wmin: int = 1, wmax: int = 255, seed: int = 0) -> CSRGraph:
    """Directed R-MAT: the same draws as rmat_graph, but every generated
    (source, target) pair is kept as a directed edge (self-loops and repeated
    pairs removed); one weight per directed edge."""
    rng_e, rng_w, _, _ = _streams(seed)
    n = 1 << scale
    ne = edge_factor * n
    src = np.zeros(ne, dtype=np.uint32)
    dst = np.zeros(ne, dtype=np.uint32)
    fa, fab, fabc = np.float32(a), np.float32(a + b), np.float32(a + b + c)
    for bit in range(scale):
        r = rng_e.random(ne, dtype=np.float32)
        go_down = r >= fab
        go_right = (r >= fa) ^ go_down ^ (r >= fabc)
        src |= go_down.view(np.uint8).astype(np.uint32) << np.uint32(bit)
        dst |= go_right.view(np.uint8).astype(np.uint32) << np.uint32(bit)
    perm = rng_e.permutation(n).astype(np.int64)
    s64 = perm[src.astype(np.int64)]
    d64 = perm[dst.astype(np.int64)]
    keep = s64 != d64
    key = np.unique(s64[keep] * n + d64[keep])
    u, v = key // n, key % n
    w = rng_w.integers(wmin, wmax + 1, size=len(u), dtype=np.int64)
    return csr_from_directed(n, u, v, w, name=f"rmat_dir_s{scale}_ef{edge_factor}")


def random_small_digraph(n: int, p: float, wmin: int, wmax: int, rng: np.random.Generator) -> CSRGraph:
    """Tiny directed G(n, p) (each ordered pair independently)."""
    iu, ju = np.nonzero(~np.eye(n, dtype=bool))
    keep = rng.random(len(iu)) < p
    u, v = iu[keep], ju[keep]
    w = rng.integers(wmin, wmax + 1, size=len(u))
    return csr_from_directed(n, u, v, w, name=f"small_dir_n{n}")


def grid_graph(rows: int, cols: int, remove: int | None = None, remove_frac: float = 0.05,
               wmin: int = 1, wmax: int = 10000, seed: int = 0) -> CSRGraph:
    """4-neighbour rows x cols lattice (vertex id = r * cols + c) with `remove`
    edges (default round(remove_frac * E)) deleted uniformly without
    replacement; one weight per remaining edge, uniform integer in [wmin, wmax]."""
    rng_e, rng_w, rng_r, _ = _streams(seed)
    del rng_e
    n = rows * cols
    rr, cc = np.meshgrid(np.arange(rows, dtype=np.int64), np.arange(cols, dtype=np.int64), indexing="ij")
    ids = rr * cols + cc
    hu, hv = ids[:, :-1].ravel(), ids[:, 1:].ravel()
    vu, vv = ids[:-1, :].ravel(), ids[1:, :].ravel()
    u = np.concatenate([hu, vu])
    v = np.concatenate([hv, vv])
    total = len(u)
    if remove is None:
        remove = int(round(remove_frac * total))
    drop = rng_r.choice(total, size=remove, replace=False)
    keep = np.ones(total, dtype=bool)
    keep[drop] = False
    u, v = u[keep], v[keep]
    w = rng_w.integers(wmin, wmax + 1, size=len(u), dtype=np.int64)
    return csr_from_undirected(n, u, v, w, name=f"grid_{rows}x{cols}_rm{remove}")


def sample_sources(n: int, k: int, seed: int = 0) -> np.ndarray:
    """k distinct sources drawn uniformly without replacement (sources stream)."""
    _, _, _, rng_s = _streams(seed)
    if k >= n:
        return np.arange(n, dtype=np.uint32)
    return np.sort(rng_s.choice(n, size=k, replace=False)).astype(np.uint32)


def random_small_graph(n: int, p: float, wmin: int, wmax: int, rng: np.random.Generator) -> CSRGraph:
    """Tiny G(n, p) graph for exhaustive checks (caller supplies the stream)."""
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    u, v = iu[keep], ju[keep]
    w = rng.integers(wmin, wmax + 1, size=len(u))
    return csr_from_undirected(n, u, v, w, name=f"small_n{n}")


# ---------------------------------------------------------------------------
# The five workloads: ER 1k, BA 65k, R-MAT scale 20, perturbed 1024^2 grid,
# and the serving pool.


def workload_er1k():
    g = er_graph(1024, 8192, 1, 100, seed=0)
    return g, np.arange(g.n, dtype=np.uint32), 0.5


def workload_ba65k():
    g = ba_graph(65536, 4, 1, 1000, seed=0)
    return g, np.arange(g.n, dtype=np.uint32), 0.5


def workload_rmat20(k: int = 4096):
    g = rmat_graph(20, 16, 0.57, 0.19, 0.19, 1, 255, seed=0)
    src = sample_sources(g.n, k, seed=0)
    return g, src, 0.5 * g.n / k


def workload_rmat20_directed(k: int = 4096):
    """Directed R-MAT scale 20 (every generated pair kept as a directed edge),
    4096 uniform sources; ordered pairs, so the sampled scale is n / k."""
    g = rmat_digraph(20, 16, 0.57, 0.19, 0.19, 1, 255, seed=0)
    src = sample_sources(g.n, k, seed=0)
    return g, src, g.n / k


def workload_grid1024(k: int = 1024):
    g = grid_graph(1024, 1024, remove=104755, wmin=1, wmax=10000, seed=0)
    src = sample_sources(g.n, k, seed=0)
    return g, src, 0.5 * g.n / k


SERVING_SIZES = (1024, 4096, 16384, 65536, 262144)
SERVING_KINDS = ("er", "ba", "grid")


def serving_graph(kind: str, n: int, seed: int = 0) -> CSRGraph:
    """One graph of the serving pool: weights uniform in [1, 1000]."""
    if kind == "er":
        return er_graph(n, 8 * n, 1, 1000, seed=seed)
    if kind == "ba":
        return ba_graph(n, 4, 1, 1000, seed=seed)
    if kind == "grid":
        side = int(round(n ** 0.5))
        return grid_graph(side, side, remove_frac=0.05, wmin=1, wmax=1000, seed=seed)
    raise ValueError(kind)


@dataclasses.dataclass
class ServingRequest:
    arrival_s: float
    kind: str
    n: int
    sources: np.ndarray
    scale: float


def serving_requests(num: int = 2000, rate_per_s: float = 100.0, sizes=SERVING_SIZES, seed: int = 0,
                     exact_max_n: int = 16384, sampled_k: int = 256):
    """Poisson request stream over the pool: graph drawn uniformly from
    kinds x sizes; exact BC (all sources, scale 0.5) for n <= exact_max_n, else
    `sampled_k` uniform sources with scale 0.5 * n / k."""
    _, _, _, rng = _streams(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=num)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    pool = [(k, n) for k in SERVING_KINDS for n in sizes]
    picks = rng.integers(0, len(pool), size=num)
    for i in range(num):
        kind, n = pool[int(picks[i])]
        if n <= exact_max_n:
            src = np.arange(n, dtype=np.uint32)
            scale = 0.5
        else:
            src = np.sort(rng.choice(n, size=sampled_k, replace=False)).astype(np.uint32)
            scale = 0.5 * n / sampled_k
        out.append(ServingRequest(float(t[i]), kind, n, src, scale))
    return out
