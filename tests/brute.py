"""Brute-force betweenness for tiny graphs, used to pin the oracle.

Nothing here shares code with ``oracle/``: distances come from Floyd-Warshall,
shortest-path counts from explicit enumeration of every simple path (each CSR
entry is a distinct edge, so parallel edges give distinct paths), and BC from
Eq. 1 of arxiv 1701.05975 (Sec. 2.1) summed over ordered pairs with exact
rational arithmetic.
"""
from __future__ import annotations

from fractions import Fraction

INF = float("inf")


def adjacency(g):
    """List of (neighbour, weight, entry index) per vertex, self-loops kept."""
    adj = [[] for _ in range(g.n)]
    for v in range(g.n):
        for e in range(int(g.row_ptr[v]), int(g.row_ptr[v + 1])):
            adj[v].append((int(g.col[e]), int(g.w[e]), e))
    return adj


def floyd_warshall(g):
    n = g.n
    d = [[INF] * n for _ in range(n)]
    for v in range(n):
        d[v][v] = 0
    for v, lst in enumerate(adjacency(g)):
        for u, w, _ in lst:
            if w < d[v][u]:
                d[v][u] = w
    for k in range(n):
        dk = d[k]
        for i in range(n):
            dik = d[i][k]
            if dik == INF:
                continue
            di = d[i]
            for j in range(n):
                if dik + dk[j] < di[j]:
                    di[j] = dik + dk[j]
    return d


def all_simple_paths(g, s):
    """Yield (target, length, vertex list, entry list) for every simple path
    starting at s (including the empty path s -> s)."""
    adj = adjacency(g)
    stack = [(s, 0, [s], [])]
    while stack:
        v, length, verts, ents = stack.pop()
        yield v, length, verts, ents
        for u, w, e in adj[v]:
            if u in verts:
                continue
            stack.append((u, length + w, verts + [u], ents + [e]))


def brute_force(g):
    """Return (dist, sigma, bc, ebc):
    dist[s][t] from Floyd-Warshall, sigma[s][t] = number of shortest s-t paths
    (by enumeration), bc[v] = sum over ordered s != v != t of
    sigma_st(v) / sigma_st (Eq. 1, Fraction), ebc[e] = sum over ordered pairs of
    the fraction of shortest s-t paths that traverse CSR entry e in its stored
    direction (Fraction)."""
    n = g.n
    dist = floyd_warshall(g)
    sigma = [[0] * n for _ in range(n)]
    bc = [Fraction(0)] * n
    ebc = [Fraction(0)] * g.nnz
    for s in range(n):
        through = [dict() for _ in range(n)]  # t -> {v: count}
        through_e = [dict() for _ in range(n)]  # t -> {entry: count}
        for t, length, verts, ents in all_simple_paths(g, s):
            if length != dist[s][t]:
                continue
            sigma[s][t] += 1
            for v in verts[1:-1]:
                through[t][v] = through[t].get(v, 0) + 1
            for e in ents:
                through_e[t][e] = through_e[t].get(e, 0) + 1
        for t in range(n):
            if t == s or sigma[s][t] == 0:
                continue
            for v, c in through[t].items():
                bc[v] += Fraction(c, sigma[s][t])
            for e, c in through_e[t].items():
                ebc[e] += Fraction(c, sigma[s][t])
    return dist, sigma, bc, ebc
