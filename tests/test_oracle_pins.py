"""Pins for the CPU oracle against things other than itself.

Each check below fixes the oracle through an independent route:
brute force (Floyd-Warshall + simple-path enumeration, exact rationals),
closed forms, the ordered-pair invariant computed with a library Dijkstra,
networkx's own betweenness, and the Eq. 3 / Eq. 4 example of Sec. 3.2
(tests/golden/fig1a_strict_vs_nonstrict.txt).
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from brute import brute_force
from paper_1701_05975_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
U64MAX = np.iinfo(np.uint64).max


def graph(n, edges):
    if edges:
        u, v, w = zip(*edges)
    else:
        u, v, w = (), (), ()
    return gen.csr_from_undirected(n, np.array(u, np.int64), np.array(v, np.int64), np.array(w, np.int64))


def close(a, b, rel=1e-12):
    """zero iff zero, else relative error <= rel (elementwise)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert a.shape == b.shape
    assert np.array_equal(a == 0, b == 0), (a, b)
    nz = b != 0
    err = np.abs(a[nz] - b[nz]) / np.abs(b[nz])
    assert err.size == 0 or err.max() <= rel, err.max()


def small_graphs(count, seed=1, nmax=7, wmax=3):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(1, nmax + 1))
        p = float(rng.choice([0.3, 0.5, 0.8]))
        yield gen.random_small_graph(n, p, 1, wmax, rng)


# ---------------------------------------------------------------------------
# brute force


def check_against_brute(g, lib=None):
    dist, sigma, bc_ref, ebc_ref = brute_force(g)
    for s in range(g.n):
        d, sg, _ = oracle.sssp(g, s, lib=lib)
        want_d = np.array([U64MAX if x == float("inf") else int(x) for x in dist[s]], dtype=np.uint64)
        assert np.array_equal(d, want_d), (s, d, want_d)
        assert np.array_equal(sg, np.array(sigma[s], dtype=np.float64)), (s, sg, sigma[s])
    allsrc = np.arange(g.n, dtype=np.uint32)
    close(oracle.bc(g, allsrc, 1.0, lib=lib), [float(x) for x in bc_ref])
    close(oracle.edge_bc(g, allsrc, 1.0, lib=lib), [float(x) for x in ebc_ref])


def test_brute_force_random_small_graphs():
    for g in small_graphs(250, seed=11):
        check_against_brute(g)


def test_brute_force_wide_weights():
    for g in small_graphs(80, seed=12, wmax=9):
        check_against_brute(g)


def test_brute_force_multigraph_and_self_loops():
    # parallel equal-weight edges double the path count; a self-loop is inert
    g = gen.csr_from_directed(4, [0, 1, 0, 1, 1, 2, 2, 3, 2], [1, 0, 1, 0, 2, 1, 3, 2, 2], [2, 2, 2, 2, 1, 1, 1, 1, 1])
    check_against_brute(g)
    d, sg, _ = oracle.sssp(g, 0)
    assert list(sg) == [1, 2, 2, 2]
    rng = np.random.default_rng(5)
    for _ in range(40):
        n = int(rng.integers(2, 6))
        k = int(rng.integers(1, 9))
        u = rng.integers(0, n, k)
        v = rng.integers(0, n, k)
        w = rng.integers(1, 3, k)
        check_against_brute(gen.csr_from_undirected(n, u, v, w))


# ---------------------------------------------------------------------------
# closed forms (undirected values: scale 1/2)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 13])
def test_path_graph_closed_form(n):
    rng = np.random.default_rng(n)
    edges = [(i, i + 1, int(rng.integers(1, 50))) for i in range(n - 1)]
    g = graph(n, edges)
    bc = oracle.bc(g, np.arange(n), 0.5)
    assert np.array_equal(bc, np.array([i * (n - 1 - i) for i in range(n)], np.float64))


@pytest.mark.parametrize("n", [3, 4, 7, 20])
def test_star_closed_form(n):
    rng = np.random.default_rng(n)
    g = graph(n, [(0, i, int(rng.integers(1, 9))) for i in range(1, n)])
    bc = oracle.bc(g, np.arange(n), 0.5)
    assert bc[0] == (n - 1) * (n - 2) / 2
    assert np.all(bc[1:] == 0)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 10, 11])
def test_cycle_closed_form(n):
    g = graph(n, [(i, (i + 1) % n, 1) for i in range(n)])
    bc = oracle.bc(g, np.arange(n), 0.5)
    want = (n - 1) * (n - 3) / 8 if n % 2 else (n - 2) ** 2 / 8
    np.testing.assert_allclose(bc, want, rtol=1e-13)


@pytest.mark.parametrize("n", [2, 4, 9])
def test_complete_graph_zero(n):
    g = graph(n, [(i, j, 3) for i in range(n) for j in range(i + 1, n)])
    assert np.all(oracle.bc(g, np.arange(n), 0.5) == 0)


def undirected_edge_sums(g, ebc):
    """Edge BC per undirected edge {a, b}: the sum of its two CSR entries."""
    rows, cols, _ = g.edges()
    und = {}
    for e, (a, b) in enumerate(zip(rows.tolist(), cols.tolist())):
        key = (min(a, b), max(a, b))
        und[key] = und.get(key, 0.0) + float(ebc[e])
    return und


@pytest.mark.parametrize("n", [2, 3, 6, 11])
def test_edge_bc_path_closed_form(n):
    # edge {i, i+1} of a path lies on the one path of every pair s <= i < t:
    # (i + 1)(n - 1 - i) unordered pairs, whatever the weights
    rng = np.random.default_rng(100 + n)
    g = graph(n, [(i, i + 1, int(rng.integers(1, 40))) for i in range(n - 1)])
    und = undirected_edge_sums(g, oracle.edge_bc(g, np.arange(n), 0.5))
    assert und == {(i, i + 1): float((i + 1) * (n - 1 - i)) for i in range(n - 1)}


@pytest.mark.parametrize("n", [2, 4, 9])
def test_edge_bc_star_closed_form(n):
    # the spoke to a leaf carries exactly the n - 1 pairs that contain the leaf
    rng = np.random.default_rng(200 + n)
    g = graph(n, [(0, i, int(rng.integers(1, 9))) for i in range(1, n)])
    und = undirected_edge_sums(g, oracle.edge_bc(g, np.arange(n), 0.5))
    assert und == {(0, i): float(n - 1) for i in range(1, n)}


@pytest.mark.parametrize("n", [3, 4, 5, 8, 9])
def test_edge_bc_unit_cycle_closed_form(n):
    # by symmetry every edge carries the same share of the pairs' hop counts:
    # odd n, n pairs at each distance k <= (n-1)/2, one path each:
    #   n (n-1)(n+1)/8 hops over n edges -> (n^2 - 1)/8 per edge;
    # even n, the n/2 antipodal pairs split over two n/2-hop paths:
    #   n^3/8 hops over n edges -> n^2/8 per edge
    g = graph(n, [(i, (i + 1) % n, 1) for i in range(n)])
    und = undirected_edge_sums(g, oracle.edge_bc(g, np.arange(n), 0.5))
    want = (n * n - 1) / 8 if n % 2 else n * n / 8
    assert len(und) == n
    np.testing.assert_allclose(list(und.values()), want, rtol=1e-13)


def test_unit_grid_binomial_counts():
    a, b = 9, 12
    edges = [(r * b + c, r * b + c + 1, 1) for r in range(a) for c in range(b - 1)]
    edges += [(r * b + c, (r + 1) * b + c, 1) for r in range(a - 1) for c in range(b)]
    g = graph(a * b, edges)
    d, sg, _ = oracle.sssp(g, 0)
    for r in range(a):
        for c in range(b):
            assert d[r * b + c] == r + c
            assert sg[r * b + c] == math.comb(r + c, r)


def test_random_tree_closed_form():
    # on a tree every pair has one path: BC(v) = ((n-1)^2 - sum_b |b|^2) / 2
    rng = np.random.default_rng(7)
    for n in (5, 30, 120):
        parent = [int(rng.integers(0, i)) for i in range(1, n)]
        g = graph(n, [(i + 1, parent[i], int(rng.integers(1, 100))) for i in range(n - 1)])
        adj = [[] for _ in range(n)]
        for i, p in enumerate(parent):
            adj[i + 1].append(p)
            adj[p].append(i + 1)
        want = []
        for v in range(n):
            sizes = []
            for start in adj[v]:
                seen = {v, start}
                stack = [start]
                while stack:
                    x = stack.pop()
                    for y in adj[x]:
                        if y not in seen:
                            seen.add(y)
                            stack.append(y)
                sizes.append(len(seen) - 1)
            want.append(((n - 1) ** 2 - sum(s * s for s in sizes)) / 2)
        bc = oracle.bc(g, np.arange(n), 0.5)
        assert np.array_equal(bc, np.array(want))
        leaves = [v for v in range(n) if len(adj[v]) == 1]
        assert np.all(bc[leaves] == 0)


# ---------------------------------------------------------------------------
# the ordered-pair invariant, with distances from scipy's Dijkstra


def invariant_total(g):
    """sum over ordered reachable pairs s != t of (E[#edges on a uniformly
    random shortest s-t path] - 1), from library distances and a hop-count
    dynamic programme over the tight edges."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import dijkstra

    n = g.n
    rows, cols, ws = g.edges()
    rows = rows.astype(np.int64)
    cols = cols.astype(np.int64)
    ws = ws.astype(np.int64)
    # scipy keeps the minimum of parallel entries via explicit min-reduction
    key = rows * n + cols
    order = np.lexsort((ws, key))
    key_s = key[order]
    first = np.ones(len(key_s), bool)
    first[1:] = key_s[1:] != key_s[:-1]
    sel = order[first]
    mat = sp.csr_matrix((ws[sel].astype(np.float64), (rows[sel], cols[sel])), shape=(n, n))
    D = dijkstra(mat, directed=True)
    total = Fraction(0)
    for s in range(n):
        ds = D[s]
        reach = np.flatnonzero(np.isfinite(ds))
        reach = reach[np.argsort(ds[reach], kind="stable")]
        sig = {int(s): 1}
        hops = {int(s): 0}  # sum over shortest paths of their edge counts
        for t in reach:
            t = int(t)
            if t == s:
                continue
            st = 0
            ht = 0
            for e in range(int(g.row_ptr[t]), int(g.row_ptr[t + 1])):
                p = int(g.col[e])
                if np.isfinite(ds[p]) and ds[p] + int(g.w[e]) == ds[t]:
                    st += sig[p]
                    ht += hops[p] + sig[p]
            sig[t] = st
            hops[t] = ht
            total += Fraction(ht, st) - 1
    return total


@pytest.mark.parametrize("maker", [
    lambda: gen.er_graph(150, 500, 1, 5, seed=3),
    lambda: gen.ba_graph(200, 3, 1, 4, seed=4),
    lambda: gen.grid_graph(12, 14, remove_frac=0.1, wmin=1, wmax=3, seed=5),
    lambda: gen.er_graph(120, 90, 1, 3, seed=6),  # many components
])
def test_ordered_pair_invariant(maker):
    g = maker()
    bc = oracle.bc(g, np.arange(g.n), 1.0)
    want = float(invariant_total(g))
    assert abs(bc.sum() - want) <= 1e-9 * max(1.0, abs(want))
    # edge form: every shortest path has (interior vertices + 1) edges
    ebc = oracle.edge_bc(g, np.arange(g.n), 1.0)
    import scipy.sparse.csgraph as csg
    import scipy.sparse as sp
    rows, cols, _ = g.edges()
    ncomp, lab = csg.connected_components(sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(g.n, g.n)))
    pairs = sum(c * (c - 1) for c in np.bincount(lab))
    assert abs(ebc.sum() - (want + pairs)) <= 1e-9 * (want + pairs)


# ---------------------------------------------------------------------------
# networkx (an independent implementation, run, not copied)


@pytest.mark.parametrize("maker", [
    lambda: gen.er_graph(300, 1500, 1, 20, seed=8),
    lambda: gen.ba_graph(400, 4, 1, 10, seed=9),
    lambda: gen.grid_graph(15, 15, remove_frac=0.05, wmin=1, wmax=4, seed=10),
])
def test_networkx_cross_check(maker):
    nx = pytest.importorskip("networkx")
    g = maker()
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    rows, cols, ws = g.edges()
    for a, b, w in zip(rows.tolist(), cols.tolist(), ws.tolist()):
        G.add_edge(a, b, weight=w)
    ref = nx.betweenness_centrality(G, weight="weight", normalized=False)
    bc = oracle.bc(g, np.arange(g.n), 0.5)
    np.testing.assert_allclose(bc, [ref[v] for v in range(g.n)], rtol=1e-9, atol=1e-9)
    eref = nx.edge_betweenness_centrality(G, weight="weight", normalized=False)
    ebc = oracle.edge_bc(g, np.arange(g.n), 0.5)
    und = {}
    for e, (a, b) in enumerate(zip(rows.tolist(), cols.tolist())):
        key = (min(a, b), max(a, b))
        und[key] = und.get(key, 0.0) + ebc[e]
    for (a, b), val in und.items():
        want = eref[(a, b)] if (a, b) in eref else eref[(b, a)]
        assert abs(val - want) <= 1e-9 * max(1.0, abs(want))


# ---------------------------------------------------------------------------
# Sec. 3.2: Eq. 3 (<=) breaks sigma, Eq. 4 (<) does not


def load_fig1a():
    edges, expects, sigma_strict, n, src = [], [], None, 0, 0
    with open(os.path.join(GOLDEN, "fig1a_strict_vs_nonstrict.txt")) as f:
        for line in f:
            tok = line.split()
            if not tok or tok[0].startswith("#"):
                continue
            if tok[0] == "n":
                n = int(tok[1])
            elif tok[0] == "source":
                src = int(tok[1])
            elif tok[0] == "edge":
                edges.append(tuple(int(x) for x in tok[1:4]))
            elif tok[0] == "expect":
                expects.append((tok[1], tok[2], int(tok[3])))
            elif tok[0] == "sigma_strict":
                sigma_strict = [int(x) for x in tok[1:]]
    return graph(n, edges), src, expects, sigma_strict


def test_fig1a_strict_vs_nonstrict():
    g, s, expects, sigma_strict = load_fig1a()
    for crit, order, want in expects:
        _, sg, _, _, _ = oracle.phased(g, s, nonstrict=(crit == "nonstrict"), reverse=(order == "reverse"))
        assert sg[3] == want, (crit, order, sg)
    _, sg, _, _, _ = oracle.phased(g, s)
    assert list(sg) == sigma_strict
    _, sg_b, _ = oracle.sssp(g, s)
    assert list(sg_b) == sigma_strict
    # the non-strict criterion still gets every distance right (Sec. 3.2)
    d_ns, _, _, _, _ = oracle.phased(g, s, nonstrict=True, reverse=True)
    d_b, _, _ = oracle.sssp(g, s)
    assert np.array_equal(d_ns, d_b)


def test_phased_unit_weights_settle_bfs_layers():
    # with every weight 1, Delta_node = 1, so Eq. 2 gives Delta_i = min_U d + 1
    # and Eq. 4 settles exactly the candidates at the smallest distance: the
    # batches are the breadth-first layers (level = hop distance from s)
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path

    rng = np.random.default_rng(31)
    graphs = [gen.er_graph(150, 260, 1, 1, seed=32), gen.grid_graph(7, 9, wmin=1, wmax=1, seed=33),
              graph(12, [(i, i + 1, 1) for i in range(11)])]
    for g in graphs:
        rows, cols, _ = g.edges()
        mat = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(g.n, g.n))
        for s in rng.choice(g.n, size=4, replace=False):
            hops = shortest_path(mat, unweighted=True, indices=int(s))
            _, _, lev, _, nlev = oracle.phased(g, int(s))
            reach = np.isfinite(hops)
            assert np.array_equal(lev[reach], hops[reach].astype(np.uint32))
            assert np.all(lev[~reach] == np.iinfo(np.uint32).max)
            assert nlev == int(hops[reach].max()) + 1


def test_phased_weighted_star_batches():
    # from the centre every leaf is a candidate with d = w and Delta_node = w,
    # so each batch takes every remaining leaf lighter than twice the lightest
    rng = np.random.default_rng(41)
    for trial in range(20):
        n = int(rng.integers(3, 14))
        ws = [int(x) for x in rng.integers(1, 30, size=n - 1)]
        g = graph(n, [(0, i + 1, ws[i]) for i in range(n - 1)])
        want = {0: 0}
        left, level = set(range(1, n)), 1
        while left:
            lightest = min(ws[v - 1] for v in left)
            batch = {v for v in left if ws[v - 1] < 2 * lightest}
            for v in batch:
                want[v] = level
            left -= batch
            level += 1
        _, _, lev, _, nlev = oracle.phased(g, 0)
        assert [int(x) for x in lev] == [want[v] for v in range(n)], (ws, lev)
        assert nlev == level


def test_phased_strict_matches_brandes_and_levels_are_legal():
    rng = np.random.default_rng(21)
    graphs = list(small_graphs(60, seed=22, wmax=4)) + [gen.er_graph(200, 700, 1, 6, seed=23),
                                                         gen.grid_graph(10, 10, wmin=1, wmax=5, seed=24)]
    for g in graphs:
        for s in rng.choice(g.n, size=min(g.n, 6), replace=False):
            s = int(s)
            for rev in (False, True):
                d, sg, lev, dl, nlev = oracle.phased(g, s, reverse=rev)
                d_b, sg_b, _ = oracle.sssp(g, s)
                assert np.array_equal(d, d_b)
                assert np.array_equal(sg, sg_b)
                dl_b = oracle.delta(g, s)
                keep = np.arange(g.n) != s
                close(dl[keep], dl_b[keep], rel=1e-12)
                rows, cols, ws = g.edges()
                for a, b, w in zip(rows.tolist(), cols.tolist(), ws.tolist()):
                    if d[a] != U64MAX and d[b] != U64MAX and int(d[a]) + w == int(d[b]):
                        assert lev[a] < lev[b]
                assert nlev == len(set(lev[lev != np.iinfo(np.uint32).max].tolist()))


# ---------------------------------------------------------------------------
# source-list semantics, threads, errors


def test_source_list_linearity_and_duplicates():
    g = gen.er_graph(80, 300, 1, 7, seed=31)
    a = np.array([0, 5, 9, 40], np.uint32)
    b = np.array([3, 77, 12], np.uint32)
    ab = oracle.bc(g, np.concatenate([a, b]), 1.0)
    np.testing.assert_allclose(ab, oracle.bc(g, a, 1.0) + oracle.bc(g, b, 1.0), rtol=1e-12)
    dup = oracle.bc(g, np.array([5, 5], np.uint32), 1.0)
    np.testing.assert_allclose(dup, 2 * oracle.bc(g, np.array([5], np.uint32), 1.0), rtol=1e-15)
    assert np.all(oracle.bc(g, np.zeros(0, np.uint32), 1.0) == 0)


def test_threads_match_single_thread():
    g = gen.ba_graph(500, 3, 1, 9, seed=32)
    src = np.arange(g.n, dtype=np.uint32)
    np.testing.assert_allclose(oracle.bc(g, src, 0.5, nthreads=4), oracle.bc(g, src, 0.5), rtol=1e-12)


def test_invalid_inputs_rejected():
    g = graph(3, [(0, 1, 1), (1, 2, 1)])
    bad = gen.CSRGraph(3, g.row_ptr.copy(), g.col.copy(), g.w.copy())
    bad.w[0] = 0
    with pytest.raises(oracle.OracleError):
        oracle.bc(bad, [0], 1.0)
    with pytest.raises(oracle.OracleError):
        oracle.bc(g, [3], 1.0)
    bad = gen.CSRGraph(3, g.row_ptr.copy(), g.col.copy(), g.w.copy())
    bad.col[0] = 7
    with pytest.raises(oracle.OracleError):
        oracle.sssp(bad, 0)


# ---------------------------------------------------------------------------
# directed graphs (Sec. 2.1: the method extends to them)


def test_directed_brute_force_small_graphs():
    rng = np.random.default_rng(61)
    for _ in range(150):
        n = int(rng.integers(1, 7))
        g = gen.random_small_digraph(n, float(rng.choice([0.2, 0.4, 0.7])), 1, 3, rng)
        dist, sigma, bc_ref, ebc_ref = brute_force(g)
        for s in range(g.n):
            d, sg, _ = oracle.sssp(g, s)
            want_d = np.array([U64MAX if x == float("inf") else int(x) for x in dist[s]], dtype=np.uint64)
            assert np.array_equal(d, want_d)
            assert np.array_equal(sg, np.array(sigma[s], dtype=np.float64))
        allsrc = np.arange(g.n, dtype=np.uint32)
        close(oracle.bc_directed(g, allsrc, 1.0), [float(x) for x in bc_ref])
        close(oracle.edge_bc(g, allsrc, 1.0), [float(x) for x in ebc_ref])


def test_directed_closed_forms():
    # directed path: v_i is interior to i * (n - 1 - i) ordered pairs
    for n in (2, 5, 9):
        g = gen.csr_from_directed(n, np.arange(n - 1), np.arange(1, n), np.full(n - 1, 3))
        assert np.array_equal(oracle.bc_directed(g, np.arange(n), 1.0), [i * (n - 1 - i) for i in range(n)])
    # directed unit cycle: every vertex (n - 1)(n - 2) / 2
    for n in (3, 4, 7):
        g = gen.csr_from_directed(n, np.arange(n), (np.arange(n) + 1) % n, np.ones(n))
        np.testing.assert_allclose(oracle.bc_directed(g, np.arange(n), 1.0), (n - 1) * (n - 2) / 2)


def test_pull_and_push_accumulation_agree_on_undirected_graphs():
    for g in [gen.er_graph(200, 900, 1, 6, seed=71), gen.ba_graph(300, 3, 1, 4, seed=72)]:
        src = np.arange(g.n, dtype=np.uint32)
        np.testing.assert_allclose(oracle.bc_directed(g, src, 0.5), oracle.bc(g, src, 0.5), rtol=1e-12, atol=0)


def test_directed_networkx_cross_check():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(73)
    g = gen.random_small_digraph(120, 0.05, 1, 9, rng)
    G = nx.DiGraph()
    G.add_nodes_from(range(g.n))
    rows, cols, ws = g.edges()
    for a, b, w in zip(rows.tolist(), cols.tolist(), ws.tolist()):
        G.add_edge(a, b, weight=w)
    ref = nx.betweenness_centrality(G, weight="weight", normalized=False)
    got = oracle.bc_directed(g, np.arange(g.n), 1.0)
    np.testing.assert_allclose(got, [ref[v] for v in range(g.n)], rtol=1e-9, atol=1e-9)
