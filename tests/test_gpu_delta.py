"""The delta-stepping schedule (BC_ALGO_DELTA) vs the CPU oracle, through the C ABI.

Same bar as the strict schedule: distances and sigma exact, BC zero exactly
where the oracle's is zero, else relative error <= 1e-9 per vertex.  The
schedule's backward levels are the hop depths of the shortest-path DAG
(longest DAG path from the source, in edges); the tests recompute those
depths from the oracle's distances and compare them level for level.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1701_05975_gb300 as bc
from paper_1701_05975_gb300 import gen
from test_gpu_parity import U64MAX, assert_bc_close, graph

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def default_config():
    c0 = bc.bc_get_config()
    yield
    bc.bc_set_config(c0)


def dag_depth(g, d):
    """Hop depth of every reached vertex in the shortest-path DAG of distances d."""
    rows, cols, ws = g.edges()
    dag = (d[rows] != U64MAX) & (d[rows] + ws.astype(np.uint64) == d[cols])
    pr, pc = rows[dag], cols[dag]
    depth = np.full(g.n, -1, np.int64)
    order = np.argsort(d, kind="stable")
    src_of = {}
    for a, b in zip(pr.tolist(), pc.tolist()):
        src_of.setdefault(b, []).append(a)
    for v in order.tolist():
        if d[v] == U64MAX:
            break
        preds = src_of.get(v, [])
        depth[v] = 0 if not preds else 1 + max(depth[p] for p in preds)
    return depth


def check_sssp(G, g, s):
    d, sg, lev = G.sssp_debug(s)
    d_ref, sg_ref, _ = oracle.sssp(g, s)
    assert np.array_equal(d, d_ref)
    assert np.array_equal(sg, sg_ref)
    depth = dag_depth(g, d_ref)
    reached = d_ref != U64MAX
    assert np.array_equal(lev[reached].astype(np.int64), depth[reached])
    assert np.all(lev[~reached] == np.iinfo(np.uint32).max)


CONFIGS = [
    dict(team_threads=32, bucket_width=1),
    dict(team_threads=128, bucket_width=0),
    dict(team_threads=256, bucket_width=7),
    dict(team_threads=512, bucket_width=1 << 40),
    dict(team_threads=1024, bucket_width=30),
]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: f"team{c['team_threads']}-w{c['bucket_width']}")
def test_small_random_graphs(cfg):
    bc.bc_set_config(algorithm=bc.BC_ALGO_DELTA, **cfg)
    rng = np.random.default_rng(707)
    for i in range(40):
        n = int(rng.integers(1, 70))
        g = gen.random_small_graph(n, float(rng.choice([0.05, 0.2, 0.6])), 1, int(rng.choice([1, 3, 50])), rng)
        src = np.arange(n, dtype=np.uint32)
        with bc.Graph(g) as G:
            assert_bc_close(G.compute(src, 1.0), oracle.bc(g, src, 1.0))
            assert G.stats().algorithm == bc.BC_ALGO_DELTA
            for s in (0, n // 2, n - 1):
                check_sssp(G, g, s)


def test_fig1a_and_edge_cases():
    g = graph(4, [(0, 1, 1), (1, 2, 1), (0, 2, 2), (2, 3, 1)])
    cases = [
        graph(1, []),
        graph(2, []),
        graph(2, [(0, 1, 7)]),
        graph(6, [(0, 1, 2), (1, 2, 2), (3, 4, 1), (4, 5, 1), (3, 5, 2)]),
        gen.csr_from_directed(4, [0, 1, 0, 1, 1, 2, 2, 3, 2, 3], [1, 0, 1, 0, 2, 1, 3, 2, 2, 3],
                              [2, 2, 2, 2, 1, 1, 1, 1, 1, 4]),
    ]
    for team in (32, 512):
        bc.bc_set_config(algorithm=bc.BC_ALGO_DELTA, team_threads=team, bucket_width=1)
        with bc.Graph(g) as G:
            d, sg, lev = G.sssp_debug(0)
        # Sec. 3.2, Fig. 1a: sigma(v3) = 2
        assert list(d) == [0, 1, 2, 3] and list(sg) == [1, 1, 2, 2]
        assert list(lev) == [0, 1, 2, 3]
        for c in cases:
            src = np.arange(c.n, dtype=np.uint32)
            with bc.Graph(c) as G:
                assert_bc_close(G.compute(src, 0.5), oracle.bc(c, src, 0.5))
                assert np.all(G.compute(np.zeros(0, np.uint32), 0.5) == 0)


@pytest.mark.parametrize("team", [32, 128, 512])
def test_er1k_workload_full(team):
    bc.bc_set_config(algorithm=bc.BC_ALGO_DELTA, team_threads=team)
    g, src, scale = gen.workload_er1k()
    want = oracle.bc(g, src, scale, nthreads=8)
    with bc.Graph(g) as G:
        assert_bc_close(G.compute(src, scale), want)
        for s in (0, 511):
            check_sssp(G, g, s)


def test_grid_sampled_sources_and_levels():
    # high-diameter case the schedule is for: 256 x 256 grid, weights 1..1000
    g = gen.grid_graph(256, 256, wmin=1, wmax=1000, seed=21)
    src = gen.sample_sources(g.n, 48, seed=22)
    want = oracle.bc(g, src, 1.0, nthreads=8)
    for team, width in ((128, 0), (256, 4000), (512, 64000)):
        bc.bc_set_config(algorithm=bc.BC_ALGO_DELTA, team_threads=team, bucket_width=width)
        with bc.Graph(g) as G:
            assert_bc_close(G.compute(src, 1.0), want)
            st = G.stats()
            assert st.sources == len(src) and st.levels > 0
            check_sssp(G, g, int(src[5]))


def test_ba65k_sampled_sources():
    g, _, _ = gen.workload_ba65k()
    src = gen.sample_sources(g.n, 128, seed=31)
    want = oracle.bc(g, src, 1.0, nthreads=8)
    with bc.Graph(g) as G:
        for team in (32, 512):
            bc.bc_set_config(algorithm=bc.BC_ALGO_DELTA, team_threads=team)
            assert_bc_close(G.compute(src, 1.0), want)
        check_sssp(G, g, int(src[0]))


def test_strict_and_delta_agree_on_rmat():
    g = gen.rmat_graph(14, 16, wmin=1, wmax=255, seed=41)
    src = gen.sample_sources(g.n, 96, seed=42)
    want = oracle.bc(g, src, 0.5, nthreads=8)
    with bc.Graph(g) as G:
        bc.bc_set_config(algorithm=bc.BC_ALGO_STRICT)
        strict = G.compute(src, 0.5)
        bc.bc_set_config(algorithm=bc.BC_ALGO_DELTA)
        delta = G.compute(src, 0.5)
    assert_bc_close(strict, want)
    assert_bc_close(delta, want)


def test_edge_bc_and_wide_weights():
    bc.bc_set_config(algorithm=bc.BC_ALGO_DELTA)
    g = gen.er_graph(300, 1200, 1, 5, seed=12)
    src = np.arange(g.n, dtype=np.uint32)
    with bc.Graph(g) as G:
        ebc, vbc = G.edge_compute(src, 0.5)
    assert_bc_close(ebc, oracle.edge_bc(g, src, 0.5))
    assert_bc_close(vbc, oracle.bc(g, src, 0.5))
    rng = np.random.default_rng(57)
    for i in range(8):
        n = int(rng.integers(2, 200))
        g = gen.random_small_graph(n, 0.1, 1, 2**31 - 1, rng)
        src = np.arange(n, dtype=np.uint32)
        with bc.Graph(g) as G:
            if g.nnz:
                assert G.info().dist_bits == 64
            assert_bc_close(G.compute(src, 1.0), oracle.bc(g, src, 1.0))
            check_sssp(G, g, 0)


def test_directed_graphs():
    rng = np.random.default_rng(909)
    for team in (32, 256):
        bc.bc_set_config(algorithm=bc.BC_ALGO_DELTA, team_threads=team)
        for i in range(20):
            n = int(rng.integers(1, 60))
            g = gen.random_small_digraph(n, float(rng.choice([0.03, 0.1, 0.3])), 1, int(rng.choice([1, 4, 60])), rng)
            src = np.arange(n, dtype=np.uint32)
            with bc.Graph(g, flags=bc.BC_DIRECTED) as G:
                assert_bc_close(G.compute(src, 1.0), oracle.bc_directed(g, src, 1.0))
                ebc, _ = G.edge_compute(src, 1.0)
                assert_bc_close(ebc, oracle.edge_bc(g, src, 1.0))
                check_sssp(G, g, n - 1)
    g = gen.rmat_digraph(14, 8, wmin=1, wmax=255, seed=5)
    src = gen.sample_sources(g.n, 64, seed=6)
    with bc.Graph(g, flags=bc.BC_DIRECTED) as G:
        assert_bc_close(G.compute(src, 1.0), oracle.bc_directed(g, src, 1.0))


def test_round_cap_and_recovery():
    # a path of 300 vertices with unit buckets needs ~300 rounds; a cap of 20
    # stops every source, restores its slab and reports BC_ERR_TIMEOUT
    g = graph(300, [(i, i + 1, 1) for i in range(299)])
    src = np.arange(0, 300, 3, dtype=np.uint32)
    with bc.Graph(g) as G:
        bc.bc_set_config(algorithm=bc.BC_ALGO_DELTA, bucket_width=1, phase_cap=20)
        with pytest.raises(bc.BCError) as ei:
            G.compute(src, 0.5)
        assert ei.value.code == bc.BC_ERR_TIMEOUT
        bc.bc_set_config(algorithm=bc.BC_ALGO_DELTA, bucket_width=1, phase_cap=0)
        assert_bc_close(G.compute(src, 0.5), oracle.bc(g, src, 0.5))


def test_autotune_considers_both_schedules():
    g = gen.grid_graph(128, 128, wmin=1, wmax=100, seed=61)
    src = gen.sample_sources(g.n, 64, seed=62)
    want = oracle.bc(g, src, 1.0, nthreads=8)
    with bc.Graph(g) as G:
        G.autotune(src)
        assert_bc_close(G.compute(src, 1.0), want)
        assert G.stats().algorithm in (bc.BC_ALGO_STRICT, bc.BC_ALGO_DELTA)
        bc.bc_set_config(algorithm=bc.BC_ALGO_STRICT)
        assert_bc_close(G.compute(src, 1.0), want)
        assert G.stats().algorithm == bc.BC_ALGO_STRICT
    with pytest.raises(bc.BCError):
        bc.bc_set_config(algorithm=3)
