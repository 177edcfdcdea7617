"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerance (BASELINE target): distances bit-exact; sigma exact (integers
below 2^53); BC zero exactly where the oracle's is zero, else relative error
<= 1e-9 per vertex.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1701_05975_gb300 as bc
from paper_1701_05975_gb300 import gen

pytestmark = pytest.mark.gpu

REL = 1e-9
U64MAX = np.iinfo(np.uint64).max


def assert_bc_close(got, want, rel=REL):
    got = np.asarray(got)
    want = np.asarray(want)
    zg, zw = got == 0, want == 0
    assert np.array_equal(zg, zw), f"zero pattern differs at {np.flatnonzero(zg != zw)[:10]}"
    nz = ~zw
    if nz.any():
        err = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
        assert err.max() <= rel, f"max rel err {err.max():.3e} at {np.flatnonzero(nz)[err.argmax()]}"


@pytest.fixture(autouse=True)
def default_config():
    c0 = bc.bc_get_config()
    yield
    bc.bc_set_config(c0)


def graph(n, edges):
    u, v, w = zip(*edges) if edges else ((), (), ())
    return gen.csr_from_undirected(n, np.array(u, np.int64), np.array(v, np.int64), np.array(w, np.int64))


CONFIGS = [
    dict(team_threads=32, settle_in=1, bucket_width=0),
    dict(team_threads=128, settle_in=2, bucket_width=1),
    dict(team_threads=256, settle_in=1, bucket_width=3),
    dict(team_threads=512, settle_in=2, bucket_width=1 << 40),
    dict(team_threads=1024, settle_in=1, bucket_width=2),
    dict(team_threads=128, settle_in=3, bucket_width=0),
    dict(team_threads=1024, settle_in=3, bucket_width=1 << 40),
]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: f"team{c['team_threads']}-in{c['settle_in']}-w{c['bucket_width']}")
def test_small_random_graphs_all_team_shapes(cfg):
    bc.bc_set_config(**cfg)
    rng = np.random.default_rng(101)
    for i in range(40):
        n = int(rng.integers(1, 70))
        g = gen.random_small_graph(n, float(rng.choice([0.05, 0.2, 0.6])), 1, int(rng.choice([1, 3, 50])), rng)
        src = np.arange(n, dtype=np.uint32)
        with bc.Graph(g) as G:
            assert_bc_close(G.compute(src, 1.0), oracle.bc(g, src, 1.0))
            for s in (0, n // 2, n - 1):
                d, sg, lev = G.sssp_debug(s)
                d_ref, sg_ref, _ = oracle.sssp(g, s)
                assert np.array_equal(d, d_ref)
                assert np.array_equal(sg, sg_ref)


def test_fig1a_strict_criterion_on_gpu():
    # Sec. 3.2: the correct sigma of v3 is 2; Eq. 3 would give 1
    g = graph(4, [(0, 1, 1), (1, 2, 1), (0, 2, 2), (2, 3, 1)])
    for team in (32, 256):
        for si in (1, 2):
            bc.bc_set_config(team_threads=team, settle_in=si)
            with bc.Graph(g) as G:
                d, sg, lev = G.sssp_debug(0)
            assert list(d) == [0, 1, 2, 3]
            assert list(sg) == [1, 1, 2, 2]
            assert lev[1] < lev[2] < lev[3]


def test_edge_cases():
    # n = 1, isolated vertices, two components, self-loops, parallel edges
    cases = [
        graph(1, []),
        graph(2, []),
        graph(2, [(0, 1, 7)]),
        graph(6, [(0, 1, 2), (1, 2, 2), (3, 4, 1), (4, 5, 1), (3, 5, 2)]),
        gen.csr_from_directed(4, [0, 1, 0, 1, 1, 2, 2, 3, 2, 3], [1, 0, 1, 0, 2, 1, 3, 2, 2, 3],
                              [2, 2, 2, 2, 1, 1, 1, 1, 1, 4]),
    ]
    for g in cases:
        src = np.arange(g.n, dtype=np.uint32)
        for team in (32, 512):
            bc.bc_set_config(team_threads=team)
            with bc.Graph(g) as G:
                assert_bc_close(G.compute(src, 0.5), oracle.bc(g, src, 0.5))
                assert np.all(G.compute(np.zeros(0, np.uint32), 0.5) == 0)
                # edge output: parallel entries and self-loops pair with their twins
                ebc, _ = G.edge_compute(src, 0.5)
                assert_bc_close(ebc, oracle.edge_bc(g, src, 0.5))


def test_levels_are_legal_and_distances_exact_on_er1k():
    g, src, scale = gen.workload_er1k()
    with bc.Graph(g) as G:
        rows, cols, ws = g.edges()
        for s in (0, 17, 1023):
            d, sg, lev = G.sssp_debug(s)
            d_ref, sg_ref, _ = oracle.sssp(g, s)
            assert np.array_equal(d, d_ref)
            assert np.array_equal(sg, sg_ref)
            dag = (d[rows] != U64MAX) & (d[rows] + ws.astype(np.uint64) == d[cols])
            assert np.all(lev[rows[dag]] < lev[cols[dag]])


@pytest.mark.parametrize("team", [32, 128, 256, 512, 1024])
def test_er1k_workload_full(team):
    bc.bc_set_config(team_threads=team)
    g, src, scale = gen.workload_er1k()
    want = oracle.bc(g, src, scale, nthreads=8)
    with bc.Graph(g) as G:
        assert_bc_close(G.compute(src, scale), want)


def test_plain_mode_matches_oracle():
    g = gen.er_graph(400, 2400, 1, 100, seed=5)
    src = np.arange(0, g.n, 7, dtype=np.uint32)
    bc.bc_set_config(mode=bc.BC_MODE_PLAIN)
    with bc.Graph(g) as G:
        assert_bc_close(G.compute(src, 0.5), oracle.bc(g, src, 0.5))


def test_ba65k_sampled_sources():
    g, _, _ = gen.workload_ba65k()
    src = gen.sample_sources(g.n, 192, seed=3)
    want = oracle.bc(g, src, 1.0, nthreads=8)
    with bc.Graph(g) as G:
        for team in (32, 256):
            bc.bc_set_config(team_threads=team)
            assert_bc_close(G.compute(src, 1.0), want)
        d, sg, _ = G.sssp_debug(int(src[0]))
        d_ref, sg_ref, _ = oracle.sssp(g, int(src[0]))
        assert np.array_equal(d, d_ref) and np.array_equal(sg, sg_ref)


def test_linearity_duplicates_and_repeatability():
    g = gen.ba_graph(3000, 3, 1, 50, seed=9)
    a = np.arange(0, 3000, 5, dtype=np.uint32)
    b = np.arange(1, 3000, 7, dtype=np.uint32)
    with bc.Graph(g) as G:
        ab = G.compute(np.concatenate([a, b]), 1.0)
        sep = G.compute(a, 1.0) + G.compute(b, 1.0)
        np.testing.assert_allclose(ab, sep, rtol=1e-11, atol=0)
        one = G.compute(np.array([11], np.uint32), 1.0)
        two = G.compute(np.array([11, 11], np.uint32), 1.0)
        np.testing.assert_allclose(two, 2 * one, rtol=1e-13)
        r1 = G.compute(a, 0.5)
        r2 = G.compute(a, 0.5)
        np.testing.assert_allclose(r1, r2, rtol=1e-12)


def test_edge_bc_matches_oracle():
    g = gen.er_graph(300, 1200, 1, 5, seed=12)
    src = np.arange(g.n, dtype=np.uint32)
    with bc.Graph(g) as G:
        ebc, vbc = G.edge_compute(src, 0.5)
    assert_bc_close(ebc, oracle.edge_bc(g, src, 0.5))
    assert_bc_close(vbc, oracle.bc(g, src, 0.5))


def test_async_status_stays_with_its_stream():
    # two streams on one graph: each stream's status (an invalid source on one
    # of them) must come back to that stream's bc_sync_status, repeatedly
    torch = pytest.importorskip("torch")
    g = gen.er_graph(2000, 12000, 1, 50, seed=31)
    good = gen.sample_sources(g.n, 200, seed=32)
    bad = good.copy()
    bad[7] = g.n
    want = oracle.bc(g, good, 1.0)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    with bc.Graph(g) as G:
        d_good = torch.from_numpy(good.astype(np.int32)).cuda()
        d_bad = torch.from_numpy(bad.astype(np.int32)).cuda()
        out_a = torch.empty(g.n, dtype=torch.float64, device="cuda")
        out_b = torch.empty(g.n, dtype=torch.float64, device="cuda")
        for it in range(4):
            G.compute_async(d_bad, out_a, 1.0, stream=sa)
            G.compute_async(d_good, out_b, 1.0, stream=sb)
            order = (sa, sb) if it % 2 else (sb, sa)
            for st in order:
                if st is sa:
                    with pytest.raises(bc.BCError) as ei:
                        G.sync(sa)
                    assert ei.value.code == bc.BC_ERR_INVALID
                else:
                    G.sync(sb)
            assert_bc_close(out_b.cpu().numpy(), want)
        G.sync(sa)  # nothing pending any more on either stream
        G.sync(sb)


def test_edge_bc_async_device_buffers():
    torch = pytest.importorskip("torch")
    for g, flags, ref in ((gen.er_graph(300, 1200, 1, 5, seed=12), 0, oracle.bc),
                          (gen.rmat_digraph(12, 8, wmin=1, wmax=255, seed=7), bc.BC_DIRECTED, oracle.bc_directed)):
        src = gen.sample_sources(g.n, 48, seed=5)
        with bc.Graph(g, flags=flags | bc.BC_RELABEL_DEGREE) as G:
            d_src = torch.from_numpy(src.astype(np.int32)).cuda()
            d_ebc = torch.full((g.nnz,), 3.0, dtype=torch.float64, device="cuda")
            d_bc = torch.full((g.n,), 3.0, dtype=torch.float64, device="cuda")
            st = torch.cuda.Stream()
            bc.bc_edge_compute_async(G.handle, d_src.data_ptr(), len(src), 0.5, d_ebc.data_ptr(), d_bc.data_ptr(),
                                     st.cuda_stream)
            bc.bc_sync_status(G.handle, st.cuda_stream)
            assert_bc_close(d_ebc.cpu().numpy(), oracle.edge_bc(g, src, 0.5))
            assert_bc_close(d_bc.cpu().numpy(), ref(g, src, 0.5))
            with pytest.raises(bc.BCError):
                bc.bc_edge_compute_async(G.handle, d_src.data_ptr(), len(src), 0.5, 0, d_bc.data_ptr(), st.cuda_stream)


def test_batches_equal_the_paper_replay_with_an_unbounded_split():
    # with the split width unbounded every candidate sits in the near queue,
    # so the threshold is exactly Eq. 2's Delta_i; with the OUT test alone
    # (Eq. 4) the kernel must settle exactly the batches of the oracle's
    # sequential replay of Algorithm 2, vertex by vertex
    rng = np.random.default_rng(808)
    graphs = [gen.random_small_graph(int(rng.integers(2, 60)), 0.15, 1, int(rng.choice([3, 40])), rng)
              for _ in range(8)]
    graphs += [gen.er_graph(800, 4000, 1, 50, seed=81), gen.ba_graph(1500, 3, 1, 200, seed=82),
               gen.grid_graph(20, 25, wmin=1, wmax=9, seed=83)]
    for team in (128, 1024):
        bc.bc_set_config(team_threads=team, bucket_width=1 << 40, settle_in=2)
        for g in graphs:
            with bc.Graph(g) as G:
                for s in (0, g.n // 3, g.n - 1):
                    d, _, lev = G.sssp_debug(s)
                    d_ref, _, lev_ref, _, _ = oracle.phased(g, s)
                    reached = d_ref != U64MAX
                    assert np.array_equal(d, d_ref)
                    assert np.array_equal(lev[reached], lev_ref[reached]), (g.n, s, team)


def test_extreme_split_widths():
    rng = np.random.default_rng(66)
    graphs = [gen.er_graph(500, 2500, 1, 100, seed=61), gen.random_small_graph(120, 0.05, 1, 2**31 - 1, rng)]
    for width in (1 << 61, (1 << 64) - 1):
        bc.bc_set_config(bucket_width=width)
        for g in graphs:
            src = np.arange(0, g.n, 7, dtype=np.uint32)
            with bc.Graph(g) as G:
                assert_bc_close(G.compute(src, 0.5), oracle.bc(g, src, 0.5))


def test_default_cap_covers_tiny_split_widths():
    # a split width far below the weights makes almost every vertex its own
    # near-queue refill and second-level refill: phases + refills reach ~3n,
    # above a 2n bound, and the default cap (4n + 64) must still not trip
    g = gen.er_graph(2000, 8000, 1, 1 << 20, seed=77)
    src = np.array([5], np.uint32)
    for team in (128, 1024):
        bc.bc_set_config(team_threads=team, bucket_width=1)
        with bc.Graph(g) as G:
            assert_bc_close(G.compute(src, 1.0), oracle.bc(g, src, 1.0))
            st = G.stats()
            assert st.phases + st.refills > 2 * g.n + 64, (st.phases, st.refills)


def test_errors_and_timeout_recovery():
    g = gen.er_graph(500, 2000, 1, 30, seed=4)
    src = np.arange(50, dtype=np.uint32)
    with bc.Graph(g) as G:
        with pytest.raises(bc.BCError) as ei:
            G.compute(np.array([0, 500], np.uint32), 1.0)
        assert ei.value.code == bc.BC_ERR_INVALID
        bc.bc_set_config(phase_cap=3)
        with pytest.raises(bc.BCError) as ei:
            G.compute(src, 1.0)
        assert ei.value.code == bc.BC_ERR_TIMEOUT
        bc.bc_set_config(phase_cap=0)
        assert_bc_close(G.compute(src, 1.0), oracle.bc(g, src, 1.0))


def test_async_with_torch_buffers():
    torch = pytest.importorskip("torch")
    g = gen.er_graph(2000, 10000, 1, 100, seed=6)
    src = np.arange(0, g.n, 3, dtype=np.uint32)
    want = oracle.bc(g, src, 0.25)
    dev = torch.device("cuda:0")
    d_src = torch.from_numpy(src.astype(np.int32)).to(dev)
    d_out = torch.empty(g.n, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream()
    with bc.Graph(g) as G:
        with torch.cuda.stream(stream):
            bc.bc_compute_async(G.handle, d_src.data_ptr(), len(src), 0.25, d_out.data_ptr(), stream.cuda_stream)
        bc.bc_sync_status(G.handle, stream.cuda_stream)
        assert_bc_close(d_out.cpu().numpy(), want)
        bad = torch.tensor([0, g.n + 5], dtype=torch.int32, device=dev)
        bc.bc_compute_async(G.handle, bad.data_ptr(), 2, 1.0, d_out.data_ptr(), stream.cuda_stream)
        with pytest.raises(bc.BCError) as ei:
            bc.bc_sync_status(G.handle, stream.cuda_stream)
        assert ei.value.code == bc.BC_ERR_INVALID


@pytest.mark.parametrize("flags", [bc.BC_RELABEL_DEGREE, bc.BC_KEEP_ORDER])
def test_relabeled_and_kept_layouts_agree_with_oracle(flags):
    rng = np.random.default_rng(77)
    for i in range(12):
        g = gen.ba_graph(int(rng.integers(6, 300)), int(rng.integers(1, 4)), 1, int(rng.choice([2, 40])), seed=i)
        src = np.arange(g.n, dtype=np.uint32)
        with bc.Graph(g, flags=flags) as G:
            assert_bc_close(G.compute(src, 0.5), oracle.bc(g, src, 0.5))
            ebc, _ = G.edge_compute(src[::3], 1.0)
            assert_bc_close(ebc, oracle.edge_bc(g, src[::3], 1.0))
            s = int(rng.integers(0, g.n))
            d, sg, lev = G.sssp_debug(s)
            d_ref, sg_ref, _ = oracle.sssp(g, s)
            assert np.array_equal(d, d_ref) and np.array_equal(sg, sg_ref)
    g = gen.er_graph(300, 1000, 1, 9, seed=3)
    bc.bc_set_config(mode=bc.BC_MODE_PLAIN)
    with bc.Graph(g, flags=flags) as G:
        assert_bc_close(G.compute(np.arange(0, 300, 11, dtype=np.uint32), 1.0),
                        oracle.bc(g, np.arange(0, 300, 11, dtype=np.uint32), 1.0))


def test_dag_edge_list_overflow_falls_back_to_entry_scan():
    # layers of 20 vertices, complete bipartite between consecutive layers,
    # unit weights: every vertex beyond the first layer has 20 predecessors,
    # far more DAG edges than the per-source list holds (2 n + 64)
    L, layers = 20, 5
    edges = [(a * L + i, (a + 1) * L + j, 1) for a in range(layers - 1) for i in range(L) for j in range(L)]
    g = graph(L * layers, edges)
    src = np.arange(g.n, dtype=np.uint32)
    for team in (32, 256):
        bc.bc_set_config(team_threads=team)
        with bc.Graph(g) as G:
            assert_bc_close(G.compute(src, 0.5), oracle.bc(g, src, 0.5))
            st = G.stats()
            assert st.pair_overflows > 0
            ebc, _ = G.edge_compute(src, 0.5)  # edge output falls back to the entry scan too
            assert_bc_close(ebc, oracle.edge_bc(g, src, 0.5))
            assert G.stats().pair_overflows > 0
            d, sg, _ = G.sssp_debug(0)
            d_ref, sg_ref, _ = oracle.sssp(g, 0)
            assert np.array_equal(d, d_ref) and np.array_equal(sg, sg_ref)
    g2 = gen.er_graph(500, 3000, 1, 1000, seed=2)
    with bc.Graph(g2) as G:
        G.compute(np.arange(500, dtype=np.uint32), 1.0)
        st = G.stats()
        assert st.pair_overflows == 0 and st.dag_edges >= 499 * 500 * 0.9


def test_wide_weights_use_unpacked_entries_and_64bit_distances():
    # 1024-thread teams hold 32-bit distances only: the request falls back to 512
    bc.bc_set_config(team_threads=1024)
    rng = np.random.default_rng(55)
    for i in range(10):
        n = int(rng.integers(2, 200))
        g = gen.random_small_graph(n, 0.1, 1, 2**31 - 1, rng)
        src = np.arange(n, dtype=np.uint32)
        with bc.Graph(g) as G:
            if g.nnz:
                assert G.info().dist_bits == 64
            assert_bc_close(G.compute(src, 1.0), oracle.bc(g, src, 1.0))
            if g.nnz:
                assert G.stats().team_threads == 512
            d, sg, _ = G.sssp_debug(0)
            d_ref, sg_ref, _ = oracle.sssp(g, 0)
            assert np.array_equal(d, d_ref) and np.array_equal(sg, sg_ref)


@pytest.mark.parametrize("team", [32, 128, 512])
def test_settled_neighbour_refinement_settles_larger_batches(team):
    """settle_in = 1 raises a candidate's Delta_node to its second smallest
    incident weight once its lightest neighbour is known to be settled: the
    results stay exact and the grid settles in clearly fewer phases than with
    Delta_node alone (settle_in = 3)."""
    g = gen.grid_graph(120, 120, remove_frac=0.05, wmin=1, wmax=10000, seed=71)
    src = gen.sample_sources(g.n, 24, seed=72)
    want = oracle.bc(g, src, 1.0, nthreads=8)
    phases = {}
    for settle_in in (3, 1):
        bc.bc_set_config(team_threads=team, settle_in=settle_in)
        with bc.Graph(g) as G:
            assert_bc_close(G.compute(src, 1.0), want)
            phases[settle_in] = G.stats().phases
            rows, cols, ws = g.edges()
            for s in (int(src[0]), int(src[1])):
                d, sg, lev = G.sssp_debug(s)
                d_ref, sg_ref, _ = oracle.sssp(g, s)
                assert np.array_equal(d, d_ref) and np.array_equal(sg, sg_ref)
                # no shortest-path DAG edge inside a settle batch
                dag = (d[rows] != U64MAX) & (d[rows] + ws.astype(np.uint64) == d[cols])
                assert np.all(lev[rows[dag]] < lev[cols[dag]])
    assert phases[1] < 0.85 * phases[3], phases


def broom_graph(seed):
    """A 400-vertex star (hub 0) with chords, plus a 100-vertex path hanging
    off leaf 399; weights 10^6 x U{4..10}.  n x max_w is above 2^31, but the
    hop eccentricity from the hub is 101, so every distance (up to ~10^9) is
    bounded by 2 x 101 x 10^7 and fits a 32-bit word."""
    rng = np.random.default_rng(seed)
    edges = [(0, i) for i in range(1, 400)] + [(i, i + 1) for i in range(399, 499)]
    chords = rng.integers(1, 400, size=(300, 2))
    edges += [(int(a), int(b)) for a, b in chords if a != b]
    u, v = np.array(edges).T
    uniq = gen._dedup_pairs(u, v, 500)
    w = 1_000_000 * rng.integers(4, 11, size=len(uniq[0]))
    return gen.csr_from_undirected(500, uniq[0], uniq[1], w)


@pytest.mark.parametrize("team", [32, 256, 1024])
def test_hop_bound_gives_32bit_distances_up_to_1e9(team):
    bc.bc_set_config(team_threads=team)
    g = broom_graph(61)
    src = np.arange(g.n, dtype=np.uint32)
    with bc.Graph(g) as G:
        assert G.info().dist_bits == 32
        assert_bc_close(G.compute(src, 1.0), oracle.bc(g, src, 1.0))
        for s in (0, 250, 499):
            d, sg, _ = G.sssp_debug(s)
            d_ref, sg_ref, _ = oracle.sssp(g, s)
            assert np.array_equal(d, d_ref) and np.array_equal(sg, sg_ref)
        assert d_ref.max() > 5e8  # the words really hold large distances


def test_distance_width_falls_back_to_64_bits():
    # a long path: the hop bound (2 x 299 x 10^7) does not fit
    n = 300
    path = graph(n, [(i, i + 1, 10_000_000) for i in range(n - 1)])
    with bc.Graph(path) as G:
        assert G.info().dist_bits == 64
        src = np.arange(0, n, 3, dtype=np.uint32)
        assert_bc_close(G.compute(src, 1.0), oracle.bc(path, src, 1.0))
    # directed graphs keep the (n - 1) max_w bound
    rng = np.random.default_rng(62)
    dg = gen.random_small_digraph(400, 0.02, 4_000_000, 10_000_000, rng)
    with bc.Graph(dg, flags=bc.BC_DIRECTED) as G:
        assert G.info().dist_bits == 64
    # an asymmetric CSR passed as undirected: the hop bound does not apply
    # (the graph is only created, not run: it is outside the undirected contract)
    b = broom_graph(63)
    w = b.w.copy()
    w[0] += 1
    asym = gen.CSRGraph(n=b.n, row_ptr=b.row_ptr, col=b.col, w=w, name="asym")
    with bc.Graph(asym) as G:
        assert G.info().dist_bits == 64


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: f"team{c['team_threads']}-in{c['settle_in']}")
def test_directed_small_graphs(cfg):
    bc.bc_set_config(**cfg)
    rng = np.random.default_rng(303)
    for i in range(25):
        n = int(rng.integers(1, 60))
        g = gen.random_small_digraph(n, float(rng.choice([0.03, 0.1, 0.3])), 1, int(rng.choice([1, 4, 60])), rng)
        src = np.arange(n, dtype=np.uint32)
        with bc.Graph(g, flags=bc.BC_DIRECTED) as G:
            assert G.info().directed == 1
            assert_bc_close(G.compute(src, 1.0), oracle.bc_directed(g, src, 1.0))
            ebc, _ = G.edge_compute(src, 1.0)
            assert_bc_close(ebc, oracle.edge_bc(g, src, 1.0))
            for s in (0, n - 1):
                d, sg, lev = G.sssp_debug(s)
                d_ref, sg_ref, _ = oracle.sssp(g, s)
                assert np.array_equal(d, d_ref) and np.array_equal(sg, sg_ref)


@pytest.mark.parametrize("layout", [bc.BC_RELABEL_DEGREE, bc.BC_KEEP_ORDER])
def test_directed_rmat(layout):
    g = gen.rmat_digraph(14, 8, wmin=1, wmax=255, seed=5)
    src = gen.sample_sources(g.n, 64, seed=6)
    want = oracle.bc_directed(g, src, 1.0)
    with bc.Graph(g, flags=bc.BC_DIRECTED | layout) as G:
        assert_bc_close(G.compute(src, 1.0), want)
        d, sg, _ = G.sssp_debug(int(src[3]))
        d_ref, sg_ref, _ = oracle.sssp(g, int(src[3]))
        assert np.array_equal(d, d_ref) and np.array_equal(sg, sg_ref)
        bc.bc_set_config(mode=bc.BC_MODE_PLAIN)
        with pytest.raises(bc.BCError) as ei:
            G.compute(src[:2], 1.0)
        assert ei.value.code == bc.BC_ERR_INVALID


@pytest.mark.parametrize("node_parallel", [True, False])
@pytest.mark.parametrize("vwarp", [1, 4, 8, 16, 32])
def test_paper_thread_mappings_match_oracle(node_parallel, vwarp):
    rng = np.random.default_rng(vwarp + 100 * node_parallel)
    graphs = [gen.random_small_graph(int(rng.integers(1, 50)), 0.2, 1, 10, rng) for _ in range(6)]
    graphs += [gen.er_graph(700, 5000, 1, 10, seed=8), gen.rmat_graph(10, 8, wmin=1, wmax=10, seed=9)]
    # a graph with unreached vertices and 32-bit distances
    graphs.append(gen.er_graph(3000, 1500, 1, 10, seed=10))
    for g in graphs:
        src = np.arange(0, g.n, max(1, g.n // 40), dtype=np.uint32)
        with bc.Graph(g) as G:
            got = G.compute_paper_variant(src, 0.5, node_parallel=node_parallel, vwarp=vwarp)
            assert_bc_close(got, oracle.bc(g, src, 0.5))
            assert G.stats().sources == len(src)
            # the replay of Algorithm 2 settles exactly the oracle replay's batches
            for s in src[:3]:
                G.compute_paper_variant(np.array([s], np.uint32), 1.0, node_parallel=node_parallel, vwarp=vwarp)
                nlev = oracle.phased(g, int(s))[4]
                assert G.stats().phases == nlev - 1
