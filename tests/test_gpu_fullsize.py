"""Full-size workloads in the launch configuration the benchmark times.

At these sizes the oracle cannot redo every source, so each workload is
checked three ways: (1) the full launch against the sum of launches over a
partition of its source list (BC is additive over sources; this holds at any
size), (2) the GPU against the oracle on a sample of sources, over all n
outputs, and (3) bit-exact distances and sigma for sampled sources.
"""
import numpy as np
import pytest

import oracle
import paper_1701_05975_gb300 as bc
from paper_1701_05975_gb300 import gen

pytestmark = pytest.mark.gpu
REL = 1e-9


def assert_close(got, want, rel=REL):
    assert np.array_equal(got == 0, want == 0), np.flatnonzero((got == 0) != (want == 0))[:10]
    nz = want != 0
    if nz.any():
        err = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
        assert err.max() <= rel, err.max()


def run_async(G, n, sources, scale):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    d_src = torch.from_numpy(np.ascontiguousarray(sources, dtype=np.uint32).view(np.int32)).to(dev)
    d_out = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.cuda.Stream()
    bc.bc_compute_async(G.handle, d_src.data_ptr(), len(sources), scale, d_out.data_ptr(), st.cuda_stream)
    bc.bc_sync_status(G.handle, st.cuda_stream)
    return d_out.cpu().numpy()


def run_step(G, n, sources, scale, launches=2):
    """The benchmark's path: one batched run captured as a CUDA graph, replayed."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    d_src = torch.from_numpy(np.ascontiguousarray(sources, dtype=np.uint32).view(np.int32)).to(dev)
    d_out = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.cuda.Stream()
    step = bc.bc_step_create(G.handle, d_src.data_ptr(), len(sources), scale, d_out.data_ptr())
    try:
        for _ in range(launches):
            bc.bc_step_launch(step, st.cuda_stream)
        bc.bc_step_sync(step, st.cuda_stream)
    finally:
        bc.bc_step_destroy(step)
    return d_out.cpu().numpy()


def check_workload(g, sources, scale, parts, n_oracle, n_debug, tune=False):
    with bc.Graph(g) as G:
        if tune:  # the benchmark tunes on a 2048-source probe before it times
            G.autotune(sources[:2048])
        full = run_step(G, g.n, sources, scale)
        stats = G.stats()
        assert stats.sources == len(sources) and stats.pair_overflows == 0
        total = np.zeros(g.n)
        for chunk in np.array_split(sources, parts):
            total += run_async(G, g.n, chunk, scale)
        assert_close(full, total, rel=1e-11)
        assert_close(run_async(G, g.n, sources, scale), full, rel=1e-11)
        # oracle on a sample of sources that reach most of the graph
        deg = g.degrees()
        sample = [int(s) for s in sources if deg[s] > 0][:n_oracle]
        got = run_async(G, g.n, np.array(sample, np.uint32), 1.0)
        want = oracle.bc(g, np.array(sample, np.uint32), 1.0, nthreads=max(1, len(sample)))
        assert_close(got, want)
        for s in sample[:n_debug]:
            d, sg, lev = G.sssp_debug(s)
            d_ref, sg_ref, _ = oracle.sssp(g, s)
            assert np.array_equal(d, d_ref)
            assert np.array_equal(sg, sg_ref)
        return full, stats


def test_rmat20_directed_full_launch():
    g, sources, scale = gen.workload_rmat20_directed()
    with bc.Graph(g, flags=bc.BC_DIRECTED) as G:
        G.autotune(sources[:2048])
        full = run_step(G, g.n, sources, scale)
        st = G.stats()
        assert st.sources == len(sources) and st.pair_overflows == 0
        total = np.zeros(g.n)
        for chunk in np.array_split(sources, 4):
            total += run_async(G, g.n, chunk, scale)
        assert_close(full, total, rel=1e-11)
        # sources with out-edges reach part of the graph; compare every output
        outdeg = np.diff(g.row_ptr)
        sample = np.array([int(s) for s in sources if outdeg[s] > 0][:6], np.uint32)
        assert_close(run_async(G, g.n, sample, 1.0), oracle.bc_directed(g, sample, 1.0))
        for s in sample[:2]:
            d, sg, _ = G.sssp_debug(int(s))
            d_ref, sg_ref, _ = oracle.sssp(g, int(s))
            assert np.array_equal(d, d_ref) and np.array_equal(sg, sg_ref)


def run_edge_async(G, g, sources, scale):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    d_src = torch.from_numpy(np.ascontiguousarray(sources, dtype=np.uint32).view(np.int32)).to(dev)
    d_ebc = torch.empty(g.nnz, dtype=torch.float64, device=dev)
    d_bc = torch.empty(g.n, dtype=torch.float64, device=dev)
    st = torch.cuda.Stream()
    bc.bc_edge_compute_async(G.handle, d_src.data_ptr(), len(sources), scale, d_ebc.data_ptr(), d_bc.data_ptr(),
                             st.cuda_stream)
    bc.bc_sync_status(G.handle, st.cuda_stream)
    return d_ebc.cpu().numpy(), d_bc.cpu().numpy()


def test_rmat20_edge_full_launch():
    g, sources, scale = gen.workload_rmat20()
    with bc.Graph(g) as G:
        G.autotune(sources[:2048])
        ebc, vbc = run_edge_async(G, g, sources, scale)
        st = G.stats()
        assert st.sources == len(sources) and st.pair_overflows == 0  # the DAG-edge backward ran
        assert_close(vbc, run_async(G, g.n, sources, scale), rel=1e-11)
        parts = [run_edge_async(G, g, c, scale)[0] for c in np.array_split(sources, 2)]
        assert_close(ebc, parts[0] + parts[1], rel=1e-11)
        # a sample of sources: every entry's share against the oracle
        deg = g.degrees()
        sample = np.array([int(s) for s in sources if deg[s] > 0][:4], np.uint32)
        assert_close(run_edge_async(G, g, sample, 1.0)[0], oracle.edge_bc(g, sample, 1.0))


def test_rmat20_full_launch():
    g, sources, scale = gen.workload_rmat20()
    full, stats = check_workload(g, sources, scale, parts=4, n_oracle=6, n_debug=2, tune=True)
    assert stats.team_threads == 1024  # the configuration the benchmark measured
    # isolated vertices never lie on a path
    assert np.all(full[g.degrees() == 0] == 0)


def test_grid1024_full_launch():
    g, sources, scale = gen.workload_grid1024()
    check_workload(g, sources, scale, parts=2, n_oracle=3, n_debug=1)


def test_ba65k_full_launch():
    g, sources, scale = gen.workload_ba65k()
    check_workload(g, sources, scale, parts=2, n_oracle=16, n_debug=2)
