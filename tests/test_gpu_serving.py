"""Serving (continuous batching): each request's result in a concurrent mix
equals the same request run alone, within the parity tolerance; admission
refuses a request that can never fit without disturbing the others."""
import time

import numpy as np
import pytest

import paper_1701_05975_gb300 as bc
from paper_1701_05975_gb300 import gen

pytestmark = pytest.mark.gpu
REL = 1e-9


def assert_close(got, want):
    assert np.array_equal(got == 0, want == 0)
    nz = want != 0
    if nz.any():
        assert (np.abs(got[nz] - want[nz]) / np.abs(want[nz])).max() <= REL


@pytest.fixture(autouse=True)
def restore_config():
    c0 = bc.bc_get_config()
    yield
    bc.bc_set_config(c0)


def test_mixed_stream_matches_requests_run_alone():
    pool = [gen.serving_graph(kind, n, seed=i) for i, (kind, n) in
            enumerate([("er", 1024), ("ba", 1024), ("grid", 1024), ("er", 4096), ("ba", 4096), ("grid", 4096),
                       ("ba", 16384)])]
    graphs = [bc.Graph(g) for g in pool]
    rng = np.random.default_rng(4)
    reqs = []
    for i in range(36):
        gi = int(rng.integers(len(pool)))
        n = pool[gi].n
        if n <= 4096:
            src = np.arange(n, dtype=np.uint32)
            scale = 0.5
        else:
            src = np.sort(rng.choice(n, 256, replace=False)).astype(np.uint32)
            scale = 0.5 * n / 256
        reqs.append((gi, src, scale))
    bc.bc_serving_reset()
    outs, ids = [], []
    for gi, src, scale in reqs:
        out = np.full(pool[gi].n, -1.0)
        outs.append(out)
        ids.append(bc.bc_request_submit(graphs[gi].handle, src, scale, out))
        time.sleep(float(rng.exponential(0.002)))
    for rid in ids:
        bc.bc_request_wait(rid, 60000)
    st = bc.bc_serving_stats_get()
    assert st.completed == len(reqs) and st.failed == 0
    assert st.max_concurrent >= 2, "requests never overlapped on the device"
    assert st.p99_ms >= st.p50_ms > 0
    for (gi, src, scale), out in zip(reqs, outs):
        alone = graphs[gi].compute(src, scale)
        assert_close(out, alone)
    for G in graphs:
        G.close()


def test_admission_refuses_oversize_request_and_keeps_others():
    small = gen.er_graph(64, 200, 1, 9, seed=1)
    big = gen.ba_graph(20000, 3, 1, 50, seed=2)
    with bc.Graph(small) as Gs, bc.Graph(big) as Gb:
        want = Gs.compute(np.arange(64, dtype=np.uint32), 0.5)
        out_small = np.zeros(64)
        rid = bc.bc_request_submit(Gs.handle, np.arange(64, dtype=np.uint32), 0.5, out_small)
        bc.bc_set_config(mem_fraction=1e-6)
        info = Gb.info()
        with pytest.raises(bc.BCError) as ei:
            bc.bc_request_submit(Gb.handle, np.arange(10, dtype=np.uint32), 1.0, np.zeros(big.n))
        assert ei.value.code == bc.BC_ERR_NOMEM, info.slab_bytes
        bc.bc_set_config(mem_fraction=0.0)
        bc.bc_request_wait(rid, 60000)
        assert_close(out_small, want)


def test_cancel_and_poll():
    g = gen.serving_graph("grid", 16384, seed=3)
    with bc.Graph(g) as G:
        src = np.arange(0, g.n, 4, dtype=np.uint32)
        outs = [np.full(g.n, -7.0) for _ in range(6)]
        ids = [bc.bc_request_submit(G.handle, src, 1.0, o) for o in outs]
        last = ids[-1]
        bc.bc_request_cancel(last)  # queued: cancelled now; running: at its next batch boundary
        for rid in ids[:-1]:
            bc.bc_request_wait(rid, 120000)
        ref = G.compute(src, 1.0)
        try:
            bc.bc_request_wait(last, 120000)
            assert_close(outs[-1], ref)  # it had finished before the cancel reached it
        except bc.BCError as e:
            assert e.code == bc.BC_ERR_CANCELLED
            assert np.all(outs[-1] == -7.0)  # a cancelled request never writes its output
        with pytest.raises(bc.BCError):
            bc.bc_request_poll(ids[0])  # forgotten after wait
        assert_close(outs[0], ref)


def test_running_request_cancels_at_a_batch_boundary_and_frees_its_workspace():
    g = gen.serving_graph("er", 16384, seed=5)
    with bc.Graph(g) as G:
        big_src = np.arange(g.n, dtype=np.uint32)  # many source batches
        out = np.full(g.n, -7.0)
        rid = bc.bc_request_submit(G.handle, big_src, 0.5, out)
        t0 = time.time()
        while bc.bc_request_poll(rid) == bc.BC_REQ_QUEUED and time.time() - t0 < 30:
            time.sleep(0.001)
        bc.bc_request_cancel(rid)
        try:
            bc.bc_request_wait(rid, 120000)
            finished = True
        except bc.BCError as e:
            assert e.code == bc.BC_ERR_CANCELLED
            finished = False
        if not finished:
            assert np.all(out == -7.0)
        # the graph's workspaces are free again: a new request completes correctly
        src = np.arange(0, g.n, 64, dtype=np.uint32)
        out2 = np.full(g.n, -7.0)
        bc.bc_request_wait(bc.bc_request_submit(G.handle, src, 1.0, out2), 120000)
        assert_close(out2, G.compute(src, 1.0))


def test_small_request_overtakes_a_large_one_between_its_batches():
    """Source batches interleave across requests: a small request submitted
    just after a large one (thousands of sources, many batches) on another
    graph completes while the large one is still running."""
    big = gen.serving_graph("er", 16384, seed=6)
    small = gen.serving_graph("ba", 1024, seed=7)
    with bc.Graph(big) as Gb, bc.Graph(small) as Gs:
        bc.bc_serving_reset()
        out_b = np.full(big.n, -7.0)
        out_s = np.full(small.n, -7.0)
        src_s = np.arange(0, small.n, 16, dtype=np.uint32)
        want_s = Gs.compute(src_s, 1.0)
        rid_b = bc.bc_request_submit(Gb.handle, np.arange(big.n, dtype=np.uint32), 0.5, out_b)
        time.sleep(0.02)
        rid_s = bc.bc_request_submit(Gs.handle, src_s, 1.0, out_s)
        bc.bc_request_wait(rid_s, 120000)
        assert bc.bc_request_poll(rid_b) == bc.BC_REQ_RUNNING
        assert_close(out_s, want_s)
        bc.bc_request_wait(rid_b, 120000)
        assert_close(out_b, Gb.compute(np.arange(big.n, dtype=np.uint32), 0.5))
        st = bc.bc_serving_stats_get()
        assert st.completed == 2 and st.max_concurrent >= 2


def test_randomised_stream_against_the_oracle():
    """Random graphs (directed ones too), random source lists (empty, repeated),
    random scales, a tight memory budget so requests queue, and cancellations:
    every completed request equals the oracle, every cancelled one is reported."""
    import oracle

    rng = np.random.default_rng(11)
    pool, flags = [], []
    for i in range(6):
        if i % 3 == 2:
            pool.append(gen.random_small_digraph(int(rng.integers(20, 90)), 0.08, 1, 50, rng))
            flags.append(bc.BC_DIRECTED)
        else:
            pool.append(gen.er_graph(int(rng.integers(200, 3000)), int(rng.integers(600, 9000)), 1,
                                     int(rng.choice([5, 1000])), seed=int(rng.integers(1 << 30))))
            flags.append(0)
    graphs = [bc.Graph(g, flags=f) for g, f in zip(pool, flags)]
    slab = max(G.info().slab_bytes for G in graphs)
    free_b = __import__("torch").cuda.mem_get_info()[0]
    # room for about forty slabs at a time: requests wait for each other
    bc.bc_set_config(mem_fraction=min(0.5, max(1e-4, 40.0 * slab / free_b)))
    reqs, outs, ids = [], [], []
    bc.bc_serving_reset()
    for i in range(60):
        gi = int(rng.integers(len(pool)))
        n = pool[gi].n
        k = int(rng.integers(0, min(n, 96) + 1))
        src = rng.choice(n, size=k, replace=bool(rng.integers(2))).astype(np.uint32)
        scale = float(rng.choice([1.0, 0.5, 2.5]))
        out = np.full(n, -7.0)
        reqs.append((gi, src, scale))
        outs.append(out)
        ids.append(bc.bc_request_submit(graphs[gi].handle, src, scale, out))
    asked = {int(j) for j in rng.choice(len(ids), size=8, replace=False)}
    for j in sorted(asked):
        bc.bc_request_cancel(ids[j])
    cancelled = set()
    for j, rid in enumerate(ids):
        if j in asked:
            try:
                bc.bc_request_wait(rid, 120000)  # it had finished before the cancel reached it
            except bc.BCError as e:
                assert e.code == bc.BC_ERR_CANCELLED
                assert np.all(outs[j] == -7.0)
                cancelled.add(j)
        else:
            bc.bc_request_wait(rid, 120000)
    for j, ((gi, src, scale), out) in enumerate(zip(reqs, outs)):
        if j in cancelled:
            continue
        ref = oracle.bc_directed if flags[gi] else oracle.bc
        assert_close(out, ref(pool[gi], src, scale))
    st = bc.bc_serving_stats_get()
    assert st.completed == len(reqs) - len(cancelled) and st.failed == 0
    for G in graphs:
        G.close()
