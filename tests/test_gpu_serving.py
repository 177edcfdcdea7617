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
        outs = [np.zeros(g.n) for _ in range(6)]
        ids = [bc.bc_request_submit(G.handle, src, 1.0, o) for o in outs]
        last = ids[-1]
        try:
            bc.bc_request_cancel(last)
            cancelled = bc.bc_request_poll(last) == bc.BC_REQ_CANCELLED
        except bc.BCError as e:
            assert e.code == bc.BC_ERR_BUSY
            cancelled = False
        for rid in ids[:-1]:
            bc.bc_request_wait(rid, 120000)
        if cancelled:
            with pytest.raises(bc.BCError) as ei:
                bc.bc_request_wait(last, 1000)
            assert ei.value.code == bc.BC_ERR_CANCELLED
        else:
            bc.bc_request_wait(last, 120000)
        with pytest.raises(bc.BCError):
            bc.bc_request_poll(ids[0])  # forgotten after wait
        ref = G.compute(src, 1.0)
        assert_close(outs[0], ref)


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
    cancelled = set()
    for j in rng.choice(len(ids), size=8, replace=False):
        try:
            bc.bc_request_cancel(ids[j])
            if bc.bc_request_poll(ids[j]) == bc.BC_REQ_CANCELLED:
                cancelled.add(int(j))
        except bc.BCError as e:
            assert e.code == bc.BC_ERR_BUSY  # already running
    for j, rid in enumerate(ids):
        if j in cancelled:
            with pytest.raises(bc.BCError) as ei:
                bc.bc_request_wait(rid, 120000)
            assert ei.value.code == bc.BC_ERR_CANCELLED
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
