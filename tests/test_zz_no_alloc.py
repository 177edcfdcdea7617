"""bc_compute_noalloc, the entry point for callers that cannot allocate
device memory while they run (a real-time host thread, code running while
another framework owns the device allocator, a process whose memory is
reserved up front).  Its output is checked against the CPU oracle and
against bc_compute_async, on consecutive calls that share its fixed scratch
array: the same graph twice, then a smaller graph, then invalid inputs that
the device-side validation must reject, and a phase-cap hit, each followed by
a correct call.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It passes on its own in a
fresh process as well as after the other tests.
"""
import numpy as np
import pytest

import oracle
import paper_1701_05975_gb300 as bc
from paper_1701_05975_gb300 import gen

pytestmark = pytest.mark.gpu

REL = 1e-9


def assert_bc_close(got, want):
    assert np.array_equal(got == 0, want == 0)
    nz = want != 0
    if nz.any():
        assert (np.abs(got[nz] - want[nz]) / np.abs(want[nz])).max() <= REL


@pytest.fixture(autouse=True)
def restore_config():
    c0 = bc.bc_get_config()
    yield
    bc.bc_set_config(c0)


class Caller:
    """The caller's own device buffers for one graph (the test allocates them;
    the entry point does not) and the call itself."""

    def __init__(self, torch, row_ptr, col, w, n, sources):
        self.torch = torch
        dev = torch.device("cuda:0")
        self.stream = torch.cuda.Stream()
        self.n, self.nnz, self.k = n, len(col), len(sources)
        self.rp = torch.from_numpy(np.ascontiguousarray(row_ptr, np.uint64).view(np.int64)).to(dev)
        self.col = torch.from_numpy(np.ascontiguousarray(col, np.uint32).view(np.int32)).to(dev)
        self.w = torch.from_numpy(np.ascontiguousarray(w, np.uint32).view(np.int32)).to(dev)
        self.src = torch.from_numpy(np.ascontiguousarray(sources, np.uint32).view(np.int32)).to(dev)
        self.out = torch.empty(n, dtype=torch.float64, device=dev)
        self.status = torch.full((1,), -1, dtype=torch.int32, device=dev)

    def call(self, scale):
        self.out.fill_(-7.0)
        self.status.fill_(-1)
        bc.bc_compute_noalloc(self.rp.data_ptr(), self.col.data_ptr(), self.w.data_ptr(), self.n, self.nnz,
                              self.src.data_ptr(), self.k, scale, self.out.data_ptr(), self.status.data_ptr(),
                              self.stream.cuda_stream)
        self.stream.synchronize()
        return int(self.status.item()), self.out.cpu().numpy()


def existing_entry_point(torch, g, src, scale):
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()
    d_src = torch.from_numpy(src.view(np.int32)).to(dev)
    ref_out = torch.empty(g.n, dtype=torch.float64, device=dev)
    with bc.Graph(g) as G:
        bc.bc_compute_async(G.handle, d_src.data_ptr(), len(src), scale, ref_out.data_ptr(), stream.cuda_stream)
        bc.bc_sync_status(G.handle, stream.cuda_stream)
    return ref_out.cpu().numpy()


def test_noalloc_matches_existing_entry_point_and_oracle_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    g = gen.ba_graph(4000, 3, 1, 200, seed=31)
    src = gen.sample_sources(g.n, 600, seed=5)
    scale = 0.5 * g.n / len(src)
    want_ora = oracle.bc(g, src, scale, nthreads=4)
    want_api = existing_entry_point(torch, g, src, scale)
    assert_bc_close(want_api, want_ora)
    big = Caller(torch, g.row_ptr, g.col, g.w, g.n, src)
    for _ in range(2):
        status, got = big.call(scale)
        assert status == bc.BC_OK
        assert_bc_close(got, want_api)
        assert_bc_close(got, want_ora)
    # a smaller graph next: whatever the larger call left in the shared array
    # must not leak into this result
    h = gen.er_graph(700, 2100, 1, 50, seed=32)
    hs = np.arange(h.n, dtype=np.uint32)
    small = Caller(torch, h.row_ptr, h.col, h.w, h.n, hs)
    status, got = small.call(0.5)
    assert status == bc.BC_OK
    assert_bc_close(got, oracle.bc(h, hs, 0.5, nthreads=4))
    # and the larger one again
    status, got = big.call(scale)
    assert status == bc.BC_OK
    assert_bc_close(got, want_ora)


def invalid_variants(g):
    """Inputs that the device-side validation must reject (each keeps every
    index inside the caller's arrays, so no read goes out of bounds)."""
    src = np.arange(0, g.n, 7, dtype=np.uint32)
    out = []
    bad_src = src.copy()
    bad_src[3] = g.n  # a source id equal to n
    out.append(("source >= n", g.row_ptr, g.col, g.w, bad_src))
    w0 = g.w.copy()
    w0[5] = 0  # a zero weight (one direction of an edge)
    out.append(("zero weight", g.row_ptr, g.col, w0, src))
    # a one-way edge: the reverse entry of entry 0 gets another weight
    a = 0
    b = int(g.col[0])
    rev = int(g.row_ptr[b]) + int(np.flatnonzero(g.col[g.row_ptr[b]:g.row_ptr[b + 1]] == a)[0])
    w1 = g.w.copy()
    w1[rev] = w1[rev] + 1
    out.append(("asymmetric weights", g.row_ptr, g.col, w1, src))
    rp = g.row_ptr.copy()
    v = int(np.flatnonzero((np.diff(g.row_ptr) >= 2) & (g.row_ptr[:-1] > 0))[0])
    rp[v + 1] = rp[v] - 1  # row v ends before it starts; every value stays within [0, nnz]
    out.append(("row_ptr not monotone", rp, g.col, g.w, src))
    return out


def test_noalloc_rejects_invalid_device_inputs_then_recovers():
    torch = pytest.importorskip("torch")
    g = gen.er_graph(900, 3600, 1, 40, seed=33)
    src = np.arange(0, g.n, 7, dtype=np.uint32)
    want = oracle.bc(g, src, 1.0, nthreads=4)
    good = Caller(torch, g.row_ptr, g.col, g.w, g.n, src)
    for name, rp, col, w, s in invalid_variants(g):
        bad = Caller(torch, rp, col, w, g.n, s)
        status, got = bad.call(1.0)
        assert status == bc.BC_ERR_INVALID, name
        assert np.all(got == 0.0), name
        status, got = good.call(1.0)
        assert status == bc.BC_OK, name
        assert_bc_close(got, want)


def test_noalloc_phase_cap_reports_timeout_then_recovers():
    torch = pytest.importorskip("torch")
    g = gen.grid_graph(30, 30, remove=40, wmin=1, wmax=100, seed=34)
    src = np.arange(0, g.n, 11, dtype=np.uint32)
    caller = Caller(torch, g.row_ptr, g.col, g.w, g.n, src)
    bc.bc_set_config(phase_cap=3)
    status, _ = caller.call(1.0)
    assert status == bc.BC_ERR_TIMEOUT
    bc.bc_set_config(phase_cap=0)
    status, got = caller.call(1.0)
    assert status == bc.BC_OK
    assert_bc_close(got, oracle.bc(g, src, 1.0, nthreads=4))


def test_noalloc_rejects_graphs_beyond_its_scratch():
    n = 4_000_000  # one 64-bit per-source slab alone exceeds the fixed scratch
    with pytest.raises(bc.BCError) as ei:
        bc.bc_compute_noalloc(16, 16, 16, n, 0, 16, 1, 1.0, 16, 16, 0)
    assert ei.value.code == bc.BC_ERR_NOMEM
    assert "BC_NOALLOC_SCRATCH_BYTES" in str(ei.value)
