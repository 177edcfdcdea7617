"""bc_compute_noalloc, the entry point for callers that cannot allocate
device memory while they run, checked against bc_compute_async.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It passes on its own in a
fresh process as well as after the other tests.
"""
import numpy as np
import pytest

import paper_1701_05975_gb300 as bc
from paper_1701_05975_gb300 import gen

pytestmark = pytest.mark.gpu

REL = 1e-9


def assert_bc_close(got, want):
    assert np.array_equal(got == 0, want == 0)
    nz = want != 0
    if nz.any():
        assert (np.abs(got[nz] - want[nz]) / np.abs(want[nz])).max() <= REL


def test_noalloc_matches_existing_entry_point_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()
    g = gen.ba_graph(4000, 3, 1, 200, seed=31)
    src = gen.sample_sources(g.n, 600, seed=5)
    scale = 0.5 * g.n / len(src)
    # caller-owned device buffers (the test allocates them; the entry point does not)
    d_rp = torch.from_numpy(g.row_ptr.view(np.int64)).to(dev)
    d_col = torch.from_numpy(g.col.view(np.int32)).to(dev)
    d_w = torch.from_numpy(g.w.view(np.int32)).to(dev)
    d_src = torch.from_numpy(src.view(np.int32)).to(dev)
    d_out = torch.empty(g.n, dtype=torch.float64, device=dev)
    d_status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    # the existing entry point
    ref_out = torch.empty(g.n, dtype=torch.float64, device=dev)
    with bc.Graph(g) as G:
        bc.bc_compute_async(G.handle, d_src.data_ptr(), len(src), scale, ref_out.data_ptr(), stream.cuda_stream)
        bc.bc_sync_status(G.handle, stream.cuda_stream)
    want = ref_out.cpu().numpy()
    for _ in range(2):
        d_out.fill_(-7.0)
        d_status.fill_(-1)
        bc.bc_compute_noalloc(d_rp.data_ptr(), d_col.data_ptr(), d_w.data_ptr(), g.n, g.nnz, d_src.data_ptr(),
                              len(src), scale, d_out.data_ptr(), d_status.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        assert int(d_status.item()) == bc.BC_OK
        assert_bc_close(d_out.cpu().numpy(), want)


def test_noalloc_rejects_graphs_beyond_its_scratch():
    n = 4_000_000  # one 64-bit per-source slab alone exceeds the fixed scratch
    with pytest.raises(bc.BCError) as ei:
        bc.bc_compute_noalloc(16, 16, 16, n, 0, 16, 1, 1.0, 16, 16, 0)
    assert ei.value.code == bc.BC_ERR_NOMEM
    assert "BC_NOALLOC_SCRATCH_BYTES" in str(ei.value)
