"""Step graphs (bc_step_*): one batched run captured as a CUDA graph and replayed.

Every replay must give the oracle's result for the sources the device buffer
holds at launch time (same tolerance as the other parity tests).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1701_05975_gb300 as bc
from paper_1701_05975_gb300 import gen
from test_gpu_parity import assert_bc_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def default_config():
    c0 = bc.bc_get_config()
    yield
    bc.bc_set_config(c0)


def dev_sources(src):
    return torch.from_numpy(np.asarray(src, np.int32)).cuda()


def test_replays_match_oracle_and_follow_rewritten_sources():
    g = gen.er_graph(300, 1500, 1, 40, seed=71)
    a = gen.sample_sources(g.n, 64, seed=72)
    b = gen.sample_sources(g.n, 64, seed=73)
    st = torch.cuda.Stream()
    with bc.Graph(g) as G:
        d_src = dev_sources(a)
        d_out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        step = bc.bc_step_create(G.handle, d_src.data_ptr(), len(a), 0.5, d_out.data_ptr())
        try:
            want_a = oracle.bc(g, a, 0.5)
            for _ in range(3):
                bc.bc_step_launch(step, st.cuda_stream)
                bc.bc_step_sync(step, st.cuda_stream)
                assert_bc_close(d_out.cpu().numpy(), want_a)
            assert G.stats().sources == len(a)
            # the step reads the source buffer at every launch
            with torch.cuda.stream(st):
                d_src.copy_(dev_sources(b))
            bc.bc_step_launch(step, st.cuda_stream)
            bc.bc_step_sync(step, st.cuda_stream)
            assert_bc_close(d_out.cpu().numpy(), oracle.bc(g, b, 0.5))
            # the graph is held while the step exists
            with pytest.raises(bc.BCError) as ei:
                bc.bc_graph_destroy(G.handle)
            assert ei.value.code == bc.BC_ERR_BUSY
        finally:
            bc.bc_step_destroy(step)


def test_two_steps_on_two_streams_and_the_1024_team():
    g1 = gen.rmat_graph(13, 16, wmin=1, wmax=255, seed=81)
    g2 = gen.ba_graph(4000, 4, 1, 1000, seed=82)
    s1 = gen.sample_sources(g1.n, 96, seed=83)
    s2 = gen.sample_sources(g2.n, 96, seed=84)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    bc.bc_set_config(team_threads=1024)
    with bc.Graph(g1) as G1, bc.Graph(g2) as G2:
        outs, steps = [], []
        for G, g, s in ((G1, g1, s1), (G2, g2, s2)):
            d_src = dev_sources(s)
            d_out = torch.empty(g.n, dtype=torch.float64, device="cuda")
            outs.append((d_src, d_out))
            steps.append(bc.bc_step_create(G.handle, d_src.data_ptr(), len(s), 1.0, d_out.data_ptr()))
        try:
            for _ in range(2):
                for step, stn in zip(steps, streams):
                    bc.bc_step_launch(step, stn.cuda_stream)
                for step, stn in zip(steps, streams):
                    bc.bc_step_sync(step, stn.cuda_stream)
                assert_bc_close(outs[0][1].cpu().numpy(), oracle.bc(g1, s1, 1.0))
                assert_bc_close(outs[1][1].cpu().numpy(), oracle.bc(g2, s2, 1.0))
            assert G1.stats().team_threads == 1024
        finally:
            for step in steps:
                bc.bc_step_destroy(step)


def test_bad_source_is_reported_and_the_step_recovers():
    g = gen.er_graph(200, 800, 1, 9, seed=91)
    src = np.arange(0, 200, 5)
    st = torch.cuda.Stream()
    with bc.Graph(g) as G:
        d_src = dev_sources(src)
        d_out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        step = bc.bc_step_create(G.handle, d_src.data_ptr(), len(src), 1.0, d_out.data_ptr())
        try:
            with torch.cuda.stream(st):
                d_src[3] = 200  # out of range
            bc.bc_step_launch(step, st.cuda_stream)
            with pytest.raises(bc.BCError) as ei:
                bc.bc_step_sync(step, st.cuda_stream)
            assert ei.value.code == bc.BC_ERR_INVALID
            with torch.cuda.stream(st):
                d_src[3] = int(src[3])
            bc.bc_step_launch(step, st.cuda_stream)
            bc.bc_step_sync(step, st.cuda_stream)
            assert_bc_close(d_out.cpu().numpy(), oracle.bc(g, src, 1.0))
        finally:
            bc.bc_step_destroy(step)
        # an empty source list gives zeros
        d_out = torch.full((g.n,), 7.0, dtype=torch.float64, device="cuda")
        step = bc.bc_step_create(G.handle, 0, 0, 1.0, d_out.data_ptr())
        try:
            bc.bc_step_launch(step, st.cuda_stream)
            bc.bc_step_sync(step, st.cuda_stream)
            assert np.all(d_out.cpu().numpy() == 0)
        finally:
            bc.bc_step_destroy(step)
        with pytest.raises(bc.BCError):
            bc.bc_step_create(G.handle, d_src.data_ptr(), len(src), 1.0, 0)


def test_python_conveniences_marshal_to_the_same_calls():
    g = gen.er_graph(400, 2000, 1, 30, seed=95)
    src = gen.sample_sources(g.n, 50, seed=96)
    want = oracle.bc(g, src, 0.5)
    st = torch.cuda.Stream()
    with bc.Graph(g) as G:
        d_src = dev_sources(src)
        d_out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        G.compute_async(d_src, d_out, 0.5, stream=st)
        G.sync(st)
        assert_bc_close(d_out.cpu().numpy(), want)
        d_ebc = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
        G.edge_compute_async(d_src, d_ebc, d_out, 0.5, stream=st)
        G.sync(st)
        assert_bc_close(d_ebc.cpu().numpy(), oracle.edge_bc(g, src, 0.5))
        with G.step(d_src, d_out, 0.5) as step:
            for _ in range(2):
                step.launch(st)
            step.sync(st)
            assert_bc_close(d_out.cpu().numpy(), want)
        reqs = [G.submit(src, 0.5) for _ in range(3)]
        for r in reqs:
            assert_bc_close(r.result(), want)
            assert_bc_close(r.result(), want)  # a second call returns the same array
