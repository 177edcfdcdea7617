"""Randomised cross-configuration parity: many small graphs of different
shapes, each under a random configuration (team size, split width, settle
rule, schedule, layout, directed or not, edge output), against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1701_05975_gb300 as bc
from paper_1701_05975_gb300 import gen
from test_gpu_parity import assert_bc_close

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def default_config():
    c0 = bc.bc_get_config()
    yield
    bc.bc_set_config(c0)


def random_graph(rng):
    kind = rng.choice(["small", "er", "ba", "rmat", "grid", "digraph", "rmatd", "big"])
    wmax = int(rng.choice([1, 7, 300, 1 << 20]))
    seed = int(rng.integers(1 << 30))
    if kind == "small":
        n = int(rng.integers(1, 120))
        return gen.random_small_graph(n, float(rng.choice([0.02, 0.1, 0.4])), 1, wmax, rng), False
    if kind == "er":
        n = int(rng.integers(50, 1500))
        return gen.er_graph(n, int(n * rng.integers(1, 8)), 1, wmax, seed=seed), False
    if kind == "ba":
        return gen.ba_graph(int(rng.integers(50, 2000)), int(rng.integers(1, 5)), 1, wmax, seed=seed), False
    if kind == "rmat":
        return gen.rmat_graph(int(rng.integers(6, 11)), 8, wmin=1, wmax=wmax, seed=seed), False
    if kind == "grid":
        r, c = int(rng.integers(2, 30)), int(rng.integers(2, 30))
        return gen.grid_graph(r, c, wmin=1, wmax=wmax, seed=seed), False
    if kind == "digraph":
        n = int(rng.integers(1, 120))
        return gen.random_small_digraph(n, float(rng.choice([0.02, 0.1, 0.3])), 1, wmax, rng), True
    if kind == "rmatd":
        return gen.rmat_digraph(int(rng.integers(6, 11)), 8, wmin=1, wmax=wmax, seed=seed), True
    # a larger graph: several chunks per batch and long queues
    return gen.rmat_graph(13, 16, wmin=1, wmax=int(rng.choice([3, 255])), seed=seed), False


@pytest.mark.parametrize("seed", [20261203, 7, 99])
def test_random_graphs_random_configurations(seed):
    rng = np.random.default_rng(seed)
    for it in range(150):
        g, directed = random_graph(rng)
        cfg = dict(team_threads=int(rng.choice([32, 128, 256, 512, 1024])),
                   bucket_width=int(rng.choice([0, 1, 5, 100, 1 << 30])),
                   settle_in=int(rng.choice([1, 2, 3])),
                   algorithm=int(rng.choice([1, 1, 2])),
                   max_slots=int(rng.choice([0, 0, 1, 7])))
        bc.bc_set_config(**cfg)
        flags = (bc.BC_DIRECTED if directed else 0) | int(rng.choice([0, bc.BC_RELABEL_DEGREE, bc.BC_KEEP_ORDER]))
        k = int(rng.integers(0, min(g.n, 64) + 1))
        src = rng.choice(g.n, size=k, replace=bool(rng.integers(2))).astype(np.uint32) if k else np.zeros(0, np.uint32)
        scale = float(rng.choice([1.0, 0.5, 3.25]))
        want = (oracle.bc_directed if directed else oracle.bc)(g, src, scale)
        ctx = f"iteration {it}: n={g.n} nnz={g.nnz} directed={directed} flags={flags} cfg={cfg} k={k}"
        with bc.Graph(g, flags=flags) as G:
            try:
                assert_bc_close(G.compute(src, scale), want)
                if it % 3 == 0:
                    ebc, vbc = G.edge_compute(src, scale)
                    assert_bc_close(ebc, oracle.edge_bc(g, src, scale))
                    assert_bc_close(vbc, want)
            except (AssertionError, bc.BCError) as e:
                raise AssertionError(f"{ctx}: {e}") from None
