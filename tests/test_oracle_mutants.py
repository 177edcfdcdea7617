"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake (a dropped term, a wrong comparison, a transposed
operand, a wrong index) in a copy of oracle/brandes.c, builds it on the CPU and
checks that at least one pin in test_oracle_pins fails against it.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins
from paper_1701_05975_gb300 import gen

SRC = os.path.join(os.path.dirname(oracle.__file__), "brandes.c")

MUTANTS = {
    "dropped_one_plus": ("wk->sigma[p] / wk->sigma[x] * (1.0 + wk->delta[x])", "wk->sigma[p] / wk->sigma[x] * (wk->delta[x])"),
    "transposed_sigma_ratio": ("wk->sigma[p] / wk->sigma[x] * (1.0 + wk->delta[x])", "wk->sigma[x] / wk->sigma[p] * (1.0 + wk->delta[x])"),
    "ties_reset_sigma": ("if (alt < wk->d[x]) {\n        /* strictly", "if (alt <= wk->d[x]) {\n        /* strictly"),
    "sigma_not_summed": ("wk->sigma[x] += wk->sigma[u];", "wk->sigma[x] = wk->sigma[u];"),
    "source_counted": ("if (x != s) acc[x] += wk->delta[x];", "acc[x] += wk->delta[x];"),
    "scale_dropped": ("out_bc[v] = scale * sum;", "out_bc[v] = sum;"),
    "wrong_relax_weight": ("uint64_t alt = wk->d[u] + (uint64_t)w[e];", "uint64_t alt = wk->d[u] + (uint64_t)w[row_ptr[u]];"),
    "phased_nonstrict": ("                           : (U[v] && d[v] < Delta);", "                           : (U[v] && d[v] <= Delta);"),
    "phased_dnode_max": ("if ((uint64_t)w[e] < m) m = w[e];", "if (m == INF_DIST || (uint64_t)w[e] > m) m = w[e];"),
    "edge_share_wrong_dir": ("out_ebc[e] += share;", "out_ebc[e] += share * (wk.d[a] == 0 ? 2.0 : 1.0);"),
    "pull_dropped_one_plus": ("dep += wk.sigma[a] / wk.sigma[b] * (1.0 + wk.delta[b]);",
                              "dep += wk.sigma[a] / wk.sigma[b] * (wk.delta[b]);"),
    "pull_source_counted": ("if (a != s) out_bc[a] += dep;", "out_bc[a] += dep;"),
}


def any_pin_fails(lib) -> bool:
    checks = [
        lambda: [pins.check_against_brute(g, lib=lib) for g in pins.small_graphs(60, seed=41)],
        lambda: [pins.check_against_brute(g, lib=lib) for g in pins.small_graphs(30, seed=42, wmax=9)],
        lambda: _closed_forms(lib),
        lambda: _fig1a(lib),
        lambda: _phased_vs_brandes(lib),
        lambda: _directed(lib),
    ]
    for c in checks:
        try:
            c()
        except AssertionError:
            return True
    return False


def _closed_forms(lib):
    for n in (5, 8):
        g = pins.graph(n, [(i, i + 1, 1 + i % 3) for i in range(n - 1)])
        assert np.array_equal(oracle.bc(g, np.arange(n), 0.5, lib=lib), [i * (n - 1 - i) for i in range(n)])
    g = pins.graph(6, [(i, (i + 1) % 6, 1) for i in range(6)])
    np.testing.assert_allclose(oracle.bc(g, np.arange(6), 0.5, lib=lib), 2.0)


def _fig1a(lib):
    g, s, expects, sigma_strict = pins.load_fig1a()
    for crit, order, want in expects:
        _, sg, _, _, _ = oracle.phased(g, s, nonstrict=(crit == "nonstrict"), reverse=(order == "reverse"), lib=lib)
        assert sg[3] == want


def _directed(lib):
    rng = np.random.default_rng(44)
    for _ in range(30):
        n = int(rng.integers(2, 6))
        g = gen.random_small_digraph(n, 0.5, 1, 3, rng)
        _, _, bc_ref, _ = pins.brute_force(g)
        pins.close(oracle.bc_directed(g, np.arange(n), 1.0, lib=lib), [float(x) for x in bc_ref])


def _phased_vs_brandes(lib):
    for g in [gen.er_graph(60, 200, 1, 6, seed=43), gen.grid_graph(6, 7, wmin=1, wmax=4, seed=44)]:
        for s in (0, 7, 31):
            d, sg, lev, _, _ = oracle.phased(g, s, reverse=True, lib=lib)
            d_b, sg_b, _ = oracle.sssp(g, s, lib=lib)
            assert np.array_equal(d, d_b) and np.array_equal(sg, sg_b)
            rows, cols, ws = g.edges()
            for a, b, w in zip(rows.tolist(), cols.tolist(), ws.tolist()):
                if int(d[a]) + w == int(d[b]):
                    assert lev[a] < lev[b]


def test_unmutated_oracle_passes_subset():
    assert not any_pin_fails(oracle.load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation site for {name} not found"
    mutated = tmp_path / "brandes.c"
    mutated.write_text(text.replace(old, new))
    out = str(tmp_path / "libmutant.so")
    import subprocess

    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", out, str(mutated), "-lpthread"], check=True)
    assert any_pin_fails(oracle.load(out)), f"mutant {name} survived every pin"
