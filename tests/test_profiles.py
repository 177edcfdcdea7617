"""The committed ncu summaries and the benchmark's use of them (CPU only).

bench.py reports the measured DRAM traffic of the batched kernel only while
the summary's recorded kernel source hash equals the current source's; these
tests check that the summaries behind the benchmark workloads describe the
kernel as it stands, and that a changed kernel turns the figure off."""
from __future__ import annotations

import os
import re

import pytest

import bench

PROFILES = os.path.join(bench.ROOT, "profiles")


def _summary(name):
    return open(os.path.join(PROFILES, name)).read()


@pytest.mark.parametrize("workload", ["rmat20", "ba65k", "grid1024"])
def test_kernel_summaries_match_the_current_kernel_source(workload):
    text = _summary(f"bc_batched_{workload}.md")
    m = re.search(r"kernel_sha256_16:\s*([0-9a-f]{16})", text)
    assert m, "summary without a kernel hash"
    assert m.group(1) == bench.kernel_digest()


@pytest.mark.parametrize("workload", ["rmat20", "ba65k"])
def test_benchmark_reads_the_measured_traffic(workload):
    t = bench.load_traffic(workload)
    assert t is not None and t > 0


def test_traffic_is_dropped_once_the_kernel_changes(monkeypatch):
    monkeypatch.setattr(bench, "kernel_digest", lambda: "0" * 16)
    assert bench.load_traffic("rmat20") is None
    assert bench.load_traffic("no-such-workload") is None


def test_summaries_name_only_committed_commands():
    # every capture command runs the committed bench.py (never a working script)
    for name in os.listdir(PROFILES):
        text = _summary(name)
        for line in text.splitlines():
            if line.lstrip().startswith(("python ", "ncu ")):
                assert "_work" not in line and "/root/" not in line, (name, line)
