"""Benchmark: weighted betweenness centrality, GTEPS and HBM roofline.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat20|ba65k|grid1024|er1k]
                [--impl ours|reference] [--no-cpu-baseline] [--plain-sample S]

One step = one batched BC run over the workload's whole source list (every
step of the hot path: SSSP in strict settle batches, sigma, the backward
dependency pass into BC), inputs resident in HBM.  GTEPS = sources x
undirected edges / second (whole job: summed over ranks, weak scaling, one
independent replica of the problem per GPU, no collective on the data path).
Rank 0 prints one JSON line.  --impl reference times the CPU oracle instead
(the reference arm of this tier), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1701_05975_gb300 import gen  # noqa: E402

WORKLOADS = {
    "serving": ("serving stream: Poisson arrivals over 15 graphs {ER avg deg 16, BA 4/vertex, perturbed grid} x "
                "n in {1k, 4k, 16k, 65k, 262k}, weights U[1,1000]; exact BC for n <= 16k, else 256 sampled sources",
                None),
    "ablation": ("the paper's thread mappings (node-parallel / work-efficient x 1-32 threads per vertex) "
                 "against the batched kernel on ER and Kronecker sweeps shaped like Fig. 4-5, weights U[1,10]",
                 None),
    "rmat20": ("R-MAT scale 20, edge factor 16, a=.57 b=.19 c=.19, symmetrised, weights U[1,255], "
               "4096 uniform sources, scale 0.5 n/k", gen.workload_rmat20),
    "ba65k": ("Barabasi-Albert n=65536, 4 edges per new vertex, weights U[1,1000], all sources, scale 0.5",
              gen.workload_ba65k),
    "grid1024": ("perturbed 1024x1024 4-neighbour grid, 5% edges removed, weights U[1,10000], 1024 sources",
                 gen.workload_grid1024),
    "er1k": ("Erdos-Renyi G(1024, 8192), weights U[1,100], all sources, scale 0.5", gen.workload_er1k),
    "rmat20-edge": ("edge BC (and vertex BC) on R-MAT scale 20, edge factor 16, a=.57 b=.19 c=.19, symmetrised, "
                    "weights U[1,255], 4096 uniform sources, scale 0.5 n/k", gen.workload_rmat20),
    "rmat20-directed": ("directed R-MAT scale 20, edge factor 16, a=.57 b=.19 c=.19, weights U[1,255], "
                        "4096 uniform sources, ordered pairs, scale n/k", gen.workload_rmat20_directed),
    "grid1024-delta": ("perturbed 1024x1024 4-neighbour grid, 5% edges removed, weights U[1,10000], 1024 sources, "
                       "delta-stepping schedule with DAG hop-depth levels", gen.workload_grid1024),
}

# per-workload options: edge output, directed graph, per-source schedule
WORKLOAD_OPTS = {"rmat20-edge": {"edge": True}, "rmat20-directed": {"directed": True},
                 "grid1024-delta": {"algorithm": 2}}


def oracle_fn(opts):
    """The oracle form for a workload: (callable(g, sources, scale) -> BC, threads it uses per call)."""
    import oracle

    if opts.get("directed"):
        return oracle.bc_directed, 1
    if opts.get("edge"):
        return oracle.edge_bc, 1
    return None, 0


def timing_oracle():
    """The oracle's C source built for timing (-O3, the host's instruction
    set): (library, flags)."""
    import oracle

    lib = oracle.timing_lib()
    return lib, " ".join(oracle.TIMING_FLAGS)


def run_oracle(g, sources, scale, opts, cores):
    """The oracle as it stands over `sources`; single-threaded forms run one
    source chunk per host core (ctypes releases the GIL during each call)."""
    import oracle

    lib, _ = timing_oracle()
    fn, _ = oracle_fn(opts)
    if fn is None:
        return oracle.bc(g, sources, scale, nthreads=cores, lib=lib)
    import concurrent.futures

    chunks = [c for c in np.array_split(np.asarray(sources), cores) if len(c)]
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(chunks)) as ex:
        parts = list(ex.map(lambda c: fn(g, c, scale, lib=lib), chunks))
    return np.sum(parts, axis=0)


def edge_units(g, opts):
    """Edges per source for TEPS: undirected edges, or directed edges."""
    return g.nnz if opts.get("directed") else g.m

# Algorithmic bytes per unit (the three-pass byte model of the method):
# per CSR entry of a reached vertex 64 B (relax 16 + sigma 24 + backward 24),
# per reached vertex 80 B.
BYTES_PER_ENTRY = 64
BYTES_PER_VERTEX = 80
KERNEL_SRC = os.path.join(ROOT, "paper_1701_05975_gb300", "csrc", "bc_batched.cuh")


def reach_model(g, sources, directed=False, sample=32):
    """Per-source reached vertices and reached CSR entries (component sizes;
    for directed graphs the mean out-reach of a sample of the sources)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order, connected_components

    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr).astype(np.int64))
    mat = sp.csr_matrix((np.ones(len(rows), np.int8), (rows, g.col.astype(np.int64))), shape=(g.n, g.n))
    if directed:
        # out-entries of the reached vertices carry the relaxation (16 B) and
        # the backward pass (24 B), their in-entries the sigma pull (24 B):
        # returned as 64-byte-equivalent entries
        deg = np.diff(g.row_ptr).astype(np.float64)
        indeg = np.bincount(g.col.astype(np.int64), minlength=g.n).astype(np.float64)
        rn, re_ = [], []
        for s in np.asarray(sources)[:: max(1, len(sources) // sample)][:sample]:
            order = breadth_first_order(mat, int(s), directed=True, return_predecessors=False)
            rn.append(len(order))
            re_.append((40.0 * deg[order].sum() + 24.0 * indeg[order].sum()) / BYTES_PER_ENTRY)
        k = len(sources)
        return np.full(k, np.mean(rn)), np.full(k, np.mean(re_))
    _, lab = connected_components(mat, directed=False)
    comp_n = np.bincount(lab)
    comp_e = np.bincount(lab, weights=np.diff(g.row_ptr).astype(np.float64))
    ls = lab[sources.astype(np.int64)]
    return comp_n[ls].astype(np.float64), comp_e[ls]


def kernel_digest():
    return hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]


def load_traffic(workload):
    """DRAM bytes per launch of the batched kernel from the committed ncu
    summary, or None when the summary is missing or the kernel changed since."""
    path = os.path.join(ROOT, "profiles", f"bc_batched_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"kernel_sha256_16:\s*([0-9a-f]{16})", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_digest():
        return None
    return float(t.group(1))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, keep_path=None):
        """Samples go to a temporary file; `keep_path` (optional) keeps the raw CSV."""
        self.gpu = gpu_index
        self.proc = None
        self.keep_path = keep_path
        fd, self.path = tempfile.mkstemp(prefix=f"clocks_rank{gpu_index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            if os.path.exists(self.path):
                os.unlink(self.path)
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if self.keep_path:
            os.makedirs(os.path.dirname(os.path.abspath(self.keep_path)), exist_ok=True)
            shutil.copyfile(self.path, self.keep_path)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Replicas:
    """Host-side coordination of N replicas (one process per GPU, launched by
    torchrun).  Sources are independent, so there is no collective on the
    data path: a barrier brackets each timed region and the slowest rank's
    time is the job's time.  `dist` is torch.distributed after
    init_process_group (nccl on GPUs, gloo in the CPU tests) or None."""

    def __init__(self, dist=None, device=None):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, x: float) -> float:
        if self.dist is None:
            return x
        import torch

        t = torch.tensor([x], device=self.device, dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def whole_job_gteps(ws: int, k: int, m: int, seconds: float) -> float:
    """Units every rank processed (each replica runs all k sources) over the slowest rank's time."""
    return ws * k * m / seconds / 1e9


def emit(line: dict, rank: int):
    """Only rank 0 prints the JSON line."""
    if rank == 0:
        print(json.dumps(line), flush=True)


def cpu_baseline(g, sources, opts=None, seconds_target=15.0, max_sample=4096):
    """Time the CPU oracle (as it stands) on a bounded prefix of the source list."""
    opts = opts or {}
    cores = os.cpu_count() or 1
    m = edge_units(g, opts)
    # probe a small prefix to size the sample
    k = min(len(sources), max(cores, 8))
    t0 = time.perf_counter()
    run_oracle(g, sources[:k], 1.0, opts, cores)
    dt = time.perf_counter() - t0
    if dt < seconds_target / 4 and k < len(sources):
        k2 = int(min(len(sources), max_sample, k * max(1.0, (seconds_target / max(dt, 1e-3)) * 0.8)))
        if k2 > k:
            k = k2
            t0 = time.perf_counter()
            run_oracle(g, sources[:k], 1.0, opts, cores)
            dt = time.perf_counter() - t0
    # one core as well (the paper's speedups are over one CPU core): about
    # eight seconds, at least four sources, spread evenly over the same prefix
    # so the mix of large and small reaches matches the all-cores sample
    k1 = max(min(4, k), min(k, int(k * 8.0 / max(dt * cores, 1e-3))))
    pick = np.asarray(sources[:k])[np.linspace(0, k - 1, k1).round().astype(np.int64)]
    t1 = time.perf_counter()
    run_oracle(g, pick, 1.0, opts, 1)
    dt1 = time.perf_counter() - t1
    return {"value": k * m / dt / 1e9, "unit": "GTEPS", "cores": cores, "kind": "oracle",
            "sample": f"first {k} of {len(sources)} sources of the same workload, {dt:.2f} s, "
                      f"{cores} host threads, oracle built with gcc {timing_oracle()[1]}",
            "single_core": {"value": k1 * m / dt1 / 1e9, "unit": "GTEPS",
                            "sample": f"{k1} sources spread over the first {k}, {dt1:.2f} s, one thread"}}


def cycle_shares(st):
    """Fractions of the batched kernel's per-source SM cycles spent in each
    section (expansion, refills, threshold + settle, backward)."""
    parts = {"expand": st.cycles_expand, "refill": st.cycles_refill, "settle": st.cycles_settle,
             "backward": st.cycles_backward}
    total = sum(parts.values())
    return {k: round(v / total, 4) for k, v in parts.items()} if total else None


def metric_name(opts):
    return ("weighted-BC GTEPS (sources x directed edges / s)" if opts.get("directed")
            else "weighted-BC GTEPS (sources x undirected edges / s)")


def run_reference(args, g, sources, scale, desc, opts=None):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    opts = opts or {}
    cores = os.cpu_count() or 1
    m = edge_units(g, opts)
    # bounded sample per step: sized so the whole run stays within minutes
    k = min(len(sources), max(cores, 16))
    t0 = time.perf_counter()
    run_oracle(g, sources[:k], scale, opts, cores)
    probe = time.perf_counter() - t0
    budget_per_step = 150.0 / max(args.steps + args.warmup, 1)
    if probe < budget_per_step / 2:
        k = int(min(len(sources), k * max(1.0, 0.8 * budget_per_step / max(probe, 1e-3))))
    for _ in range(args.warmup):
        run_oracle(g, sources[:k], scale, opts, cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        run_oracle(g, sources[:k], scale, opts, cores)
        times.append(time.perf_counter() - t0)
    t = max(statistics.mean(times), 1e-9)
    value = k * m / t / 1e9
    line = {
        "impl": "reference", "metric": metric_name(opts), "value": value,
        "unit": "GTEPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "n": g.n, "m": m, "sources_per_step": k, "sources_in_workload": len(sources)},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": cores, "kind": "oracle",
                         "sample": f"first {k} of {len(sources)} sources per step, oracle built with gcc "
                                   f"{timing_oracle()[1]}"},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def ablation_graphs():
    """ER and Kronecker graphs shaped like the paper's Fig. 4(a-d) and Fig. 5(c, d)
    (sizes, average degrees), weights uniform in [1, 10] as in its Sec. 4.1."""
    out = []
    for lg in (14, 16, 18):  # Fig. 4(a, b): average degree 32
        out.append((f"ER n=2^{lg} deg 32", gen.er_graph(1 << lg, 16 << lg, 1, 10, seed=0)))
        out.append((f"Kronecker 2^{lg} ef 16", gen.rmat_graph(lg, 16, wmin=1, wmax=10, seed=0)))
    for deg in (4, 16, 64):  # Fig. 4(c, d): degree sweeps
        out.append((f"ER n=20000 deg {deg}", gen.er_graph(20000, 10000 * deg, 1, 10, seed=0)))
        out.append((f"Kronecker 2^15 ef {deg // 2}", gen.rmat_graph(15, deg // 2, wmin=1, wmax=10, seed=0)))
    out.append(("ER n=2^17 deg 4", gen.er_graph(1 << 17, 2 << 17, 1, 10, seed=0)))  # Fig. 5(c)
    out.append(("Kronecker 2^17 ef 2", gen.rmat_graph(17, 2, wmin=1, wmax=10, seed=0)))  # Fig. 5(d)
    return out


def run_ablation(args, desc):
    """Per graph: each paper mapping and the batched kernel on the same sampled
    sources; one JSON line per graph (seconds per source, phases per source =
    the average search depth of Fig. 4(e))."""
    import torch

    import paper_1701_05975_gb300 as bc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    k = args.sources or 4
    rows = []
    for name, g in ablation_graphs():
        deg = g.degrees()
        cand = np.flatnonzero(deg > 0)
        src = np.sort(np.random.default_rng(0).choice(cand, size=min(k, len(cand)), replace=False)).astype(np.uint32)
        res = {"graph": name, "n": g.n, "m": g.m, "sources": len(src)}
        with bc.Graph(g) as G:
            ref = None
            for npar in (True, False):
                for vw in (1, 4, 8, 16, 32):
                    G.compute_paper_variant(src[:1], 1.0, node_parallel=npar, vwarp=vw)  # warm
                    t0 = time.perf_counter()
                    out = G.compute_paper_variant(src, 1.0, node_parallel=npar, vwarp=vw)
                    dt = (time.perf_counter() - t0) / len(src)
                    st = G.stats()
                    res[f"{'np' if npar else 'we'}{vw}_ms_per_source"] = dt * 1e3
                    res["depth_per_source"] = st.phases / max(st.sources, 1)
                    if ref is None:
                        ref = out.copy()
                    assert np.allclose(out, ref, rtol=1e-9, atol=0)
            G.compute(src[:1], 1.0)
            t0 = time.perf_counter()
            out = G.compute(src, 1.0)
            res["batched_ms_per_source_few"] = (time.perf_counter() - t0) / len(src) * 1e3
            assert np.allclose(out, ref, rtol=1e-9, atol=0)
            many = np.arange(0, g.n, max(1, g.n // 2048), dtype=np.uint32)
            t0 = time.perf_counter()
            G.compute(many, 1.0)
            res["batched_ms_per_source_2048"] = (time.perf_counter() - t0) / len(many) * 1e3
        keys = [kk for kk in res if kk.endswith("_ms_per_source")]
        res["best_paper_mapping"] = min(keys, key=lambda kk: res[kk]).replace("_ms_per_source", "")
        rows.append(res)
        if rank == 0:
            print(json.dumps(res), flush=True)
    if rank == 0:
        we_better = sum(1 for r in rows if min(r[f"we{v}_ms_per_source"] for v in (1, 4, 8, 16, 32))
                        <= min(r[f"np{v}_ms_per_source"] for v in (1, 4, 8, 16, 32)))
        print(json.dumps({"metric": "ablation summary", "graphs": len(rows),
                          "work_efficient_beats_node_parallel": we_better, "workload": desc}), flush=True)


def run_serving_reference(args, desc):
    """The oracle over a bounded prefix of the same request stream."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    cores = os.cpu_count() or 1
    reqs = gen.serving_requests(num=args.requests, rate_per_s=1.0, seed=0)
    pool = {}
    done, edges, t_total = 0, 0, 0.0
    for r in reqs:
        if t_total > 120.0:
            break
        key = (r.kind, r.n)
        if key not in pool:
            pool[key] = gen.serving_graph(r.kind, r.n, seed=0)
        g = pool[key]
        t0 = time.perf_counter()
        oracle.bc(g, r.sources, r.scale, nthreads=cores, lib=timing_oracle()[0])
        t_total += time.perf_counter() - t0
        done += 1
        edges += len(r.sources) * g.m
    value = edges / t_total / 1e9
    line = {"impl": "reference", "metric": "serving: aggregate GTEPS and p50/p99 latency (submit -> done)",
            "value": value, "unit": "GTEPS", "n_gpus": args.gpus, "steps": 1, "warmup": 0,
            "ms_per_step": t_total * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {"workload": desc, "requests_timed": done},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": cores, "kind": "oracle",
                             "sample": f"first {done} of {len(reqs)} requests, run back to back, oracle built "
                                       f"with gcc {timing_oracle()[1]}"},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serving_measure(args):
    """The serving stream: saturated throughput first (a burst of requests),
    then the Poisson stream at 0.7 of it; p50/p99 from submit to done.
    Returns the measurement as a dict (one rank's view)."""
    import paper_1701_05975_gb300 as bc

    pool = {}
    for kind in gen.SERVING_KINDS:
        for n in gen.SERVING_SIZES:
            pool[(kind, n)] = gen.serving_graph(kind, n, seed=0)
    graphs = {key: bc.Graph(g) for key, g in pool.items()}
    reqs = gen.serving_requests(num=args.requests, rate_per_s=1.0, seed=0)

    def run_stream(batch, rate):
        bc.bc_serving_reset()
        outs, ids = [], []
        t_start = time.perf_counter()
        for i, r in enumerate(batch):
            if rate is not None:
                due = t_start + r.arrival_s / rate
                while True:
                    now = time.perf_counter()
                    if now >= due:
                        break
                    time.sleep(min(due - now, 0.002))
            out = np.empty(r.n, np.float64)
            outs.append(out)
            ids.append(bc.bc_request_submit(graphs[(r.kind, r.n)].handle, r.sources, r.scale, out))
        for rid in ids:
            bc.bc_request_wait(rid, -1)
        makespan = time.perf_counter() - t_start
        return makespan, bc.bc_serving_stats_get()

    try:
        # warm-up: one request per graph (workspace allocation)
        warm = [gen.ServingRequest(0.0, k, n, np.arange(min(n, 64), dtype=np.uint32), 1.0) for (k, n) in pool]
        run_stream(warm, None)
        burst = reqs[: min(200, len(reqs))]
        mk_sat, _ = run_stream(burst, None)
        sat_rate = len(burst) / mk_sat
        rate = 0.7 * sat_rate
        makespan, st = run_stream(reqs, rate)
        edges = sum(len(r.sources) * pool[(r.kind, r.n)].m for r in reqs)
        gteps = edges / makespan / 1e9
        # optional load sweep: shorter streams (the first --sweep-requests
        # requests) at other fractions of the saturated rate
        sweep = []
        for load in ([float(x) for x in args.sweep.split(",")] if args.sweep else []):
            sub = reqs[: args.sweep_requests]
            mk, sst = run_stream(sub, load * sat_rate)
            e = sum(len(r.sources) * pool[(r.kind, r.n)].m for r in sub)
            sweep.append({"load": load, "requests": len(sub), "gteps": e / mk / 1e9, "p50_ms": sst.p50_ms,
                          "p99_ms": sst.p99_ms, "mean_ms": sst.mean_ms})
    finally:
        for G in graphs.values():
            G.close()
    return {"gteps": gteps, "makespan_s": makespan, "requests": len(reqs), "arrival_rate_per_s": rate,
            "saturated_rate_per_s": sat_rate, "load": 0.7,
            "latency_ms": {"p50": st.p50_ms, "p99": st.p99_ms, "mean": st.mean_ms},
            "completed": int(st.completed), "failed": int(st.failed), "max_concurrent": int(st.max_concurrent),
            "sweep": sweep,
            "h2d_bytes": int(sum(4 * len(r.sources) for r in reqs)),
            "d2h_bytes": int(sum(8 * r.n for r in reqs))}


def run_serving(args, desc):
    """Serving workload as the headline of its own line."""
    ws, rank, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    sv = serving_measure(args)
    line = {
        "metric": "serving: aggregate GTEPS and p50/p99 latency (submit -> done)", "value": sv["gteps"],
        "unit": "GTEPS", "n_gpus": ws, "steps": 1, "warmup": 1, "ms_per_step": sv["makespan_s"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "requests": sv["requests"], "arrival_rate_per_s": sv["arrival_rate_per_s"],
                   "saturated_rate_per_s": sv["saturated_rate_per_s"], "load": sv["load"]},
        "latency_ms": sv["latency_ms"], "completed": sv["completed"], "failed": sv["failed"],
        "max_concurrent": sv["max_concurrent"], "sweep": sv["sweep"],
        "e2e": {"value": sv["gteps"], "unit": "GTEPS", "h2d_bytes_per_step": sv["h2d_bytes"],
                "d2h_bytes_per_step": sv["d2h_bytes"]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat20", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-sample", type=int, default=16,
                    help="also time the plain one-source-at-a-time form on this many sources (0: skip)")
    ap.add_argument("--autotune", type=int, default=-1,
                    help="probe sources for the autotuner (-1: automatic size, 0: off)")
    ap.add_argument("--requests", type=int, default=2000, help="serving workload: number of requests")
    ap.add_argument("--sweep", default="", help="serving workload: extra loads, e.g. 0.3,0.5,0.9 (default: none)")
    ap.add_argument("--sweep-requests", type=int, default=300, help="serving workload: requests per sweep load")
    ap.add_argument("--sources", type=int, default=0,
                    help="use only the first K sources of the workload (small profiling cases); 0 = all")
    ap.add_argument("--max-slots", type=int, default=0, help="cap on sources in flight (0 = automatic)")
    ap.add_argument("--team", type=int, default=0, help="threads per source (0 = automatic / autotuned)")
    ap.add_argument("--width", type=int, default=0, help="near/far split width (0 = automatic / autotuned)")
    ap.add_argument("--algorithm", type=int, default=0, help="per-source schedule: 0 = automatic / autotuned, "
                    "1 = strict, 2 = delta-stepping")
    ap.add_argument("--warp-degree", type=int, default=0, help="rows with at least this many entries get a warp "
                    "(0 = automatic / autotuned)")
    ap.add_argument("--team-degree", type=int, default=0, help="rows with at least this many entries get the whole "
                    "team (0 = automatic / autotuned)")
    ap.add_argument("--settle-in", type=int, default=0, help="settle test: 1 = OUT or IN with the settled-neighbour "
                    "bound, 2 = OUT, 3 = OUT or IN (0 = automatic / autotuned)")
    ap.add_argument("--clocks-csv", default="", help="also keep the raw nvidia-smi clock samples at this path "
                    "({rank} is replaced by the rank)")
    ap.add_argument("--no-graph", action="store_true", help="enqueue each step with bc_compute_async instead of "
                    "replaying a captured step graph")
    ap.add_argument("--no-serving", action="store_true", help="leave the serving stream (p50/p99 latency, aggregate "
                    "GTEPS over 2000 requests) out of a single-GPU line of the other workloads")
    args = ap.parse_args()

    desc, maker = WORKLOADS[args.workload]
    if args.impl == "reference" or not args.no_cpu_baseline:
        timing_oracle()  # compile the timing build of the oracle before any GPU work
    if args.workload == "ablation":
        run_ablation(args, desc)
        return
    if args.workload == "serving":
        if args.impl == "reference":
            run_serving_reference(args, desc)
        else:
            run_serving(args, desc)
        return
    opts = WORKLOAD_OPTS.get(args.workload, {})
    g, sources, scale = maker()
    if args.sources:
        scale = scale * len(sources) / min(args.sources, len(sources))
        sources = sources[: args.sources]
    m = edge_units(g, opts)
    edge = bool(opts.get("edge"))

    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, g, sources, scale, desc, opts)
        return

    import torch

    import paper_1701_05975_gb300 as bc

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    dev = torch.device("cuda", local)
    ranks = Replicas(dist, dev)
    barrier = ranks.barrier
    if args.max_slots:
        bc.bc_set_config(max_slots=args.max_slots)
    if args.team:
        bc.bc_set_config(team_threads=args.team)
    if args.width:
        bc.bc_set_config(bucket_width=args.width)
    if opts.get("algorithm") or args.algorithm:
        bc.bc_set_config(algorithm=args.algorithm or opts["algorithm"])
    if args.warp_degree or args.team_degree:
        bc.bc_set_config(warp_degree=args.warp_degree, team_degree=args.team_degree)
    if args.settle_in:
        bc.bc_set_config(settle_in=args.settle_in)
    t0 = time.perf_counter()
    G = bc.Graph(g, flags=bc.BC_DIRECTED if opts.get("directed") else 0)
    prep_s = time.perf_counter() - t0  # graph prep: validation, relabeling, upload, packing, Delta_node
    probe = args.autotune if args.autotune >= 0 else min(len(sources), 2048)
    tune_s = 0.0
    if probe:
        t0 = time.perf_counter()
        G.autotune(sources[:probe])
        tune_s = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=dev)
    d_src = torch.from_numpy(sources.astype(np.int32)).to(dev)
    d_out = torch.empty(g.n, dtype=torch.float64, device=dev)
    d_ebc = torch.empty(g.nnz, dtype=torch.float64, device=dev) if edge else None
    k = len(sources)

    # a step is one batched run over all sources, captured once as a CUDA
    # graph (bc_step_create) and replayed; --no-graph enqueues it call by call
    # (edge output always does)
    use_graph = not args.no_graph and not edge
    step_h = bc.bc_step_create(G.handle, d_src.data_ptr(), k, scale, d_out.data_ptr()) if use_graph else None

    def step():
        if step_h is not None:
            bc.bc_step_launch(step_h, stream.cuda_stream)
        elif edge:
            bc.bc_edge_compute_async(G.handle, d_src.data_ptr(), k, scale, d_ebc.data_ptr(), d_out.data_ptr(),
                                     stream.cuda_stream)
        else:
            bc.bc_compute_async(G.handle, d_src.data_ptr(), k, scale, d_out.data_ptr(), stream.cuda_stream)

    def sync_status():
        if step_h is not None:
            bc.bc_step_sync(step_h, stream.cuda_stream)
        else:
            bc.bc_sync_status(G.handle, stream.cuda_stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        sync_status()
    st = G.stats()
    barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local, args.clocks_csv.replace("{rank}", str(rank)) if args.clocks_csv else None)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        t_end.record(stream)
    torch.cuda.synchronize(dev)
    sync_status()
    barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = ranks.max_over_ranks(total_ms / args.steps)
    value = whole_job_gteps(ws, k, m, ms_step * 1e-3)

    # end to end through the public synchronous call: host sources in, host BC out
    host_out = np.empty(g.n, np.float64)
    host_ebc = np.empty(g.nnz, np.float64) if edge else None
    e2e_times = []
    for i in range(max(1, min(args.steps, 3)) + 1):
        barrier()
        t0 = time.perf_counter()
        if edge:
            bc.bc_edge_compute(G.handle, sources, scale, host_ebc, host_out)
        else:
            bc.bc_compute(G.handle, sources, scale, host_out)
        dt = time.perf_counter() - t0
        if i > 0:
            e2e_times.append(dt)
    e2e_s = ranks.max_over_ranks(statistics.mean(e2e_times))

    # roofline of the dominant kernel (the batched kernel is > 99% of a step)
    rn, re_ = reach_model(g, sources, directed=bool(opts.get("directed")))
    alg_bytes = float(BYTES_PER_ENTRY * re_.sum() + BYTES_PER_VERTEX * rn.sum())
    launch_avg_s = statistics.mean(launch_ms) * 1e-3
    achieved = alg_bytes / launch_avg_s / 1e9
    peak, peak_kind = peaks()
    traffic = load_traffic(args.workload)

    line = {
        "metric": metric_name(opts),
        "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "n": g.n, "m": m, "nnz": g.nnz, "sources": k, "scale": scale,
                   "l2": "inputs larger than L2: graph %.0f MB + %d per-source slabs of %.1f MB"
                         % (G.info().device_bytes / 1e6, int(st.slots), G.info().slab_bytes / 1e6),
                   "team_threads": int(st.team_threads), "slots": int(st.slots),
                   "bucket_width": int(st.bucket_width), "warp_degree": int(st.warp_degree),
                   "team_degree": int(st.team_degree),
                   "settle_test": {1: "OUT or IN, settled-neighbour bound", 2: "OUT (Eq. 2 + Eq. 4)",
                                   3: "OUT or IN"}.get(int(st.settle_in), "n/a"),
                   "parallelism": f"replicas x{ws}",
                   "autotune": {"probe_sources": probe, "seconds": round(tune_s, 2)},
                   "graph_prep_s": round(prep_s, 3),
                   "launch": "CUDA graph (bc_step_launch)" if use_graph else (
                       "bc_edge_compute_async per step" if edge else "bc_compute_async per step"),
                   "algorithm": "delta-stepping" if int(st.algorithm) == 2 else "strict",
                   "relabeled_by_degree": bool(G.info().relabeled), "dist_bits": int(G.info().dist_bits)},
        "e2e": {"value": whole_job_gteps(ws, k, m, e2e_s), "unit": "GTEPS", "h2d_bytes_per_step": 4 * k,
                "d2h_bytes_per_step": 8 * g.n + (8 * g.nnz if edge else 0)},
        # per step: source check, the batched kernel, then one scale pass per output when scale != 1
        "gpu_launches": (2 + (scale != 1.0) * (2 if edge else 1)) * args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     # ncu-measured DRAM bytes per launch over the same launch time
                     "frac_measured": (traffic / launch_avg_s / 1e9 / peak) if traffic else None,
                     "alg_bytes_per_launch": alg_bytes, "kernel": "bc_batched_kernel"},
        "clocks": clk,
        "run_stats": {"phases_per_source": st.phases / max(st.sources, 1),
                      "refills_per_source": st.refills / max(st.sources, 1),
                      "reached_per_source": st.reached / max(st.sources, 1),
                      "near_entries_scanned_per_source": st.near_scanned / max(st.sources, 1),
                      "far_entries_scanned_per_source": st.far_scanned / max(st.sources, 1),
                      # share of each source's SM cycles (team leader's clock) per section
                      "cycle_shares": cycle_shares(st)},
    }
    if args.plain_sample and rank == 0 and not edge and not opts.get("directed"):
        sub = sources[: args.plain_sample]
        c0 = bc.bc_get_config()
        bc.bc_set_config(mode=bc.BC_MODE_PLAIN)
        out = np.empty(g.n, np.float64)
        bc.bc_compute(G.handle, sub[:2], scale, out)
        t0 = time.perf_counter()
        bc.bc_compute(G.handle, sub, scale, out)
        dt = time.perf_counter() - t0
        bc.bc_set_config(c0)
        line["plain"] = {"value": len(sub) * m / dt / 1e9, "unit": "GTEPS", "sources": len(sub)}
    if step_h is not None:
        bc.bc_step_destroy(step_h)
        step_h = None
    G.close()
    if ws == 1 and not args.no_serving and args.workload == "rmat20":
        # the serving half of the metric (p50/p99 latency, aggregate GTEPS),
        # measured after the batched workload's graph and workspaces are freed;
        # a failure there is reported in the line instead of losing the line
        try:
            sv = serving_measure(args)
            line["serving"] = {"workload": WORKLOADS["serving"][0], "gteps": sv["gteps"], "unit": "GTEPS",
                               "latency_ms": sv["latency_ms"], "requests": sv["requests"], "load": sv["load"],
                               "arrival_rate_per_s": sv["arrival_rate_per_s"],
                               "saturated_rate_per_s": sv["saturated_rate_per_s"], "completed": sv["completed"],
                               "failed": sv["failed"], "max_concurrent": sv["max_concurrent"]}
        except Exception as exc:  # noqa: BLE001 - any failure of the serving half is reported as such
            line["serving"] = {"workload": WORKLOADS["serving"][0], "error": f"{type(exc).__name__}: {exc}"}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, sources, opts)
    emit(line, rank)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
