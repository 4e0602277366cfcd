#!/usr/bin/env python3
"""Benchmark of the cover-edge triangle count (CETC) on GB300.

One step = one pass of the whole cover-edge path over one graph resident in
HBM: graph ingest (checks, long-row chunks, max-degree root), BFS levels,
cover-edge extraction, intersection with the count-once rule, reduction to a
uint64.
Workload (default): R-MAT scale 22, edgefactor 16, Graph500 a/b/c/d,
edge seed 2, relabelled (Fisher-Yates stream 2 + 2^32), symmetrised and
de-duplicated.  Metric: undirected edges |E| / step time (edges/s).

Also measured in the same run:
  * the plain direction-oriented all-edge count (same GPU, same inputs);
  * end to end through the C ABI with pinned HOST buffers (H2D copy of the
    CSR and D2H of the count inside the timed region);
  * the intersection kernel's duration (CUDA events on its stream) against
    the HBM roofline, with algorithmic bytes per launch = 4 B per list
    element the kernel must stream (level segments of both endpoints,
    counted by the kernel) + 72 B of per-edge metadata;
  * the CPU oracle on a bounded sample of the same workload (rank 0, N=1).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun the ranks count ONE graph together by default (--shard):
each rank counts a work-balanced slice of the cover edges and the slice
counts are summed by one int64 all-reduce (strong scaling); with
--no-shard every rank counts its own graph of the same recipe (weak
scaling, no collective on the data path).

The default single-GPU line also carries the batched (4,096 mixed graphs)
and serving (resident R-MAT scale 26 + a Poisson request stream)
configurations of the same metric, and the CPU oracle measured in full on
all host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cover-edge TC edges/s, % HBM roofline vs plain all-edge GPU TC; serve p50/p99"
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 129 * 1024 * 1024
INTERSECT_SOURCE = os.path.join(ROOT, "paper_2210_00389_gb300", "csrc", "hashsect.cu")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat22",
                    choices=["rmat22", "rmat10", "rmat18", "rmat20", "rmat26", "chunglu23",
                             "batch", "serve", "kstudy"])
    ap.add_argument("--kstudy-max-scale", type=int, default=26,
                    help="kstudy: largest R-MAT scale (from 6)")
    ap.add_argument("--requests", type=int, default=20000, help="serve: stream length")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: offered requests/s")
    ap.add_argument("--serve-scale", type=int, default=26, help="serve: resident R-MAT scale")
    ap.add_argument("--arm", default="all", choices=["all", "cover", "plain", "both"],
                    help="'cover' or 'plain' runs only that device-resident arm "
                         "(for profiling one step), 'both' the two in turn (one line "
                         "each); 'all' is the benchmark")
    ap.add_argument("--intersect", default="hash", choices=["hash", "merge"],
                    help="with --arm: the owner-grouped hash intersection (the product "
                         "path) or the warp merge / binary-search kernels (Sec. V-A's other "
                         "two techniques), same graph, same result")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-runs", type=int, default=1,
                    help="runs of the all-core oracle in the default line (median)")
    ap.add_argument("--ref-sample-div", type=int, default=16,
                    help="reference arm: each step counts 1/this of the cover edges")
    ap.add_argument("--shard", dest="shard", action="store_true", default=None,
                    help="count one graph with all ranks (edge-range shards, strong "
                         "scaling); the default under torchrun")
    ap.add_argument("--no-shard", dest="shard", action="store_false",
                    help="under torchrun: every rank counts its own graph (weak scaling)")
    ap.add_argument("--no-batch", action="store_true",
                    help="default workload: skip the batch object")
    ap.add_argument("--no-serve", action="store_true",
                    help="default workload: skip the serve object")
    return ap.parse_args()


# ---------------------------------------------------------------- workload

def make_graph(workload: str, rank: int):
    import graphgen as gg
    if workload == "rmat22":
        seed = 2 + rank * 1000
        g = gg.rmat(22, 16, seed, relabel_seed=seed + 2**32)
        desc = ("R-MAT scale 22, edgefactor 16, a/b/c/d=.57/.19/.19/.05, edge seed %d, "
                "relabel stream %d+2^32, symmetrised, deduplicated" % (seed, seed))
    elif workload == "rmat26":
        seed = 5 + rank * 1000
        g = gg.rmat(26, 16, seed, relabel_seed=seed + 2**32)
        desc = ("R-MAT scale 26, edgefactor 16, a/b/c/d=.57/.19/.19/.05, edge seed %d, "
                "relabel stream %d+2^32, symmetrised, deduplicated" % (seed, seed))
    elif workload in ("rmat18", "rmat20"):
        sc = int(workload[4:])
        g = gg.rmat(sc, 16, 2 + rank * 1000, relabel_seed=2 + rank * 1000 + 2**32)
        desc = f"R-MAT scale {sc}, edgefactor 16, relabelled"
    elif workload == "rmat10":
        g = gg.rmat(10, 16, 1 + rank * 1000)
        desc = "R-MAT scale 10, edgefactor 16, seed 1"
    elif workload == "chunglu23":
        g = gg.chung_lu_islands(1 << 23, seed=7 + rank * 1000)
        desc = ("Chung-Lu n=2^23, gamma 2.1, mean degree 32, cap 65536, "
                "10% Erdos-Renyi islands of 16-256 vertices, seed 7")
    else:
        raise ValueError(f"{workload} is not a single-graph workload")
    return g, desc


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.path = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def gpu_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ---------------------------------------------------------------- roofline

def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if
    the kernel source has not changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))[kernel]
    except Exception:
        return None
    src = hashlib.sha256(open(INTERSECT_SOURCE, "rb").read()).hexdigest()[:16]
    if d.get("source_sha256_16") != src:
        return None
    return d


# ---------------------------------------------------------------- CPU oracle

def oracle_sample(g, target_s: float, seed: int = 0):
    """Time the CPU oracle on a bounded sample: BFS levels and cover-edge
    extraction over the whole graph, the count-once intersection on a
    uniform random sample of cover edges; the intersection time is scaled by
    |H| / sample.  Returns (estimated full seconds, description)."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    L, _ = oracle.bfs_levels(g)
    t1 = time.perf_counter()
    H = oracle.cover_edges(g, L)
    t2 = time.perf_counter()
    rng = np.random.default_rng(seed)
    h = len(H)
    if h == 0:
        return t2 - t0, "BFS + cover on the full graph (no cover edges)"
    probe = H[rng.choice(h, size=min(h, 2000), replace=False)]
    tp0 = time.perf_counter()
    oracle.cetc_edge_counts(g, L, probe)
    per_edge = (time.perf_counter() - tp0) / len(probe)
    budget = max(0.5, target_s - (t2 - t0))
    k = int(min(h, max(len(probe), budget / max(per_edge, 1e-9))))
    idx = rng.choice(h, size=k, replace=False)
    ts0 = time.perf_counter()
    oracle.cetc_edge_counts(g, L, H[idx])
    ts = time.perf_counter() - ts0
    est = (t1 - t0) + (t2 - t1) + ts * h / k
    desc = (f"oracle BFS ({t1 - t0:.2f} s) and cover extraction ({t2 - t1:.2f} s) on the full "
            f"graph; count-once intersection on a uniform random sample of {k} of {h} cover "
            f"edges ({ts:.2f} s), scaled by |H|/sample; single thread")
    return est, desc


def cpu_info():
    """Host core count and CPU model name (lscpu's "Model name", which names
    Arm cores too, else /proc/cpuinfo's)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"host_cores": os.cpu_count(), "cpu": model or "unknown"}


def oracle_full_all_cores(g, runs: int = 1):
    """The CPU oracle's Alg. 1 on the whole graph, measured in full: BFS
    levels and the cover-edge pass (single-threaded, as the oracle does
    them) and the count-once intersection over every cover edge with its
    outer loop shared among all host cores (OpenMP).  Median of `runs`
    runs.  Returns (seconds, T, description)."""
    import oracle
    times, T, parts = [], None, None
    threads = os.cpu_count() or 1
    for _ in range(max(1, runs)):
        t0 = time.perf_counter()
        L, _ = oracle.bfs_levels(g)
        t1 = time.perf_counter()
        nh = oracle.num_cover(g, L)
        t2 = time.perf_counter()
        T = oracle.cetc_count_mt(g, L, threads)
        t3 = time.perf_counter()
        times.append(t3 - t0)
        parts = (t1 - t0, t2 - t1, t3 - t2, nh)
    t = statistics.median(times)
    desc = (f"oracle Alg. 1 on the whole graph, measured in full (median of {len(times)} "
            f"run(s)): BFS {parts[0]:.2f} s and cover-edge pass {parts[1]:.2f} s on one "
            f"thread, count-once intersection of all {parts[3]} cover edges {parts[2]:.2f} s "
            f"on {threads} threads (OpenMP)")
    return t, T, desc


# ---------------------------------------------------------------- arms

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def reduce_max(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_graph_sample(gs, target_s: float, seed: int = 0):
    """Time the CPU oracle (Alg. 1: BFS, cover edges, count) graph by graph
    on a uniform random sample of the list gs, for about target_s seconds.
    Returns (edges per second, description)."""
    import random
    import oracle
    order = list(range(len(gs)))
    random.Random(seed).shuffle(order)
    edges, t0 = 0, time.perf_counter()
    done = 0
    for i in order:
        oracle.cetc(gs[i])
        edges += gs[i].num_edges
        done += 1
        if time.perf_counter() - t0 > target_s:
            break
    dt = time.perf_counter() - t0
    return edges / dt, (f"oracle BFS + cover edges + count-once intersection, one graph at a "
                        f"time, on {done} of {len(gs)} graphs drawn uniformly ({dt:.2f} s); "
                        f"single thread")


def golden_large():
    """Oracle results for the benchmark-size graphs, written by
    tests/golden/make_golden_large.py (which calls only the oracle)."""
    try:
        return json.load(open(os.path.join(ROOT, "tests", "golden", "large_counts.json")))
    except Exception:
        return {}


GOLDEN_NAME = {"rmat22": "rmat_s22", "rmat26": "rmat_s26", "chunglu23": "chung_lu_2_23"}


def single_graph_config(g, desc, num_cover, nlevels, max_degree, triangles, world):
    """The `config` object of a single-graph workload (the same keys and
    values in both arms)."""
    csr_bytes = 8 * (g.n + 1) + 4 * g.nnz
    return {"workload": desc, "n": g.n, "num_edges": g.num_edges, "nnz": g.nnz,
            "generated_edges": g.generated_edges, "num_cover": int(num_cover),
            "k_cover_fraction": int(num_cover) / max(g.num_edges, 1),
            "nlevels": int(nlevels), "max_degree": int(max_degree),
            "triangles": None if triangles is None else int(triangles),
            "parallelism": f"independent graphs x{world}",
            "l2": f"inputs larger than L2 (CSR {csr_bytes / 1e9:.2f} GB > 129 MB)"}


def oracle_counts_threads(g, L, uv, threads):
    """Per-edge Alg. 1 counts of the edge list uv, split among host threads
    (each thread runs the oracle's single-threaded per-edge function on its
    share; ctypes releases the interpreter lock during the call)."""
    import numpy as np
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    parts = np.array_split(np.arange(len(uv)), threads * 8)
    with ThreadPoolExecutor(threads) as ex:
        outs = list(ex.map(lambda ix: oracle.cetc_edge_counts(g, L, uv[ix]), parts))
    return np.concatenate(outs) if outs else np.zeros(0, dtype=np.uint32)


def run_reference(args, world, rank):
    """The oracle as the reference arm, on this arm's workload, config,
    metric and unit.  Each step is a bounded sample of the workload and
    ms_per_step is the time the steps actually took."""
    if rank != 0:
        return
    import numpy as np
    threads = os.cpu_count() or 1
    if args.workload in ("batch", "serve"):
        # one step = the oracle counting a fixed-size random sample of the
        # workload's graphs, one graph per host thread; value = the sample's
        # edges / the step's time
        import graphgen as gg
        import oracle
        from concurrent.futures import ThreadPoolExecutor
        seed = 3 if args.workload == "batch" else 11
        specs = gg.mixed_graph_specs(4096, seed=seed)
        rng = np.random.default_rng(seed)
        per_step = 128
        times, edges = [], []
        with ThreadPoolExecutor(threads) as ex:
            for i in range(args.warmup + args.steps):
                pick = rng.choice(len(specs), size=per_step, replace=False)
                gs = list(ex.map(gg.graph_from_spec, [specs[k] for k in pick]))
                t0 = time.perf_counter()
                list(ex.map(oracle.cetc, gs))
                dt = time.perf_counter() - t0
                if i >= args.warmup:
                    times.append(dt)
                    edges.append(sum(g.num_edges for g in gs))
        value = sum(edges) / sum(times)
        sample = (f"each step: the oracle's Alg. 1 (BFS, cover edges, count) on {per_step} "
                  f"graphs drawn at random from the 4,096-graph recipe (seed {seed}), one graph "
                  f"per host thread ({threads} threads); value = sampled edges / time")
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": BATCH_DESC if args.workload == "batch" else
                       serve_desc(args)},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": threads,
                             "kind": "oracle", "sample": sample, **cpu_info()},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    import oracle
    g, desc = make_graph(args.workload, 0)
    # setup (untimed): the cover edges to draw each step's sample from
    L0, nl = oracle.bfs_levels(g)
    H = oracle.cover_edges(g, L0)
    h = len(H)
    frac = 1.0 / max(1, args.ref_sample_div)
    k = max(1, min(h, int(h * frac)))
    rng = np.random.default_rng(0)
    steps, rates = [], []
    for i in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(h, size=k, replace=False)) if h else np.zeros(0, dtype=np.int64)
        t0 = time.perf_counter()
        L, _ = oracle.bfs_levels(g)
        t1 = time.perf_counter()
        oracle.num_cover(g, L)
        t2 = time.perf_counter()
        if k and h:
            oracle_counts_threads(g, L, H[idx], threads)
        t3 = time.perf_counter()
        if i >= args.warmup:
            steps.append(t3 - t0)
            est = (t1 - t0) + (t2 - t1) + (t3 - t2) * h / max(k, 1)
            rates.append(g.num_edges / est)
    value = statistics.mean(rates)
    gold = golden_large().get(GOLDEN_NAME.get(args.workload, ""), {})
    sample = (f"each step: the oracle's BFS and cover-edge pass over the whole graph (one "
              f"thread) and its count-once intersection of a uniform random 1/"
              f"{args.ref_sample_div} of the {h} cover edges ({k} edges, {threads} threads); "
              f"value = |E| / (BFS + cover pass + intersection time x {h}/{k}), an estimate "
              f"of the full pipeline; ms_per_step = the time each step took")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": single_graph_config(g, desc, h, nl, g.degrees().max(), gold.get("T"), world),
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": threads, "kind": "oracle",
                         "sample": sample, **cpu_info()},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2210_00389_gb300 as tc

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    g, desc = make_graph(args.workload, rank)
    stream = torch.cuda.current_stream(dev)
    off_d = torch.from_numpy(g.offsets).to(dev)
    cols_d = torch.from_numpy(g.cols).to(dev)
    off_h = torch.from_numpy(g.offsets).pin_memory()
    cols_h = torch.from_numpy(g.cols).pin_memory()
    torch.cuda.synchronize()

    def step(mode, host=False):
        if host:
            h = tc.tc_graph_create(off_h, cols_h, g.n, tc.TC_GRAPH_VALIDATE, stream)
        else:
            h = tc.tc_graph_create(off_d, cols_d, g.n,
                                   tc.TC_GRAPH_BORROW | tc.TC_GRAPH_VALIDATE, stream)
        T = tc.tc_count(h, mode)
        st = tc.tc_graph_stats(h)
        info = tc.tc_graph_info(h)
        tc.tc_graph_destroy(h)
        return T, st, info

    def timed(mode, host=False):
        for _ in range(args.warmup):
            step(mode, host)
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = tc.tc_kernel_launches()
        e0.record(stream)
        res = [step(mode, host) for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = e0.elapsed_time(e1) / args.steps
        return ms, res, tc.tc_kernel_launches() - l0

    if args.arm != "all":
        for arm in (("cover", "plain") if args.arm == "both" else (args.arm,)):
            mode = tc.TC_MODE_COVER if arm == "cover" else tc.TC_MODE_PLAIN
            if args.intersect == "merge":
                mode |= tc.TC_INTERSECT_MERGE
            ms, res, launches = timed(mode)
            if rank == 0:
                print(json.dumps({"arm": arm, "intersect": args.intersect, "ms_per_step": ms,
                                  "triangles": res[0][0], "stats": res[0][1],
                                  "gpu_launches": launches, "workload": desc}), flush=True)
        return

    sampler = ClockSampler(gpu_uuid(torch, dev))
    sampler.start()
    ms_cover, res_cover, launches = timed(tc.TC_MODE_COVER)
    clocks = sampler.stop()
    T = res_cover[0][0]
    assert all(r[0] == T for r in res_cover), "count changed between steps"
    ms_plain, res_plain, _ = timed(tc.TC_MODE_PLAIN)
    assert all(r[0] == T for r in res_plain), "plain count differs from cover count"
    ms_e2e, res_e2e, _ = timed(tc.TC_MODE_COVER, host=True)
    assert all(r[0] == T for r in res_e2e)

    ms_cover_max = reduce_max(ms_cover, world, dev)
    ms_plain_max = reduce_max(ms_plain, world, dev)
    ms_e2e_max = reduce_max(ms_e2e, world, dev)
    units = reduce_sum(float(g.num_edges), world, dev)
    value = units / (ms_cover_max / 1e3)

    # roofline of the dominant kernel (the cover hash intersection).
    # Algorithmic bytes per launch: 4 B per probe-list element it must read
    # (counted by the kernel) plus 72 B of per-edge metadata (task index,
    # H entry, two offset pairs, segment descriptor, H offset).
    st0, info0 = res_cover[0][1], res_cover[0][2]
    ms_k = statistics.mean(r[1]["ms_main_kernel"] for r in res_cover)
    nh = info0["num_cover"]
    alg_bytes = float(4 * st0["list_elems"] + 72 * nh)
    with tc.Graph(off_d, cols_d, g.n, tc.TC_GRAPH_BORROW, stream) as G:
        H = G.cover_edges()
    deg = g.degrees()
    u = H[:, 0].astype(np.int64)
    v = H[:, 1].astype(np.int64)
    merge_bytes = float((4 * deg[u] + 4 * deg[v] + 16).sum() + 8 * len(H))
    del H, u, v
    peak, peak_kind = measured_hbm_peak()
    achieved = alg_bytes / (ms_k / 1e3) / 1e9
    stp = res_plain[0][1]
    ms_kp = statistics.mean(r[1]["ms_main_kernel"] for r in res_plain)
    plain_bytes = float(4 * stp["list_elems"] + 72 * g.num_edges)
    # the committed DRAM captures are per workload (R-MAT scale 22 and 26)
    tr = ncu_traffic("k_hash_intersect<cover>" +
                     ("" if args.workload == "rmat22" else "|" + args.workload))
    stages = {k: statistics.mean(r[1][k] for r in res_cover)
              for k in ("ms_bfs", "ms_cover", "ms_bucket", "ms_intersect", "ms_main_kernel", "ms_total")}
    stages_plain = {"ms_intersect": ms_kp,
                    "intersect_GBps": plain_bytes / (ms_kp / 1e3) / 1e9,
                    "list_elems": stp["list_elems"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_or, T_or, sdesc = oracle_full_all_cores(g, args.cpu_runs)
        assert T_or == T, f"oracle T {T_or} != GPU T {T}"
        cpu = {"value": g.num_edges / t_or, "unit": "edges/s", "cores": os.cpu_count(),
               "kind": "oracle", "sample": sdesc, "seconds": t_or, "equals_gpu_count": True,
               **cpu_info()}

    csr_bytes = 8 * (g.n + 1) + 4 * g.nnz
    dram_frac = None
    if tr:
        dram_gbs = tr["bytes_per_launch"] / (ms_k / 1e3) / 1e9
        dram_frac = dram_gbs / peak
    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_cover_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": single_graph_config(g, desc, info0["num_cover"], info0["nlevels"],
                                      info0["max_degree"], T, world),
        "stages_ms": stages,
        "plain": {"value": units / (ms_plain_max / 1e3), "unit": "edges/s",
                  "ms_per_step": ms_plain_max, "stages_ms": stages_plain,
                  "cover_speedup_vs_plain": ms_plain_max / ms_cover_max},
        "e2e": {"value": units / (ms_e2e_max / 1e3), "unit": "edges/s",
                "ms_per_step": ms_e2e_max, "h2d_bytes_per_step": csr_bytes,
                "d2h_bytes_per_step": 8},
        # achieved: the kernel's algorithmic bytes (4 per looked-up element
        # + 72 per edge) over its CUDA-event time; dram_frac: the ncu DRAM
        # bytes of the same launches (when the capture is of this source)
        # over the same time; merge_equivalent: the bytes a merge of both
        # full lists per edge would stream (an effective figure, not a bound)
        "roofline": {"bound": "hbm", "kernel": "k_hash_intersect<cover>", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "frac_of_8tbs_nominal": achieved / 8000.0,
                     "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms": ms_k,
                     "list_elems": st0["list_elems"],
                     "traffic": tr["bytes_per_launch"] if tr else None,
                     "traffic_source": tr.get("source") if tr else None,
                     "dram_frac": dram_frac,
                     "merge_equivalent_bytes": merge_bytes,
                     "merge_equivalent_GBps": merge_bytes / (ms_k / 1e3) / 1e9},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if args.workload == "rmat22" and world == 1:
        # the batched and serving configurations of the same metric, measured
        # in the same run on the same GPU
        del off_d, cols_d, off_h, cols_h
        torch.cuda.empty_cache()
        if not args.no_batch:
            b = measure_batch(args, world, rank, local)
            line["batch"] = {"workload": b["config"]["workload"],
                             "ms_per_call": b["ms_per_step"], "value": b["value"],
                             "unit": "edges/s", "graphs": b["config"]["graphs"],
                             "looped_plain_ms": b["looped_plain"]["ms_per_step"],
                             "speedup_vs_looped_plain": b["looped_plain"]["batched_speedup"],
                             "e2e": b["e2e"], "gpu_launches": b["gpu_launches"],
                             "options": b["config"]["options"]}
        if not args.no_serve:
            sv = measure_serve(args, world, rank, local)
            line["serve"] = {"workload": sv["config"]["workload"], **sv["serve"],
                             "offered_req_per_s": sv["config"]["offered_req_per_s"],
                             "value": sv["value"], "unit": "edges/s",
                             "fifo_plain": sv["fifo_plain"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


BATCH_DESC = ("mixed batch of 4096 graphs (R-MAT s6-14 ef8-32 / ER n256-4096 p=10/(n-1) / "
              "K20-K200, seed 3), one batched launch")


def serve_desc(args):
    return (f"serving: resident R-MAT scale {args.serve_scale} + Poisson stream of "
            f"{args.requests} requests at {args.rate:g} req/s (seed 11)")


def run_batch(args, world, rank, local):
    line = measure_batch(args, world, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_batch(args, world, rank, local):
    """The mixed small-graph batch (4,096 graphs: R-MAT scale 6-14 with
    edgefactor 8-32, Erdos-Renyi G(n, 10/(n-1)) with n in 256-4096, complete
    graphs K_20..K_200; seed 3): one batched cover-edge launch per step
    against the plain count looped graph by graph."""
    import numpy as np
    import torch
    import graphgen as gg
    import paper_2210_00389_gb300 as tc

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    specs = gg.mixed_graph_specs(4096, seed=3 + rank * 1000)
    gs = [gg.graph_from_spec(s) for s in specs]
    units = float(sum(g.num_edges for g in gs))
    dviews = [(torch.from_numpy(g.offsets).to(dev), torch.from_numpy(g.cols).to(dev)) for g in gs]
    hviews = [(g.offsets, g.cols) for g in gs]
    stream = torch.cuda.current_stream(dev)
    opt = tc.autotuned_options()
    torch.cuda.synchronize()

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = tc.tc_kernel_launches()
        e0.record(stream)
        outs = [fn() for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return e0.elapsed_time(e1) / steps, outs, tc.tc_kernel_launches() - l0

    def batched():
        c, s = tc.tc_count_batch(dviews, tc.TC_MODE_COVER, opt, stream)
        assert (s == tc.TC_OK).all()
        return c

    def looped_plain():
        out = np.zeros(len(gs), dtype=np.uint64)
        for i, (o, c) in enumerate(dviews):
            h = tc.tc_graph_create(o, c, None, tc.TC_GRAPH_BORROW | tc.TC_GRAPH_VALIDATE, stream)
            out[i] = tc.tc_count(h, tc.TC_MODE_PLAIN)
            tc.tc_graph_destroy(h)
        return out

    def batched_host():
        c, s = tc.tc_count_batch(hviews, tc.TC_MODE_COVER, opt, stream)
        return c

    ms_b, outs_b, launches = timed(batched, args.steps)
    ms_l, outs_l, _ = timed(looped_plain, max(1, min(args.steps, 2)))
    assert (outs_b[0] == outs_l[0]).all(), "batched cover counts differ from looped plain counts"
    ms_e, _, _ = timed(batched_host, args.steps)
    ms_b = reduce_max(ms_b, world, dev)
    ms_l = reduce_max(ms_l, world, dev)
    ms_e = reduce_max(ms_e, world, dev)
    units = reduce_sum(units, world, dev)
    h2d = sum(8 * (g.n + 1) + 4 * g.nnz for g in gs)
    line = {
        "metric": METRIC, "value": units / (ms_b / 1e3), "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": BATCH_DESC,
                   "graphs": len(gs), "num_edges": int(units), "triangles": int(outs_b[0].sum()),
                   "options": ({"block_threads": opt.block_threads,
                                "blocks_per_sm": opt.blocks_per_sm, "skew": opt.skew,
                                "tiny_max_nnz": opt.tiny_max_nnz, "source": "autotune.json"}
                               if opt else "built-in")},
        "looped_plain": {"value": units / (ms_l / 1e3), "unit": "edges/s", "ms_per_step": ms_l,
                         "batched_speedup": ms_l / ms_b},
        "e2e": {"value": units / (ms_e / 1e3), "unit": "edges/s", "ms_per_step": ms_e,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 12 * len(gs)},
        "gpu_launches": launches,
    }
    return line


def run_serve(args, world, rank, local):
    line = measure_serve(args, world, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_serve(args, world, rank, local):
    """Serving: a resident R-MAT scale 26 graph (relabel seed 5) and an
    open-loop Poisson stream of requests (seed 11) drawn like the mixed
    batch with 5% R-MAT scale 18-22; latency = scheduled arrival -> poll sees
    the result.  Compared with one-at-a-time FIFO plain counting of the same
    stream.  Request graphs come from a seeded pool (every distinct small
    spec of the first 2,000, and 2 graphs per large scale), generated before
    timing."""
    import random
    import threading

    import numpy as np
    import torch
    import graphgen as gg
    import paper_2210_00389_gb300 as tc

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nreq, rate = args.requests, args.rate
    rng = random.Random(11)
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    threads = os.cpu_count() or 4
    big = gg.rmat(args.serve_scale, 16, 5, relabel_seed=5 + 2**32)
    small_specs = gg.mixed_graph_specs(2000, seed=11)
    large_specs = gg.serve_large_specs()
    with ThreadPoolExecutor(threads) as ex:
        pool_small = list(ex.map(gg.graph_from_spec, small_specs))
        pool_large = list(ex.map(gg.graph_from_spec, large_specs))
    # request mix: request 0 is the resident graph; then 5% large, the rest
    # drawn from the small pool (which already has the 84/10/1 mix)
    reqs = [("resident", None)]
    for _ in range(nreq - 1):
        if rng.random() < 0.05:
            reqs.append(("large", rng.randrange(len(pool_large))))
        else:
            reqs.append(("small", rng.randrange(len(pool_small))))
    t_arr = np.cumsum([0.0] + [rng.expovariate(rate) for _ in range(nreq - 1)])

    def graph_of(kind, i):
        return big if kind == "resident" else (pool_large[i] if kind == "large" else pool_small[i])

    # expected counts: every distinct graph counted alone on the GPU, and
    # the oracle's counts (small graphs: counted here, one graph per host
    # thread; large ones and the resident graph: the oracle-written golden
    # file, when it holds them)
    alone = {}
    for kind, pool in (("small", pool_small), ("large", pool_large)):
        for i, g in enumerate(pool):
            with tc.Graph(g.offsets, g.cols) as G:
                alone[(kind, i)] = G.count(tc.TC_MODE_COVER)
    with ThreadPoolExecutor(threads) as ex:
        oracle_small = list(ex.map(lambda g: oracle.cetc(g)["T"], pool_small))
    gold = golden_large()
    oracle_T = {("small", i): t for i, t in enumerate(oracle_small)}
    for i, sp in enumerate(large_specs):
        e = gold.get("serve_rmat_s{scale}_seed{seed}".format(**sp))
        if e and e["nnz"] == pool_large[i].nnz:
            oracle_T[("large", i)] = e["T"]
    e = gold.get(f"rmat_s{args.serve_scale}")
    if e and e["nnz"] == big.nnz:
        oracle_T[("resident", None)] = e["T"]
    units = [graph_of(k, i).num_edges for k, i in reqs]

    # ---- served, continuous batching
    # the request pools outlive the run, so the server borrows their arrays
    # instead of copying each one on the submitting thread
    s = tc.tc_serve_create(150 << 30, slots=64, queue_capacity=1 << 16, wait_limit_ms=600000,
                           borrow_views=True)
    gid = tc.tc_serve_register(s, big.offsets, big.cols)
    done_at = [None] * nreq
    result = [None] * nreq
    tickets = [None] * nreq
    submit_lag = [0.0] * nreq  # submission time - scheduled arrival
    lock = threading.Lock()
    finished = threading.Event()

    new_items = []  # submitted indices not yet seen by the poller

    def poller():
        pending, ndone = [], 0
        while ndone < nreq:
            with lock:
                pending.extend(new_items)
                new_items.clear()
            still = []
            for i in pending:
                d, c, st = tc.tc_serve_poll(s, tickets[i])
                if d:
                    done_at[i] = time.perf_counter()
                    result[i] = (c, st)
                    ndone += 1
                else:
                    still.append(i)
            pending = still
            time.sleep(0.0002)
        finished.set()

    th = threading.Thread(target=poller, daemon=True)
    t0 = time.perf_counter()
    th.start()
    for i, (kind, j) in enumerate(reqs):
        wait = t0 + t_arr[i] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        if kind == "resident":
            t = tc.tc_serve_submit(s, None, gid, tc.TC_MODE_COVER)
        else:
            g = graph_of(kind, j)
            t = tc.tc_serve_submit(s, (g.offsets, g.cols), 0, tc.TC_MODE_COVER)
        submit_lag[i] = time.perf_counter() - (t0 + t_arr[i])
        with lock:
            tickets[i] = t
            new_items.append(i)
    finished.wait(timeout=1800)
    t_end = time.perf_counter()
    tc.tc_serve_destroy(s)
    lat = np.array([done_at[i] - (t0 + t_arr[i]) for i in range(nreq)]) * 1e3
    resident_T = result[0][0]
    ok = all(result[i][1] == tc.TC_OK for i in range(nreq))
    same = all(result[i][0] == (resident_T if reqs[i][0] == "resident" else alone[reqs[i]])
               for i in range(nreq))
    checked = [i for i in range(nreq) if reqs[i] in oracle_T]
    equals_oracle = all(result[i][0] == oracle_T[reqs[i]] for i in checked)

    # ---- baseline: one at a time, FIFO, plain count
    base_done = [0.0] * nreq
    with tc.Graph(torch.from_numpy(big.offsets).to(dev), torch.from_numpy(big.cols).to(dev)) as B:
        b0 = time.perf_counter()
        for i, (kind, j) in enumerate(reqs):
            wait = b0 + t_arr[i] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            if kind == "resident":
                c = B.count(tc.TC_MODE_PLAIN)
            else:
                g = graph_of(kind, j)
                with tc.Graph(g.offsets, g.cols) as G:
                    c = G.count(tc.TC_MODE_PLAIN)
            assert c == (resident_T if kind == "resident" else alone[(kind, j)])
            base_done[i] = time.perf_counter()
        b_end = time.perf_counter()
    blat = np.array([base_done[i] - (b0 + t_arr[i]) for i in range(nreq)]) * 1e3

    def pct(a, q):
        return float(np.percentile(a, q))

    line = {
        "metric": METRIC, "value": sum(units) / (t_end - t0), "unit": "edges/s",
        "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": (t_end - t0) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": serve_desc(args),
                   "requests": nreq, "offered_req_per_s": rate,
                   "resident_edges": big.num_edges, "resident_triangles": resident_T},
        "serve": {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "max_ms": float(lat.max()),
                  "achieved_req_per_s": nreq / (t_end - t0), "all_ok": ok,
                  "each_equals_alone": same, "equals_oracle": equals_oracle,
                  "oracle_checked_requests": len(checked),
                  "submit_lag_ms": {"p50": pct(np.array(submit_lag) * 1e3, 50),
                                    "max": float(max(submit_lag)) * 1e3},
                  "small_p50_ms": pct(lat[[k for k in range(nreq) if reqs[k][0] == "small"]], 50),
                  "small_p99_ms": pct(lat[[k for k in range(nreq) if reqs[k][0] == "small"]], 99),
                  "large_p50_ms": pct(lat[[k for k in range(nreq) if reqs[k][0] == "large"]], 50)},
        "fifo_plain": {"p50_ms": pct(blat, 50), "p99_ms": pct(blat, 99),
                       "achieved_req_per_s": nreq / (b_end - b0),
                       "value": sum(units) / (b_end - b0)},
    }
    return line


def run_kstudy(args, world, rank):
    """The cover-edge fraction k = |H| / |E| of R-MAT graphs against the scale
    on the GPU, with the max-degree root rule and with one uniformly random
    root (the rest rooted at their lowest id), next to the paper's fit
    k = 1.1773 e^(-0.036 scale) (Sec. IV-A), and the Comm-CETC communication
    model (Sec. III-B) evaluated with the measured k and levels against the
    wedge-checking volume from the exact wedge count, for p = 128.  One JSON
    line; not a benchmark metric."""
    import random

    import numpy as np
    import torch

    import graphgen as gg
    import paper_2210_00389_gb300 as tc
    from paper_2210_00389_gb300 import comm

    if rank != 0:
        return
    dev = torch.device("cuda", 0)
    rows = []
    for scale in range(6, args.kstudy_max_scale + 1):
        g = gg.rmat(scale, 16, seed=scale, relabel_seed=scale + 2 ** 32)
        off = torch.from_numpy(g.offsets).to(dev)
        cols = torch.from_numpy(g.cols).to(dev)
        deg = np.diff(g.offsets)
        with tc.Graph(off, cols, n=g.n, flags=tc.TC_GRAPH_BORROW) as G:
            _, nl = G.levels()
            h_max = G.cover_edge_count()
            r = random.Random(scale).choice(np.flatnonzero(deg > 0).tolist())
            _, nl_r = G.levels([r])
            h_rand = G.cover_edge_count()
        m = g.num_edges
        wedges = int((deg.astype(np.int64) * (deg.astype(np.int64) - 1) // 2).sum())
        log_d = comm.clog2(max(nl, 2))
        ours = comm.comm_cetc_bits(g.n, m, h_max / m, 128, log_d) / 8
        prev = comm.wedge_check_bits(wedges, g.n) / 8
        # Comm-CETC's volume counted on 128 virtual processors (the BFS's
        # cut edge traversals, the cover-edge exchange, the reduction)
        meas = comm.measured_volume(g.offsets, g.cols, h_max, nl, 128)
        rows.append({"scale": scale, "n": g.n, "edges": m, "levels": nl,
                     "k_max_degree_root": h_max / m, "k_random_root": h_rand / m,
                     "levels_random_root": nl_r, "k_fit": comm.k_fit(scale),
                     "wedges": wedges, "comm_cetc_bytes_p128": ours,
                     "comm_cetc_measured_bytes_p128": meas["measured_bits"] / 8,
                     "bfs_cut_fraction_p128": meas["cut_directed_traversals"] / max(g.nnz, 1),
                     "wedge_check_bytes": prev, "reduction_p128": prev / ours})
        del off, cols
    print(json.dumps({"study": "cover-edge fraction k vs R-MAT scale (edgefactor 16, "
                               "relabelled, seed = scale)",
                      "fit": "k = 1.1773 exp(-0.036 scale)", "rows": rows}), flush=True)


def shard_steps(make_graph_obj, mode, steps, warmup, rank, world, all_reduce, sync, clock):
    """The sharded step loop: every step builds the rank's graph object
    (levels and cover edges are computed inside it, the same on every rank),
    takes its work-balanced slice (tc_shard_bounds), counts it
    (tc_count_range) and sums the slice counts with one all-reduce.  Returns
    (per-step seconds of the timed steps, the totals).  `sync()` is a
    barrier plus a device synchronisation; `clock()` a host timer."""
    from paper_2210_00389_gb300.shard import count_sharded

    def one():
        with make_graph_obj() as G:
            return count_sharded(G, mode, rank, world, all_reduce)[1]

    for _ in range(warmup):
        one()
    sync()
    t0 = clock()
    totals = [one() for _ in range(steps)]
    sync()
    return (clock() - t0) / max(steps, 1), totals


def run_shard(args, world, rank, local):
    """One graph counted by all ranks (strong scaling): edge-range shards of
    the cover edges, one int64 all-reduce per step (NCCL)."""
    import torch
    import torch.distributed as dist
    import paper_2210_00389_gb300 as tc
    from paper_2210_00389_gb300.shard import torch_all_reduce_sum

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    g, desc = make_graph(args.workload, 0)  # the same graph on every rank
    off_d = torch.from_numpy(g.offsets).to(dev)
    cols_d = torch.from_numpy(g.cols).to(dev)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()

    def sync():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    launches0 = tc.tc_kernel_launches()
    sec, totals = shard_steps(
        lambda: tc.Graph(off_d, cols_d, g.n, tc.TC_GRAPH_BORROW | tc.TC_GRAPH_VALIDATE, stream),
        tc.TC_MODE_COVER, args.steps, args.warmup, rank, world, torch_all_reduce_sum(dev),
        sync, time.perf_counter)
    launches = tc.tc_kernel_launches() - launches0
    assert len(set(totals)) == 1
    sec = reduce_max(sec, world, dev)
    line = {
        "metric": METRIC, "value": g.num_edges / sec, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": desc, "n": g.n, "num_edges": g.num_edges, "nnz": g.nnz,
                   "triangles": int(totals[0]),
                   "parallelism": f"edge-range shards of H x{world}, one int64 all-reduce",
                   "timing": "host clock around the steps, barrier + device sync on both sides"},
        "gpu_launches": launches,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_init()
    shard = args.shard if args.shard is not None else (world > 1)
    if args.impl == "ours" and shard and args.workload in ("rmat22", "rmat26", "chunglu23",
                                                           "rmat18", "rmat20"):
        run_shard(args, world, rank, local)
    elif args.workload == "serve" and args.impl == "ours":
        run_serve(args, world, rank, local)
    elif args.workload == "batch" and args.impl == "ours":
        run_batch(args, world, rank, local)
    elif args.workload == "kstudy":
        run_kstudy(args, world, rank)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
