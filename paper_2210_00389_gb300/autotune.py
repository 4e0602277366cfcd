"""Autotuner of the batched kernel (tc_count_batch).

Sweeps, on a sample of the mixed small-graph workload (R-MAT scale 6-14,
Erdos-Renyi, complete graphs): the size threshold between the persistent
per-graph kernel and the disjoint-union path (tiny_max_nnz), the per-graph
kernel's block shape (threads per block, resident blocks per SM) and its
merge / binary-search switch ratio (skew).  Every setting must give the same
counts; the fastest is written to ``autotune.json`` next to this file, and
the Python binding passes it to ``tc_count_batch`` when the caller gives no
options.

Run on the GPU: ``python paper_2210_00389_gb300/autotune.py [--graphs 2048]``.
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

TABLE = os.path.join(HERE, "autotune.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=2048)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()

    import torch

    import graphgen as gg
    import paper_2210_00389_gb300 as tc

    specs = gg.mixed_graph_specs(4096, seed=3)[:args.graphs]
    gs = [gg.graph_from_spec(s) for s in specs]
    dev = [(torch.from_numpy(g.offsets).cuda(), torch.from_numpy(g.cols).cuda()) for g in gs]
    torch.cuda.synchronize()
    results = []
    ref = None

    def run(threads, per_sm, skew, tiny):
        nonlocal ref
        opt = tc.Options(threads, per_sm, skew, tiny)
        counts, status = tc.tc_count_batch(dev, tc.TC_MODE_COVER, opt)  # warm-up
        if ref is None:
            ref = counts.copy()
        assert (status == tc.TC_OK).all() and (counts == ref).all(), (threads, per_sm, skew, tiny)
        best = float("inf")
        for _ in range(args.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tc.tc_count_batch(dev, tc.TC_MODE_COVER, opt)
            best = min(best, time.perf_counter() - t0)
        results.append({"block_threads": threads, "blocks_per_sm": per_sm, "skew": skew,
                        "tiny_max_nnz": tiny, "seconds": best})
        print(json.dumps(results[-1]), flush=True)
        return best

    # block shape and split threshold at the default skew, then the skew
    for threads, per_sm, tiny in itertools.product((128, 256, 512), (1, 2, 4, 8),
                                                   (1 << 11, 1 << 13, 1 << 15, 1 << 17)):
        if threads * per_sm <= 2048:
            run(threads, per_sm, 24, tiny)
    b = min(results, key=lambda r: r["seconds"])
    for skew in (8, 64):
        run(b["block_threads"], b["blocks_per_sm"], skew, b["tiny_max_nnz"])
    win = min(results, key=lambda r: r["seconds"])
    table = {"batch": {k: win[k] for k in ("block_threads", "blocks_per_sm", "skew",
                                           "tiny_max_nnz")},
             "sample": f"first {args.graphs} graphs of the mixed recipe (seed 3), cover mode",
             "sweep": results}
    with open(TABLE, "w") as f:
        json.dump(table, f, indent=1)
        f.write("\n")
    print("best", json.dumps(table["batch"]))


if __name__ == "__main__":
    main()
