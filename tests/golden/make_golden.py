"""Write the stored expected values under tests/golden/ from the CPU oracle.

Calls only the oracle and the input generators.  Run from the repo root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    g = gg.rmat_s10()
    r = oracle.cetc(g)
    gold = {
        "workload": "R-MAT scale 10, edgefactor 16, a/b/c/d=.57/.19/.19/.05, seed 1, no relabel",
        "n": g.n, "nnz": g.nnz, "num_edges": g.num_edges,
        "T": r["T"], "num_cover": int(len(r["H"])), "nlevels": r["nlevels"],
        "level_histogram": np.bincount(r["levels"]).tolist(),
        "plain_T": oracle.plain_count(g),
    }
    with open(os.path.join(HERE, "rmat_s10.json"), "w") as f:
        json.dump(gold, f, indent=1)
        f.write("\n")
    print(gold)


if __name__ == "__main__":
    main()
