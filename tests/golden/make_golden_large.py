"""Write tests/golden/large_counts.json: the CPU oracle's results on the
benchmark-size graphs (R-MAT scale 22, Chung-Lu 2^23, R-MAT scale 26 and the
serving stream's ten large R-MAT requests).

Calls only the oracle and the input generators: levels by the oracle's BFS
(Def. 2 / Alg. 1 with the max-degree root rule), |H| by its horizontal pass
(Thm. 1), T by its all-core Alg. 1 loop and again by its all-core plain
edge iterator (Sec. I, V-A), which must agree.  Scale 26 takes tens of
minutes on a few cores.  Run from the repo root:
    python tests/golden/make_golden_large.py [name ...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "large_counts.json")


def graphs():
    yield "rmat_s22", gg.rmat_s22
    yield "chung_lu_2_23", gg.chung_lu_2_23
    for sp in gg.serve_large_specs():
        name = "serve_rmat_s{scale}_seed{seed}".format(**sp)
        yield name, (lambda sp=sp: gg.graph_from_spec(sp))
    yield "rmat_s26", gg.rmat_s26


def main(names):
    gold = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name, make in graphs():
        if names and name not in names:
            continue
        t0 = time.time()
        g = make()
        L, nl = oracle.bfs_levels(g)
        nh = oracle.num_cover(g, L)
        T = oracle.cetc_count_mt(g, L)
        P = oracle.plain_count_mt(g)
        assert T == P, (name, T, P)
        gold[name] = {"n": g.n, "nnz": g.nnz, "num_edges": g.num_edges, "num_cover": int(nh),
                      "nlevels": nl, "T": T,
                      "level_histogram": np.bincount(L).tolist()}
        print(name, gold[name]["T"], f"{time.time() - t0:.0f} s", flush=True)
        with open(OUT, "w") as f:
            json.dump(gold, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
