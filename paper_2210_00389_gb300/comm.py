"""Communication model of Comm-CETC (Alg. 2) and the paper's size fits.

Closed forms from Sec. III and IV of Bader et al., "Triangle Counting Through
Cover-Edges" (analytic, host-side; nothing here runs on the GPU):

* total communication of Comm-CETC on p processors, in bits: the BFS moves
  ceil(log D) + 3 ceil(log n) bits per edge traversal (level, vertex pair,
  degree), the exchange of the k m cover edges moves p ceil(log n) bits per
  edge, the final reduction (p - 1) ceil(log n) bits (Sec. III-B);
* the wedge-checking baseline moves 2 ceil(log n) bits per wedge (Sec. IV-A);
* the exponential fit of the cover-edge fraction k for Graph500 R-MAT graphs
  against the scale, and the triangle-count fit against n (Sec. IV-A).

Units follow the paper: 1 TB = 2^40, 1 PB = 2^50, 1 EB = 2^60 bytes.
"""
from __future__ import annotations

import math

TB, PB, EB = 2 ** 40, 2 ** 50, 2 ** 60


def clog2(x: float) -> int:
    """ceil(log2 x) for x >= 1."""
    return max(0, math.ceil(math.log2(x)))


def comm_cetc_bits(n: int, m: int, k: float, p: int, log_d: int) -> float:
    """Total communication of Comm-CETC in bits:
    m (ceil(log D) + (k p + 3) ceil(log n)) + (p - 1) ceil(log n)."""
    ln = clog2(n)
    return m * (log_d + (k * p + 3) * ln) + (p - 1) * ln


def wedge_check_bits(wedges: float, n: int) -> float:
    """Wedge-checking baseline: 2 ceil(log n) bits per wedge."""
    return wedges * 2 * clog2(n)


def k_fit(scale: float) -> float:
    """Cover-edge fraction of Graph500 R-MAT graphs: 1.1773 e^(-0.036 scale)."""
    return 1.1773 * math.exp(-0.036 * scale)


def triangles_fit(n: float) -> float:
    """Triangles of Graph500 R-MAT graphs: 77.422 n^1.125."""
    return 77.422 * n ** 1.125


def wedges_exact(degrees) -> int:
    """Sum over vertices of C(d, 2): the wedges a wedge-checking algorithm
    generates on the undirected graph."""
    return int(sum(int(d) * (int(d) - 1) // 2 for d in degrees))


def rmat_row(scale: int, k: float, p: int, wedges: float, log_d: int = 4) -> dict:
    """One R-MAT row of the paper's communication table: n = 2^scale,
    m = 16 n, the given k, p and wedge count; volumes in bytes."""
    n = 2 ** scale
    m = 16 * n
    ours = comm_cetc_bits(n, m, k, p, log_d) / 8
    prev = wedge_check_bits(wedges, n) / 8
    return {"scale": scale, "n": n, "m": m, "k": k, "p": p, "previous_bytes": prev,
            "this_bytes": ours, "reduction": prev / ours}


def vertex_partition(offsets, p: int):
    """Sec. III's 1-D partition: contiguous vertex ranges with about 2m/p
    edge endpoints each.  Returns p + 1 vertex bounds."""
    import numpy as np
    off = np.asarray(offsets, dtype=np.int64)
    n = off.size - 1
    nnz = int(off[-1])
    targets = (np.arange(1, p, dtype=np.int64) * nnz) // p
    cuts = np.searchsorted(off[1:], targets, side="left") + 1
    return np.concatenate([[0], np.minimum(cuts, n), [n]]).astype(np.int64)


def measured_volume(offsets, cols, num_cover: int, nlevels: int, p: int) -> dict:
    """Comm-CETC's communication counted on p virtual processors of one
    graph (host-side, from the CSR, the measured |H| and the number of BFS
    levels), next to the model:

    * BFS: a level-synchronous BFS expands every vertex once and sends one
      message (level, vertex pair, degree: ceil(log D) + 3 ceil(log n) bits)
      per directed edge traversal whose endpoints sit on different
      processors; the model charges all m edge traversals as remote;
    * cover-edge exchange: each processor's partial set S_i goes to each of
      the p - 1 others in the XOR rounds of Alg. 2, at ceil(log n) bits per
      edge as in the model (which charges p transfers per edge);
    * reduction: (p - 1) ceil(log n) bits.

    D is taken as the number of BFS levels (an upper bound on the depth, at
    most diameter + 1).  Volumes in bits."""
    import numpy as np
    off = np.asarray(offsets, dtype=np.int64)
    n = off.size - 1
    nnz = int(off[-1])
    m = nnz // 2
    ln, ld = clog2(max(n, 2)), clog2(max(nlevels, 2))
    bounds = vertex_partition(off, p)
    part_of = np.repeat(np.arange(p, dtype=np.int64), np.diff(bounds))
    deg = np.diff(off)
    row_part = np.repeat(part_of, deg)
    col_part = part_of[np.asarray(cols, dtype=np.int64)]
    cut_directed = int(np.count_nonzero(row_part != col_part))
    bfs = cut_directed * (ld + 3 * ln)
    exchange = num_cover * (p - 1) * ln
    reduce_ = (p - 1) * ln
    k = num_cover / max(m, 1)
    model = comm_cetc_bits(n, m, k, p, ld)
    return {"p": p, "n": n, "m": m, "k": k, "cut_directed_traversals": cut_directed,
            "bfs_bits": bfs, "exchange_bits": exchange, "reduce_bits": reduce_,
            "measured_bits": bfs + exchange + reduce_, "model_bits": model,
            "model_bfs_bits": m * (ld + 3 * ln), "model_exchange_bits": k * m * p * ln}
