"""The multi-GPU driver's host logic (paper_2210_00389_gb300.shard) with
world_size 2 and 3 gloo ranks on CPU.  The device calls are replaced by a
test double backed by the oracle: per-cover-edge counts of Alg. 1 summed
over each rank's slice.  Also: a rank that dies before the all-reduce makes
the others fail with an error instead of waiting forever."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleGraph:
    """shard_bounds / count_range over the oracle's per-edge counts."""

    def __init__(self, per_edge):
        self.per = np.asarray(per_edge, dtype=np.int64)

    def shard_bounds(self, mode, nshards):
        m = len(self.per)
        return [m * k // nshards for k in range(nshards + 1)]

    def count_range(self, mode, begin, end):
        return int(self.per[begin:end].sum())

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


def _graph():
    import graphgen as gg
    import oracle
    g = gg.rmat(10, 16, seed=13, relabel_seed=14)
    L, _ = oracle.bfs_levels(g, None)
    H = oracle.cover_edges(g, L)
    return oracle.cetc_edge_counts(g, L, H), oracle.cetc_count(g, L)


def _worker(rank, world, port, q, die_rank):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from paper_2210_00389_gb300.shard import count_sharded, torch_all_reduce_sum
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    per, T = _graph()
    try:
        if rank == die_rank:
            q.put((rank, "died", None, T))
            q.close()
            q.join_thread()  # the message is sent before the process ends
            os._exit(3)  # leaves between steps: nothing of it is in flight
        local, total = count_sharded(OracleGraph(per), 0, rank, world, torch_all_reduce_sum())
        q.put((rank, "ok", local, total == T))
    except Exception as e:  # noqa: BLE001 -- reported to the parent
        q.put((rank, "error", type(e).__name__, str(e)[:200]))
    finally:
        if rank != die_rank:
            try:
                dist.destroy_process_group()
            except Exception:
                pass


def _run(world, die_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, die_rank)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return sorted(out)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sum_equals_total(world):
    out = _run(world)
    assert [o[1] for o in out] == ["ok"] * world
    assert all(o[3] for o in out)          # every rank sees the total T
    per, T = _graph()
    assert sum(o[2] for o in out) == T     # the slices partition H


def test_dead_rank_is_reported():
    out = _run(2, die_rank=1)
    assert out[1][1] == "died"
    assert out[0][1] == "error"            # rank 0's all-reduce failed, no hang


def _bench_worker(rank, world, port, q):
    """bench.py's sharded step loop (the default under torchrun) on gloo
    ranks, with the oracle-backed graph object in place of the device."""
    import sys
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2210_00389_gb300.shard import torch_all_reduce_sum
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    per, T = _graph()
    try:
        sec, totals = bench.shard_steps(lambda: OracleGraph(per), 0, 3, 2, rank, world,
                                        torch_all_reduce_sum(), dist.barrier, time.perf_counter)
        q.put((rank, "ok", sec >= 0, totals == [T] * 3))
    except Exception as e:  # noqa: BLE001 -- reported to the parent
        q.put((rank, "error", type(e).__name__, str(e)[:200]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_bench_shard_mode(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert [o[1] for o in out] == ["ok"] * world, out
    assert all(o[2] and o[3] for o in out)
