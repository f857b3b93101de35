"""Multi-rank logic of bench.py on CPU (gloo, world size 2): every rank runs its
own replica; the reported time is the maximum over ranks, and only rank 0
prints.  No GPU and no data-path collective are involved."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    out[rank] = (ws, r, bench.max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (2, 0, 15.0)
    assert out[1] == (2, 1, 15.0)


def test_max_over_ranks_without_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5


# ----------------------------------------------------------------------------
# independent instances sharded over ranks (no exchange)
# ----------------------------------------------------------------------------

def _c5(count=64):
    import sys
    sys.path.insert(0, ROOT)
    from paper_2303_03026_gb300 import workloads as wl
    return wl.c5_instances(count=count, nmin=32, nmax=160, precision="fp64")


def test_partition_covers_and_balances():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2303_03026_gb300 import shard
    W = _c5()
    cells = shard.instance_cells(W)
    assert sum(cells) == W.interior_cells()
    for n in (1, 2, 3, 4, 8):
        parts = shard.partition_instances(cells, n)
        flat = sorted(q for p in parts for q in p)
        assert flat == list(range(len(cells)))          # every instance exactly once
        loads = [sum(cells[q] for q in p) for p in parts]
        # greedy largest-first: no rank exceeds the mean by more than one instance
        assert max(loads) <= sum(cells) / n + max(cells)
        assert all(p for p in parts)
    assert shard.partition_instances(cells, 1) == [list(range(len(cells)))]


def test_instance_subset_keeps_each_instance():
    import sys
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_2303_03026_gb300 import shard
    W = _c5(16)
    parts = shard.partition_instances(shard.instance_cells(W), 3)
    total = 0
    for p in parts:
        S = shard.instance_subset(W, p)
        total += S.interior_cells()
        for new_q, q in enumerate(p):
            a = W.block_meta[:, 0] == q
            b = S.block_meta[:, 0] == new_q
            assert np.array_equal(W.block_meta[a, 1:], S.block_meta[b, 1:])
            assert np.array_equal(W.U[:, a], S.U[:, b])
            assert S.instances[new_q] is W.instances[q]
    assert total == W.interior_cells()


def _shard_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2303_03026_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    W = _c5(32)
    parts = shard.partition_instances(shard.instance_cells(W), world)
    mine = shard.instance_subset(W, parts[rank])
    seen = [None] * world
    dist.all_gather_object(seen, (parts, mine.interior_cells()))
    out[rank] = seen
    dist.barrier()
    dist.destroy_process_group()


def test_ranks_agree_on_the_partition_gloo_world2():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_shard_worker, args=(2, port, out), nprocs=2, join=True)
    seen0, seen1 = out[0], out[1]
    assert seen0 == seen1                                 # same view on both ranks
    assert seen0[0][0] == seen0[1][0]                      # computed independently, equal
    assert seen0[0][1] + seen0[1][1] == _c5(32).interior_cells()


def _empty_shard_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2303_03026_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    W = _c5(1)
    # the check runs on every rank before the process group exists: no rank
    # is left waiting in a collective for one that failed
    try:
        shard.check_ranks(len(W.instances), world)
        out[rank] = "accepted"
    except ValueError as e:
        out[rank] = "refused: " + str(e)
        return
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    dist.destroy_process_group()


def test_more_ranks_than_instances_refused_on_every_rank_gloo_world2():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_empty_shard_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0].startswith("refused") and out[1].startswith("refused")
    import sys
    sys.path.insert(0, ROOT)
    from paper_2303_03026_gb300 import shard
    with pytest.raises(ValueError):
        shard.partition_instances([100], 2)
    assert shard.partition_instances([100, 50], 2) == [[0], [1]]
