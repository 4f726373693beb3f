"""Multi-rank forest host logic on CPU (gloo, world size 2).

Trees shard by id (t mod world) with no data-path collective; the only
exchange is the final gather of tree arrays on rank 0.  The trainer is a
host stand-in that returns a deterministic record per tree id, so the test
needs no GPU.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2603_00326_b300 import forest as F


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fake_tree(t):
    return {"tree_id": t, "n_nodes": 2 * t + 1}


def _worker(rank, world, port, n_trees, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg = F.ForestConfig(n_trees=n_trees, n_proj=8, lam=1.5, cap=8)
        seen = []

        def trainer(t):
            seen.append(t)
            return _fake_tree(t)

        trees, _ = F.train_forest(cfg, rank=rank, world=world, trainer=trainer)
        q.put((rank, seen, trees))
    finally:
        dist.destroy_process_group()


def test_tree_assignment_is_a_partition():
    for n_trees in (0, 1, 7, 128):
        for world in (1, 2, 3, 8):
            got = sorted(t for r in range(world) for t in F.trees_of_rank(n_trees, r, world))
            assert got == list(range(n_trees))
    with pytest.raises(ValueError):
        F.trees_of_rank(4, 2, 2)


@pytest.mark.parametrize("n_trees", [5, 8])
def test_two_rank_forest_gather(n_trees):
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_trees, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = {}
    for _ in range(world):
        rank, seen, trees = q.get(timeout=120)
        results[rank] = (seen, trees)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results[0][0] == list(range(0, n_trees, 2))
    assert results[1][0] == list(range(1, n_trees, 2))
    assert results[1][1] == []
    assert results[0][1] == [_fake_tree(t) for t in range(n_trees)]


def test_single_rank_bootstrap_roots_are_inputs():
    cfg = F.ForestConfig(n_trees=3, n_proj=8, lam=1.5, cap=8)
    a = F.root_indices(1000, 1, cfg)
    b = F.root_indices(1000, 1, cfg)
    c = F.root_indices(1000, 2, cfg)
    assert (a == b).all() and not (a == c).all()
    assert a.shape == (1000,) and (a[:-1] <= a[1:]).all() and a.min() >= 0 and a.max() < 1000
