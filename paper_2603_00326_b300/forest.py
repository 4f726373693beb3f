"""Forests of sparse-oblique trees on one or more GPUs.

Trees are independent (the paper trains them on a pool of worker threads,
Section 4): tree t of a forest is trained by rank t mod world_size, each rank
on its own GPU with the data replicated, and the finished tree arrays are
gathered on rank 0 at the end -- the only exchange, so no collective touches
the data path.  Each tree grows to purity from a bootstrap of the n samples
(drawn by the input generator, so the root sample list is an input of the
tree call) through so_train_tree.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, List, Optional

import numpy as np

from . import datagen as G
from . import soforest as S


@dataclasses.dataclass
class ForestConfig:
    n_trees: int
    n_proj: int
    lam: float
    cap: int
    n_bins: int = 256
    sort_below: int = 1024
    hist_only: bool = False
    seed: int = G.PROJ_SEED_BASE + 3
    bootstrap: bool = True
    max_depth: int = -1
    bin_rule: int = 0  # 0 equal-width bins, 1 random-width bins (node keys of each tree)
    criterion: int = 0  # 0 Gini decrease, 1 information gain


def trees_of_rank(n_trees: int, rank: int, world: int) -> List[int]:
    """Tree ids trained by `rank`: t with t mod world == rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return list(range(rank, n_trees, world))


def root_indices(n: int, tree_id: int, cfg: ForestConfig) -> np.ndarray:
    return G.bootstrap_indices(n, tree_id, seed=cfg.seed) if cfg.bootstrap else G.all_indices(n)


def _gpu_trainer(ds: "S.DeviceDataset", cfg: ForestConfig):
    import torch

    def train(tree_id: int) -> S.Tree:
        root = torch.from_numpy(root_indices(ds.X.shape[1], tree_id, cfg)).to(ds.X.device)
        tp = S.tree_params(cfg.n_proj, cfg.lam, cfg.cap, cfg.n_bins, cfg.sort_below, cfg.hist_only, cfg.seed,
                           tree_id, cfg.max_depth, bin_rule=cfg.bin_rule, criterion=cfg.criterion)
        return S.so_train_tree(ds, root, tp)

    return train


def train_forest(cfg: ForestConfig, ds: Optional["S.DeviceDataset"] = None, rank: int = 0, world: int = 1,
                 trainer: Optional[Callable[[int], object]] = None, gather: bool = True):
    """Trains this rank's share of the forest.

    Returns (trees, seconds): with gather=True and world > 1 (torch.distributed
    initialised), rank 0 receives every tree in tree-id order and the other
    ranks receive []; otherwise each rank returns its own trees (id order).
    `trainer(tree_id)` defaults to so_train_tree on `ds`.
    """
    if trainer is None:
        if ds is None:
            raise ValueError("a device dataset or a trainer is required")
        trainer = _gpu_trainer(ds, cfg)
    mine = trees_of_rank(cfg.n_trees, rank, world)
    t0 = time.perf_counter()
    own = [(t, trainer(t)) for t in mine]
    secs = time.perf_counter() - t0
    if not gather or world == 1:
        return [tr for _, tr in own], secs
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, own)
    if rank != 0:
        return [], secs
    allt = sorted((t, tr) for part in parts for (t, tr) in part)
    if [t for t, _ in allt] != list(range(cfg.n_trees)):
        raise RuntimeError("gathered tree ids do not cover the forest")
    return [tr for _, tr in allt], secs
