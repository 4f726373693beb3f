"""Whole trees at the benchmark's full sizes, checked node by node against
the oracle (tests/tree_check.py): every node's samples, counts and children by
routing the root samples with the oracle's projection arithmetic, and a
spread of nodes (root, each depth band, random internal nodes, searched
leaves) re-searched by the oracle from its own projection sampler; then the
tree's predictions for 50,000 rows against the oracle's traversal.

* forest_2m: n=2M, d=256 lognormal features, 8-sparse median-centred labels
  with 10% flips, bootstrap root, 128 projections/node, T=1024, with the
  row-major feature copy -- tree 0 of the forest the benchmark times;
* wide_counts: n=500k, d=4096, 90% zeros, zero-truncated Poisson(3)
  nonzeros, 5 classes, 128 projections/node with 1+Poisson(3) nonzeros
  (cap 16), T=1024, grown to purity;
* trunk: n=1M, p=1024 Trunk Gaussians, 48 projections/node of 1+Poisson(1)
  nonzeros, T=1024, grown to purity.
"""
import numpy as np
import pytest

from oracle import so_oracle as O
from paper_2603_00326_b300 import datagen as G
from tests import gpu_util as U
from tests.tree_check import choose_nodes, route_and_sample

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2603_00326_b300 import soforest
    soforest.lib()
    return soforest


def _grow_and_check(S, ds_np, root, p, seed, tree_id, n_internal, row_major=False):
    ds = U.upload_dataset(ds_np.X, ds_np.y, ds_np.n_classes)
    if row_major:
        ds = ds.with_row_major()
    tp = S.tree_params(p["n_proj"], p["lam"], p["cap"], p["n_bins"], p["sort_below"], False, seed, tree_id, -1)
    gt = S.so_train_tree(ds, U.i32(root), tp)
    # inference with the full-size tree on a sample of rows
    rows = np.sort(np.random.default_rng(tree_id + 7).choice(ds_np.n, size=50000, replace=False)).astype(np.int32)
    pred, _ = S.so_predict(ds.X, S.upload_forest([gt], ds_np.n_classes))
    np.testing.assert_array_equal(pred.cpu().numpy()[rows], O.predict_tree_c(gt, ds_np.X, rows))
    del ds, pred
    U.torch_cuda().cuda.empty_cache()
    ids = choose_nodes(gt, n_internal=n_internal, n_leaves=6, seed=tree_id + 1)
    n = route_and_sample(gt, ds_np.X, ds_np.y, ds_np.n_classes, root, n_proj=p["n_proj"], lam=p["lam"],
                         cap=p["cap"], n_bins=p["n_bins"], sort_below=p["sort_below"], seed=seed,
                         tree_id=tree_id, check_ids=ids)
    assert n >= min(len(ids), 8)
    return gt


def test_forest_2m_tree_full_size(S):
    from paper_2603_00326_b300 import forest as F
    ds_np = G.forest_2m()
    p = G.WORKLOAD_PARAMS["forest_2m"]
    cfg = F.ForestConfig(n_trees=p["n_trees"], n_proj=p["n_proj"], lam=p["lam"], cap=p["cap"],
                         sort_below=p["sort_below"])
    root = F.root_indices(ds_np.n, 0, cfg)
    gt = _grow_and_check(S, ds_np, root, p, cfg.seed, 0, n_internal=16, row_major=True)
    assert set(np.unique(gt.path)) >= {0, 1}


def test_wide_counts_tree_full_size(S):
    ds_np = G.wide_counts()
    p = G.WORKLOAD_PARAMS["wide_counts"]
    root = G.all_indices(ds_np.n)
    gt = _grow_and_check(S, ds_np, root, p, G.PROJ_SEED_BASE + 4, 0, n_internal=16)
    assert set(np.unique(gt.path)) >= {0, 1}


def test_trunk_1m_tree_full_size(S):
    ds_np = G.trunk(n=1_000_000, p=1024)
    p = G.WORKLOAD_PARAMS["trunk"]
    root = G.all_indices(ds_np.n)
    gt = _grow_and_check(S, ds_np, root, p, G.PROJ_SEED_BASE + 5, 0, n_internal=12, row_major=True)
    assert set(np.unique(gt.path)) >= {0, 1}
