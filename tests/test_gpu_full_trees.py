"""Whole trees at the benchmark's full sizes, identical to the oracle's.

The oracle grows the same tree on every host core (orc_train_tree_mt, pinned
to the single-threaded grower in tests/test_oracle_tree_mt.py) and the GPU
tree must equal it field by field, bit for bit: every node's projection,
candidate, path, threshold, FP64 gain, sample and class counts, children,
depth and leaf class.  The tree's predictions for 50,000 rows are checked
against the oracle's traversal too.

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

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2603_00326_b300 import soforest
    soforest.lib()
    return soforest


def _grow_and_check(S, ds_np, root, p, seed, tree_id, row_major=False):
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
    ot = U.oracle_tree_all_cores(ds_np.X, ds_np.y, ds_np.n_classes, root, n_proj=p["n_proj"], lam=p["lam"],
                                 cap=p["cap"], n_bins=p["n_bins"], sort_below=p["sort_below"], seed=seed,
                                 tree_id=tree_id)
    U.assert_tree_equal(gt, ot)
    return gt


def test_forest_2m_tree_full_size(S):
    from paper_2603_00326_b300 import forest as F
    ds_np = G.forest_2m()
    p = G.WORKLOAD_PARAMS["forest_2m"]
    cfg = F.ForestConfig(n_trees=p["n_trees"], n_proj=p["n_proj"], lam=p["lam"], cap=p["cap"],
                         sort_below=p["sort_below"])
    root = F.root_indices(ds_np.n, 0, cfg)
    gt = _grow_and_check(S, ds_np, root, p, cfg.seed, 0, row_major=True)
    assert set(np.unique(gt.path)) >= {0, 1}


def test_wide_counts_tree_full_size(S):
    ds_np = G.wide_counts()
    p = G.WORKLOAD_PARAMS["wide_counts"]
    root = G.all_indices(ds_np.n)
    gt = _grow_and_check(S, ds_np, root, p, G.PROJ_SEED_BASE + 4, 0)
    assert set(np.unique(gt.path)) >= {0, 1}


def test_trunk_1m_tree_full_size(S):
    ds_np = G.trunk(n=1_000_000, p=1024)
    p = G.WORKLOAD_PARAMS["trunk"]
    root = G.all_indices(ds_np.n)
    gt = _grow_and_check(S, ds_np, root, p, G.PROJ_SEED_BASE + 5, 0, row_major=True)
    assert set(np.unique(gt.path)) >= {0, 1}
