"""Forest prediction in the oracle (CPU): two independent traversals agree,
a tree grown to purity on continuous data classifies its own training samples
perfectly, and vote ties go to the lowest class."""
import copy

import numpy as np

from oracle import so_oracle as O
from paper_2603_00326_b300 import datagen as G


def _tree():
    ds = G.tree_small(n=1200, d=10, seed=81)
    root = G.all_indices(ds.n)
    t = O.train_tree(ds.X, ds.y, 2, root, n_proj=8, lam=1.5, cap=8, n_bins=64, sort_below=150, seed=3)
    return ds, root, t


def test_python_and_c_traversals_agree():
    ds, root, t = _tree()
    rng = np.random.default_rng(0)
    Xq = rng.standard_normal((ds.d, 300)).astype(np.float32)
    rows = np.arange(300, dtype=np.int32)
    np.testing.assert_array_equal(O.predict_tree(t, Xq, rows), O.predict_tree_c(t, Xq, rows))
    np.testing.assert_array_equal(O.predict_tree(t, ds.X, root[:200]), O.predict_tree_c(t, ds.X, root[:200]))


def test_pure_tree_fits_its_training_samples():
    ds, root, t = _tree()
    leaves = t.left < 0
    assert np.all(np.count_nonzero(t.class_counts[leaves], axis=1) == 1)  # every leaf pure
    pred = O.predict_tree_c(t, ds.X, root)
    np.testing.assert_array_equal(pred, ds.y[root])


def test_vote_ties_go_to_the_lowest_class():
    ds, root, t = _tree()
    a = copy.deepcopy(t)
    b = copy.deepcopy(t)
    a.leaf_class[:] = 1
    b.leaf_class[:] = 0
    pred, votes = O.predict_forest([a, b], ds.X, root[:50], 2)
    assert np.all(votes == 1) and np.all(pred == 0)
    pred, votes = O.predict_forest([a, a, b], ds.X, root[:50], 2)
    assert np.all(pred == 1) and np.all(votes[:, 1] == 2)
